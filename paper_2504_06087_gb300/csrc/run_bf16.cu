// Pipeline instantiation for the BF16_FP64 form: float32 activations,
// float64 LU / slogdet and final reduction.
#include "pipeline.cuh"

namespace fire {

int run_bf16(const Plan& pl, const CallArgs& a) {
  int rc = set_smem_limits<float, double>();
  if (rc) return rc;
  Runner<float, double, double> rn(pl, a);
  // the gradient of the BF16_FP64 form runs in fp32 (FP64 LU); so do the
  // Metropolis moves of the FP32 form (FP64 refresh)
  if (pl.dm.op == FIRE_OP_MCMC) return rn.run_mcmc();
  return pl.dm.op == FIRE_OP_GRAD_LOGPSI ? rn.run_grad() : rn.run();
}

}  // namespace fire
