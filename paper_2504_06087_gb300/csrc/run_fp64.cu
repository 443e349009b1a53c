// Pipeline instantiation for the fp64 form.
#include "pipeline.cuh"

namespace fire {

int run_fp64(const Plan& pl, const CallArgs& a) {
  int rc = set_smem_limits<double, double>();
  if (rc) return rc;
  Runner<double, double, double> rn(pl, a);
  if (pl.dm.op == FIRE_OP_MCMC) return rn.run_mcmc();
  return pl.dm.op == FIRE_OP_GRAD_LOGPSI ? rn.run_grad() : rn.run();
}

}  // namespace fire
