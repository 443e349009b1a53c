// Pipeline instantiation for the fp32 form.
#include "pipeline.cuh"

namespace fire {

int run_fp32(const Plan& pl, const CallArgs& a) {
  int rc = set_smem_limits<float, float>();
  if (rc) return rc;
  Runner<float, float, float> rn(pl, a);
  return pl.dm.op == FIRE_OP_GRAD_LOGPSI ? rn.run_grad() : rn.run();
}

}  // namespace fire
