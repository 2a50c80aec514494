// placeholder: replaced by the tcgen05 implementation
#include "common.h"
namespace dmrg2d {
int tc_prepare(dmrg2d_ops* ops, cudaStream_t) { ops->tc_ok = 0; return DMRG2D_OK; }
void tc_release(dmrg2d_ops*) {}
int launch_hv_tc(const dmrg2d_ops*, const void*, float*, int, cudaStream_t) {
  return set_error(DMRG2D_EUNSUPPORTED, "tensor-core path not built");
}
}
