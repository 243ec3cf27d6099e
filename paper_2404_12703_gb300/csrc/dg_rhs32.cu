// dg_rhs32.cu -- FP32-bulk instantiation of the stage kernels (dg_stage.cuh):
// flux, volume and surface arithmetic in FP32 on shifted primitives; the
// state, RK register, metrics and the final combination stay in FP64.
#include "dg_stage.cuh"

namespace dg {

cudaError_t init_kernel_attributes_fp32(int N) {
  DG_DISPATCH(N, return (stage_set_attrs<NN, float>()));
  return cudaSuccess;
}

cudaError_t launch_rhs_fp32(dg_ctx* c, const double* U, int mode, double rkA, double rkB, int first) {
  DG_DISPATCH(c->N, return (stage_launch<NN, float>(c, U, mode, rkA, rkB, first)));
  return cudaSuccess;
}

}  // namespace dg
