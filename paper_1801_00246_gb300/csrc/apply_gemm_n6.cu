// FP32 SIPDG apply as register-blocked GEMMs, degree N = 6.
// (Eq. ellipticOp3 as two dense products per element tile; see apply_gemm.cuh.)
#define GA_N 6
#define GA_NS ga6
#include "apply_gemm.cuh"

namespace dgx {
cudaError_t launch_apply_f32_n6(const dg_mesh* m, int B, double lambda, const float* u, float* Au, float2* face,
                                cudaStream_t st) {
  return ga6::launch(m, B, lambda, u, Au, face, st);
}
}  // namespace dgx
