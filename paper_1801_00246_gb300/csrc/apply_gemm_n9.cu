// FP32 SIPDG apply as register-blocked GEMMs, degree N = 9.
// (Eq. ellipticOp3 as two dense products per element tile; see apply_gemm.cuh.)
#define GA_N 9
#define GA_NS ga9
#include "apply_gemm.cuh"

namespace dgx {
cudaError_t launch_apply_f32_n9(const dg_mesh* m, int B, double lambda, const float* u, float* Au, float2* face,
                                cudaStream_t st) {
  return ga9::launch(m, B, lambda, u, Au, face, st);
}
}  // namespace dgx
