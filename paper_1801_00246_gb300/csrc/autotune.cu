// Per-mesh choice of the apply kernel.
//
// Several kernels evaluate the same operator (tile, FP32 GEMM, tensor-core
// FP64, element per thread); which one is fastest depends on the degree, the
// precision, the batch and the mesh size. dg_autotune times every valid
// candidate on the mesh itself (random input, L2 flushed before every timed
// launch, best of three) and keeps the fastest in the mesh's kernel table,
// which launch_apply (and through it every solve) consults. The paper has no
// counterpart: it tunes its kernels per degree by hand (Section 5.2).
#include <cmath>
#include <cstring>

#include "dg_internal.h"

namespace dgx {
namespace {

// U(-1, 1) from a 64-bit mix of (seed, index): only a timing input
__global__ void k_fill_uniform(int64_t n, uint64_t seed, double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * uint64_t(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double v = double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    a[i] = v;
    b[i] = float(v);
  }
}

constexpr int kCandidates[] = {DG_KERNEL_TILE, DG_KERNEL_GEMM, DG_KERNEL_TENSOR, DG_KERNEL_EPT, DG_KERNEL_TENSOR_PIPE,
                               DG_KERNEL_TC05, DG_KERNEL_TC64};

struct Scratch {
  void* p[5] = {};
  ~Scratch() {
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

}  // namespace
}  // namespace dgx

using namespace dgx;

extern "C" {

dg_status dg_set_apply_kernel(dg_mesh* m, int degree, dg_prec prec, int helmholtz, int kernel) {
  if (!m) { set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (degree < 1 || degree > kMaxN) { set_error("degree must be in 1..10"); return DG_ERR_ARG; }
  if (prec != DG_F64 && prec != DG_F32) { set_error("precision must be DG_F64 or DG_F32"); return DG_ERR_ARG; }
  if (kernel != DG_KERNEL_AUTO && !kernel_valid(kernel, degree, prec == DG_F64)) {
    set_error("kernel not available for this degree and precision");
    return DG_ERR_ARG;
  }
  m->kern[degree][prec == DG_F32 ? 1 : 0][helmholtz ? 1 : 0] = int8_t(kernel);
  ++m->kern_gen;
  return DG_OK;
}

dg_status dg_wait_selftest(double seconds, void* stream) {
  if (!(seconds > 0.0) || seconds > 10.0) {
    set_error("dg_wait_selftest: seconds must be in (0, 10]");
    return DG_ERR_ARG;
  }
  int* flag = nullptr;
  int host = -1;
  cudaError_t e = cudaMalloc(&flag, sizeof(int));
  if (e == cudaSuccess) e = launch_wait_selftest(seconds, flag, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  cudaFree(flag);
  if (e != cudaSuccess) {
    set_error(std::string("dg_wait_selftest: ") + cudaGetErrorString(e));
    return DG_ERR_CUDA;
  }
  if (host == 1) {
    set_error("dg_wait_selftest: the bounded wait gave up as designed");
    return DG_ERR_TIMEOUT;
  }
  return DG_OK;
}

int dg_tensor_timeouts(void) {
  int flag = 0, flag05 = 0, flag64 = 0;
  if (tensor_pipe_error(&flag) != cudaSuccess || tc05_error(&flag05) != cudaSuccess ||
      tc64_error(&flag64) != cudaSuccess)
    return -1;
  return flag + flag05 + flag64;
}

int dg_get_apply_kernel(const dg_mesh* m, int degree, dg_prec prec, int helmholtz) {
  if (!m || degree < 1 || degree > kMaxN || (prec != DG_F64 && prec != DG_F32)) return -1;
  const int k = m->kern[degree][prec == DG_F32 ? 1 : 0][helmholtz ? 1 : 0];
  return k == DG_KERNEL_AUTO ? default_kernel(degree, prec == DG_F64) : k;
}

dg_status dg_autotune(dg_mesh* m, int B, double lambda, int degree_lo, int degree_hi, float* times, void* stream) {
  if (!m) { set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (B < 1 || B > DG_MAX_BATCH) { set_error("batch must be in 1..64"); return DG_ERR_ARG; }
  if (degree_lo < 1 || degree_hi > kMaxN || degree_lo > degree_hi) {
    set_error("need 1 <= degree_lo <= degree_hi <= 10");
    return DG_ERR_ARG;
  }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  if (times) std::memset(times, 0, sizeof(float) * (kMaxN + 1) * 2 * 2 * DG_NUM_KERNELS);
  cudaStream_t st = (cudaStream_t)stream;
  auto fail = [](cudaError_t e) {
    set_error(std::string("dg_autotune: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
  };
  try {
    const int64_t n = int64_t(B) * m->K * ((degree_hi + 1) * (degree_hi + 2) / 2);
    const size_t flush_bytes = size_t(256) << 20;  // larger than L2
    Scratch s;
    cudaError_t e = cudaSuccess;
    for (int d = degree_lo; d <= degree_hi && e == cudaSuccess; ++d) e = ensure_ops(m, d);
    if (e == cudaSuccess) e = cudaMalloc(&s.p[0], n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s.p[1], n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s.p[2], n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s.p[3], n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&s.p[4], flush_bytes);
    if (e != cudaSuccess) return fail(e);
    k_fill_uniform<<<1024, 256, 0, st>>>(n, 12345, static_cast<double*>(s.p[0]), static_cast<float*>(s.p[2]));
    note_launch();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int d = degree_lo; d <= degree_hi && e == cudaSuccess; ++d)
      for (int p = 0; p < 2 && e == cudaSuccess; ++p)
        for (int h = 0; h < (lambda > 0 ? 2 : 1) && e == cudaSuccess; ++h) {
          const bool f64 = p == 0;
          const double lam = h ? lambda : 0.0;
          const void* u = f64 ? s.p[0] : s.p[2];
          void* out = f64 ? s.p[1] : s.p[3];
          const int8_t before = m->kern[d][p][h];
          int best = DG_KERNEL_AUTO;
          float best_ms = 1e30f;
          for (int k : kCandidates) {
            if (!kernel_valid(k, d, f64)) continue;
            m->kern[d][p][h] = int8_t(k);
            e = launch_apply(m, d, f64 ? DG_F64 : DG_F32, B, lam, u, out, st);  // warm: lazy set-up
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
              e = cudaMemsetAsync(s.p[4], rep, flush_bytes, st);
              if (e == cudaSuccess) e = cudaEventRecord(e0, st);
              if (e == cudaSuccess) e = launch_apply(m, d, f64 ? DG_F64 : DG_F32, B, lam, u, out, st);
              if (e == cudaSuccess) e = cudaEventRecord(e1, st);
              if (e == cudaSuccess) e = cudaEventSynchronize(e1);
              float ms = 0.f;
              if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
              if (e == cudaSuccess && ms < ms_min) ms_min = ms;
            }
            if (e != cudaSuccess) break;
            if (times) times[((d * 2 + p) * 2 + h) * DG_NUM_KERNELS + k] = ms_min;
            if (ms_min < best_ms) {
              best_ms = ms_min;
              best = k;
            }
          }
          m->kern[d][p][h] = e == cudaSuccess ? int8_t(best) : before;
          if (h == 0 && e == cudaSuccess) m->kern[d][p][1] = int8_t(best);  // Helmholtz: the same unless timed
        }
    ++m->kern_gen;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e);
    return DG_OK;
  } catch (const std::exception& ex) {
    set_error(ex.what());
    return DG_ERR_ARG;
  }
}

}  // extern "C"
