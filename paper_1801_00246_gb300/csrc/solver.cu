// Batched preconditioned conjugate gradients with a p-multigrid preconditioner.
//
// Section 3: the SIPDG systems are symmetric positive definite and are solved
// by PCG; the screened-Poisson (velocity) systems with the scaled inverse mass
// matrix of each element as preconditioner, the pressure system with a
// multigrid preconditioner that first coarsens the polynomial degree
// (matrix-free, N -> ... -> 1) and smooths with a degree-2 Chebyshev iteration.
// The coarsest degree is solved in FP64 by CG to a loose relative tolerance,
// plain or preconditioned by an algebraic-multigrid V-cycle (amg.cu; the
// paper's pMG-AMG combination). With single-precision
// multigrid levels the preconditioner is not a fixed SPD operator, so the outer
// iteration is flexible CG (beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k).
//
// All B right-hand sides advance together; every right-hand side has its own
// scalars (alpha, beta, r.z, ...) in device memory and freezes (alpha = 0) once
// it has converged. Inner products use a fixed two-pass reduction, so reruns
// are bitwise identical.
//
// By default a solve runs as one CUDA graph: every loop whose trip count the
// residual decides (the outer iteration, the coarse CG) is a conditional WHILE
// node, closed by a one-thread kernel that reads the activity flags and sets
// the node's condition, so no iteration waits on the host.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <random>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dgx {

// Partial sums per right-hand side: 8 resident blocks of 256 threads on each of
// the 152 SMs, enough loads in flight for the FP64 vector updates to reach HBM
// bandwidth. Fixed, so every sum is taken in the same order (deterministic).
constexpr int kRedBlocks = 152 * 8;
constexpr int kRedThreads = 256;
constexpr int kNS = 16;          // scalars per right-hand side

// scalar slots
enum { S_RZ = 0, S_PAP, S_ALPHA, S_RR, S_RZOLD, S_BETA, S_BB, S_ACTIVE, S_ITERS, S_RELRES, S_BREAK, S_TOL2 };
// graph counters: kernels run inside loop bodies, outer passes, coarse passes
// (whole solve), coarse passes of the current coarse solve
enum { G_KERNELS = 0, G_OUTER, G_COARSE_TOTAL, G_COARSE, G_NCTR };
// capture streams: the top level, outer WHILE, its IF, coarse WHILE, its IF
constexpr int kCapDepth = 5;

template <typename T>
struct LevelVecs {
  T *rhs = nullptr, *x = nullptr, *res = nullptr, *d = nullptr, *Ad = nullptr, *dinv = nullptr;
};

struct Workspace {
  int B = 0;
  int64_t K = 0;
  int N = 0;
  // outer FP64 vectors
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *dinv = nullptr;
  double* scal = nullptr;     // [B][kNS]
  double* partial = nullptr;  // [B][kRedBlocks][2]
  double* h_scal = nullptr;   // pinned host mirror
  // coarse CG (FP64)
  double *crhs = nullptr, *cx = nullptr, *cr = nullptr, *cp = nullptr, *cAp = nullptr, *cscal = nullptr,
         *cpartial = nullptr;
  // multigrid levels (FP32 or FP64 per mode)
  std::vector<LevelVecs<float>> lv32;
  std::vector<LevelVecs<double>> lv64;
  std::vector<void*> allocs;
  // cached configuration
  std::string dinv_key, pmg_key;
  std::vector<double> rho;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // algebraic multigrid for the coarsest degree, keyed by (degree, lambda, B)
  Amg* amg = nullptr;
  std::string amg_key;
  uint64_t amg_gen = 0;  // bumped on every AMG (re)build
  size_t pmg_bytes = 0;  // device bytes of the p-multigrid levels' and coarse solve's vectors
  double* cz = nullptr;  // coarse preconditioned residual
  // whole-solve CUDA graph
  double *gb = nullptr, *gx = nullptr;  // staged right-hand side and iterate (the graph's fixed addresses)
  unsigned long long* gctr = nullptr;   // device counters, slots G_*
  unsigned long long* h_gctr = nullptr; // pinned mirror
  cudaStream_t cap[kCapDepth] = {};     // capture streams, one per loop nesting depth
  cudaGraphExec_t gexec = nullptr;
  std::string gkey;
  uint64_t g_top = 0;                   // kernels of the graph outside any loop body
};

static void free_one(Workspace* w) {
  if (!w) return;
  for (void* p : w->allocs) cudaFree(p);
  amg_free(w->amg);
  if (w->h_scal) cudaFreeHost(w->h_scal);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  if (w->gexec) cudaGraphExecDestroy(w->gexec);
  for (cudaStream_t c : w->cap)
    if (c) cudaStreamDestroy(c);
  if (w->h_gctr) cudaFreeHost(w->h_gctr);
  delete w;
}

void free_workspace(dg_mesh* m) {
  for (auto& kv : m->ws_cache) free_one(kv.second);
  m->ws_cache.clear();
  m->ws = nullptr;
}

namespace {

template <typename T>
cudaError_t walloc(Workspace* w, T** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
  if (e == cudaSuccess) w->allocs.push_back(*p);
  if (e == cudaSuccess) e = poison(*p, count * sizeof(T) + 16, POISON_SOLVER);
  return e;
}

inline int npd(int N) { return (N + 1) * (N + 2) / 2; }

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < int(blockDim.x >> 5); ++k) t += sh[k];
  return t;  // valid in thread 0
}

// partial[b][blk][0] = sum x.y over the block's slice of right-hand side b
template <typename TX, typename TY>
__global__ void k_dot(int64_t n, const TX* __restrict__ x, const TY* __restrict__ y, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  const TX* xb = x + size_t(b) * n;
  const TY* yb = y + size_t(b) * n;
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += double(xb[i]) * double(yb[i]);
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(size_t(b) * kRedBlocks + blockIdx.x) * 2] = t;
}

// x += alpha p; r -= alpha Ap; partial: r.r and r.zold (zold may be null)
__global__ void k_update_xr(int64_t n, const double* __restrict__ scal, double* __restrict__ x,
                            double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ Ap,
                            const double* __restrict__ zold, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  const double alpha = scal[b * kNS + S_ALPHA];
  const size_t off = size_t(b) * n;
  double rr = 0.0, rz = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[off + i] += alpha * p[off + i];
    const double ri = r[off + i] - alpha * Ap[off + i];
    r[off + i] = ri;
    rr += ri * ri;
    if (zold) rz += ri * zold[off + i];
  }
  double t = block_sum(rr, sh);
  if (threadIdx.x == 0) partial[(size_t(b) * kRedBlocks + blockIdx.x) * 2] = t;
  t = block_sum(rz, sh);
  if (threadIdx.x == 0) partial[(size_t(b) * kRedBlocks + blockIdx.x) * 2 + 1] = t;
}

enum FinMode { FIN_INIT_BB = 0, FIN_INIT_RZ, FIN_ALPHA, FIN_RR, FIN_BETA, FIN_BETA_FLEX };

// Thread t's share of one partial slot: blocks t, t + blockDim.x, ... in order.
__device__ __forceinline__ double partial_share(const double* pb, int slot) {
  double v = 0.0;
  for (int k = threadIdx.x; k < kRedBlocks; k += blockDim.x) v += pb[2 * k + slot];
  return v;
}

// Sums the partials of right-hand side b in a fixed order and updates its scalars.
__global__ void k_finalize(int mode, double* __restrict__ scal, const double* __restrict__ partial) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const double* pb = partial + size_t(b) * kRedBlocks * 2;
  const double v0 = partial_share(pb, 0);
  const double v1 = partial_share(pb, 1);
  const double s0 = block_sum(v0, sh);
  const double s1 = (mode == FIN_RR) ? block_sum(v1, sh) : 0.0;
  if (threadIdx.x != 0) return;
  double* s = scal + b * kNS;
  const bool active = s[S_ACTIVE] != 0.0;
  switch (mode) {
    case FIN_INIT_BB:
      s[S_BB] = s0;
      break;
    case FIN_INIT_RZ:  // after r = b - A x0 and z = M^{-1} r: s0 = r.z
      s[S_RZ] = s0;
      break;
    case FIN_ALPHA:
      s[S_PAP] = s0;
      if (active) {
        if (!(s0 > 0.0) || !isfinite(s0)) {
          s[S_BREAK] = 1.0;
          s[S_ACTIVE] = 0.0;
          s[S_ALPHA] = 0.0;
        } else {
          s[S_ALPHA] = s[S_RZ] / s0;
        }
      } else {
        s[S_ALPHA] = 0.0;
      }
      break;
    case FIN_RR: {
      s[S_RR] = s0;
      s[S_RZOLD] = s1;
      if (active) {
        s[S_ITERS] += 1.0;
        s[S_RELRES] = s[S_BB] > 0.0 ? sqrt(s0 / s[S_BB]) : 0.0;
        if (!isfinite(s0)) {
          s[S_BREAK] = 1.0;
          s[S_ACTIVE] = 0.0;
        } else if (s0 <= s[S_TOL2] * s[S_BB]) {
          s[S_ACTIVE] = 0.0;
        }
      }
      break;
    }
    case FIN_BETA:
    case FIN_BETA_FLEX:
      if (active) {
        const double num = (mode == FIN_BETA_FLEX) ? (s0 - s[S_RZOLD]) : s0;
        s[S_BETA] = num / s[S_RZ];
        s[S_RZ] = s0;
      } else {
        s[S_BETA] = 0.0;
      }
      break;
  }
}

__global__ void k_init_scal(int B, double* scal, double tol2) {
  const int b = threadIdx.x;
  if (b >= B) return;
  double* s = scal + b * kNS;
  for (int k = 0; k < kNS; ++k) s[k] = 0.0;
  s[S_ACTIVE] = 1.0;
  s[S_TOL2] = tol2;
}

// after initial residual: relres and activity from r.r and b.b (slot S_RR given by partial)
__global__ void k_init_check(double* scal, const double* partial) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const double* pb = partial + size_t(b) * kRedBlocks * 2;
  const double s0 = block_sum(partial_share(pb, 0), sh);
  if (threadIdx.x != 0) return;
  double* s = scal + b * kNS;
  s[S_RR] = s0;
  s[S_RELRES] = s[S_BB] > 0.0 ? sqrt(s0 / s[S_BB]) : 0.0;
  if (s0 <= s[S_TOL2] * s[S_BB]) s[S_ACTIVE] = 0.0;
}

// p = z + beta p (per right-hand side); with init: p = z (p is not read: it may
// hold anything, and 0 * NaN would not vanish)
__global__ void k_update_p(int64_t n, const double* __restrict__ scal, const double* __restrict__ z,
                           double* __restrict__ p, int init) {
  const int b = blockIdx.y;
  const size_t off = size_t(b) * n;
  if (init) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
      p[off + i] = z[off + i];
    return;
  }
  if (scal[b * kNS + S_ACTIVE] == 0.0) return;
  const double beta = scal[b * kNS + S_BETA];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[off + i] = z[off + i] + beta * p[off + i];
}

// ------------------------------------------------- device-side loop control
__device__ __forceinline__ bool any_active(const double* scal, int B) {
  bool any = false;
  for (int b = 0; b < B; ++b) any = any || scal[b * kNS + S_ACTIVE] != 0.0;
  return any;
}

// Before a loop's first pass: reset its pass count, enter if any right-hand
// side is active and the cap allows a pass.
__global__ void k_loop_head(const double* __restrict__ scal, int B, unsigned long long* __restrict__ ctr, int slot,
                            int max_iter, cudaGraphConditionalHandle hw) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctr[slot] = 0;
  cudaGraphSetConditional(hw, (max_iter > 0 && any_active(scal, B)) ? 1u : 0u);
}

// End of a loop body: count the pass (and the body's kernels), continue while
// a right-hand side is active and the cap is not reached; `hi` (if has_if)
// guards the rest of the pass (the preconditioner and the next direction),
// which runs only when another pass follows.
__global__ void k_loop_tail(const double* __restrict__ scal, int B, unsigned long long* __restrict__ ctr, int slot,
                            int total_slot, int max_iter, unsigned long long kernels, cudaGraphConditionalHandle hw,
                            cudaGraphConditionalHandle hi, int has_if) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const bool any = any_active(scal, B);
  const unsigned long long it = ++ctr[slot];
  if (total_slot >= 0) ++ctr[total_slot];
  ctr[G_KERNELS] += kernels;
  cudaGraphSetConditional(hw, (any && it < (unsigned long long)max_iter) ? 1u : 0u);
  if (has_if) cudaGraphSetConditional(hi, (any && it < (unsigned long long)max_iter) ? 1u : 0u);
}

__global__ void k_count(unsigned long long* __restrict__ ctr, unsigned long long kernels) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctr[G_KERNELS] += kernels;
}

// r = b - Ax
template <typename T>
__global__ void k_sub(int64_t n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = a[i] - b[i];
}

// z = dinv * r (dinv shared across the batch: index modulo n)
template <typename T, typename TD>
__global__ void k_scale(int64_t n, int64_t ntot, const TD* __restrict__ dinv, const T* __restrict__ r, T* __restrict__ z) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < ntot; i += int64_t(gridDim.x) * blockDim.x)
    z[i] = T(dinv[i % n]) * r[i];
}

template <typename T>
__global__ void k_scaled_copy(int64_t n, T s, const T* __restrict__ a, T* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = s * a[i];
}

template <typename T>
__global__ void k_recip(int64_t n, T* d) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    d[i] = T(1) / d[i];
}

template <typename TO, typename TI>
__global__ void k_convert(int64_t n, const TI* __restrict__ a, TO* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = TO(a[i]);
}

// z_e = (lambda J_e)^{-1} Minv r_e  (scaled inverse-mass block preconditioner)
__global__ void k_invmass(int Np, int64_t K, int B, const double* __restrict__ geo, const double* __restrict__ Minv,
                          double lambda, const double* __restrict__ r, double* __restrict__ z) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(B) * K * Np) return;
  const bool small = int64_t(B) * K * Np < (int64_t(1) << 31);  // 32-bit divisions where they fit
  const int64_t be = small ? int64_t(uint32_t(idx) / uint32_t(Np)) : idx / Np;
  const int i = int(idx - be * Np);
  const int64_t e = B == 1 ? be : (small ? int64_t(uint32_t(be) % uint32_t(K)) : be % K);
  const double* g = geo + 4 * e;
  const double J = 1.0 / (g[0] * g[3] - g[2] * g[1]);
  const double* re = r + be * Np;
  double acc = 0.0;
  for (int j = 0; j < Np; ++j) acc += Minv[size_t(i) * Np + j] * re[j];
  z[idx] = acc / (lambda * J);
}

// ------------------------------------------------------------- multigrid pieces
// Chebyshev first step: if zero_x: res = rhs, d = c0 dinv rhs, x = d;
//                       else      d = c0 dinv res, x += d.
template <typename T>
__global__ void k_cheb_first(int64_t n, int64_t ntot, const T* __restrict__ dinv, const T* __restrict__ rhs,
                             const T* __restrict__ Ax, T* __restrict__ res, T* __restrict__ d, T* __restrict__ x,
                             T c0) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < ntot; i += int64_t(gridDim.x) * blockDim.x) {
    const T ri = Ax ? rhs[i] - Ax[i] : rhs[i];  // Ax null: x = 0
    res[i] = ri;
    const T di = c0 * dinv[i % n] * ri;
    d[i] = di;
    x[i] = Ax ? x[i] + di : di;
  }
}

// res -= Ad; d = c1 d + c2 dinv res; x += d
template <typename T>
__global__ void k_cheb_step(int64_t n, int64_t ntot, const T* __restrict__ dinv, const T* __restrict__ Ad,
                            T* __restrict__ res, T* __restrict__ d, T* __restrict__ x, T c1, T c2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < ntot; i += int64_t(gridDim.x) * blockDim.x) {
    const T ri = res[i] - Ad[i];
    res[i] = ri;
    const T di = c1 * d[i] + c2 * dinv[i % n] * ri;
    d[i] = di;
    x[i] += di;
  }
}

// rc[e][j] = sum_i P[i][j] (res[e][i] - Ad[e][i]) (restriction R = P^T of the
// residual after the last smoothing step, which nothing else reads)
template <typename T>
__global__ void k_sub_restrict(int Npf, int Npc, int64_t nE, const T* __restrict__ P, const T* __restrict__ res,
                               const T* __restrict__ Ad, T* __restrict__ rc) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= nE * Npc) return;
  const int64_t e = nE * Npc < (int64_t(1) << 31) ? int64_t(uint32_t(idx) / uint32_t(Npc)) : idx / Npc;
  const int j = int(idx - e * Npc);
  const T* re = res + e * Npf;
  const T* ae = Ad + e * Npf;
  T acc = T(0);
  for (int i = 0; i < Npf; ++i) acc += P[size_t(i) * Npc + j] * (re[i] - ae[i]);
  rc[idx] = acc;
}

// xf[e][i] += sum_j P[i][j] xc[e][j]
template <typename T>
__global__ void k_prolong(int Npf, int Npc, int64_t nE, const T* __restrict__ P, const T* __restrict__ xc,
                          T* __restrict__ xf) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= nE * Npf) return;
  const int64_t e = nE * Npf < (int64_t(1) << 31) ? int64_t(uint32_t(idx) / uint32_t(Npf)) : idx / Npf;
  const int i = int(idx - e * Npf);
  const T* ce = xc + e * Npc;
  T acc = T(0);
  for (int j = 0; j < Npc; ++j) acc += P[size_t(i) * Npc + j] * ce[j];
  xf[idx] += acc;
}

// Reductions always run kRedBlocks blocks per right-hand side (blocks past the
// end of the data write zero partials), so the finalisation reads a fixed set.
inline dim3 vgrid(int64_t n, int B) {
  (void)n;
  return dim3(unsigned(kRedBlocks), unsigned(B));
}
inline int egrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return int(b < 1 ? 1 : b);
}

// the first failing call of a solve, for the error message
thread_local char g_fail_where[160] = "";
inline cudaError_t note_fail(cudaError_t e, const char* what, int line) {
  if (g_fail_where[0] == 0) std::snprintf(g_fail_where, sizeof g_fail_where, "%.120s (solver.cu:%d)", what, line);
  return e;
}

#define CK(x)                                                 \
  do {                                                        \
    cudaError_t e_ = (x);                                     \
    if (e_ != cudaSuccess) return note_fail(e_, #x, __LINE__); \
  } while (0)

struct GraphState;

struct Ctx {
  dg_mesh* m;
  const dg_solver_opts* o;
  int B;
  double lambda;
  cudaStream_t st;
  Workspace* w;
  GraphState* g = nullptr;  // non-null while the solve is being captured
};

// Capture bookkeeping: the stream of each open loop body, and the kernel count
// at its start (so each body's closing kernel can count its own kernels).
struct Frame {
  cudaStream_t outer;
  uint64_t n0;
  uint64_t nested;  // kernels captured in bodies nested inside this one
};
struct GraphState {
  int depth = 0;
  std::vector<Frame> frames;
  uint64_t root_nested = 0;
};

// Creates a condition handle in the graph being captured on c.st.
cudaError_t cond_handle(Ctx& c, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, g, 0, 0);
}

// Appends a conditional node after the work captured so far on c.st and
// redirects c.st into its body until cond_close.
cudaError_t cond_open(Ctx& c, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
  GraphState* G = c.g;
  if (G->depth + 1 >= kCapDepth) return cudaErrorNotSupported;
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c.st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  CK(cudaStreamUpdateCaptureDependencies(c.st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t body = c.w->cap[G->depth + 1];
  CK(cudaStreamBeginCaptureToGraph(body, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  G->frames.push_back({c.st, launch_count(), 0});
  ++G->depth;
  c.st = body;
  return cudaSuccess;
}

// kernels captured so far in the innermost open body, plus one for the kernel about to close it
uint64_t body_kernels(Ctx& c) {
  const Frame& f = c.g->frames.back();
  return launch_count() - f.n0 - f.nested + 1;
}

cudaError_t cond_close(Ctx& c) {
  GraphState* G = c.g;
  const Frame f = G->frames.back();
  G->frames.pop_back();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.st, &g);
  c.st = f.outer;
  --G->depth;
  const uint64_t total = launch_count() - f.n0;
  if (G->frames.empty()) G->root_nested += total;
  else G->frames.back().nested += total;
  return e;
}

cudaError_t ensure_transfer(dg_mesh* m, int Nf, int Nc) {
  auto key = std::make_pair(Nf, Nc);
  if (m->transfer.count(key)) return cudaSuccess;
  const std::vector<double> P = interpolation_matrix(Nf, Nc);
  std::vector<float> Pf(P.begin(), P.end());
  DevTransfer t;
  CK(cudaMalloc(&t.P64, P.size() * sizeof(double)));
  CK(cudaMalloc(&t.P32, P.size() * sizeof(float)));
  CK(cudaMemcpy(t.P64, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(t.P32, Pf.data(), Pf.size() * sizeof(float), cudaMemcpyHostToDevice));
  m->transfer[key] = t;
  return cudaSuccess;
}

cudaError_t setup_workspace(Ctx& c) {
  dg_mesh* m = c.m;
  const dg_solver_opts* o = c.o;
  Workspace* w = m->ws;
  const bool pmg = o->precond == DG_PREC_PMG;
  std::string key = std::to_string(c.B) + "/" + std::to_string(pmg) + "/" + std::to_string(o->mixed);
  if (pmg)
    for (int l = 0; l < o->nlevels; ++l) key += "," + std::to_string(o->degrees[l]);
  auto it = m->ws_cache.find(key);
  if (it != m->ws_cache.end()) {
    m->ws = it->second;
    return cudaSuccess;
  }
  w = new Workspace();
  m->ws_cache[key] = w;
  m->ws = w;
  w->B = c.B;
  w->K = m->K;
  w->N = m->N;
  w->pmg_key = key;
  const int64_t n = int64_t(m->K) * npd(m->N);
  const size_t nt = size_t(n) * c.B;
  CK(walloc(w, &w->r, nt));
  CK(walloc(w, &w->z, nt));
  CK(walloc(w, &w->p, nt));
  CK(walloc(w, &w->Ap, nt));
  CK(walloc(w, &w->dinv, size_t(n)));
  CK(walloc(w, &w->scal, size_t(c.B) * kNS));
  CK(walloc(w, &w->partial, size_t(c.B) * kRedBlocks * 2));
  CK(cudaMallocHost(&w->h_scal, sizeof(double) * c.B * kNS));
  CK(cudaEventCreate(&w->ev0));
  CK(cudaEventCreate(&w->ev1));
  if (pmg) {
    const int L = o->nlevels;
    for (int l = 0; l + 1 < L; ++l) CK(ensure_transfer(m, o->degrees[l], o->degrees[l + 1]));
    for (int l = 0; l < L; ++l) CK(ensure_ops(m, o->degrees[l]));
    if (o->mixed) w->lv32.resize(L);
    else w->lv64.resize(L);
    for (int l = 0; l < L; ++l) {
      const size_t nl = size_t(m->K) * npd(o->degrees[l]);
      if (o->mixed) {
        LevelVecs<float>& v = w->lv32[l];
        CK(walloc(w, &v.rhs, nl * c.B));
        CK(walloc(w, &v.x, nl * c.B));
        CK(walloc(w, &v.res, nl * c.B));
        CK(walloc(w, &v.d, nl * c.B));
        CK(walloc(w, &v.Ad, nl * c.B));
        CK(walloc(w, &v.dinv, nl));
      } else {
        LevelVecs<double>& v = w->lv64[l];
        CK(walloc(w, &v.rhs, nl * c.B));
        CK(walloc(w, &v.x, nl * c.B));
        CK(walloc(w, &v.res, nl * c.B));
        CK(walloc(w, &v.d, nl * c.B));
        CK(walloc(w, &v.Ad, nl * c.B));
        CK(walloc(w, &v.dinv, nl));
      }
      w->pmg_bytes += (o->mixed ? sizeof(float) : sizeof(double)) * nl * (5 * size_t(c.B) + 1);
    }
    const size_t nc = size_t(m->K) * npd(o->degrees[L - 1]) * c.B;
    w->pmg_bytes += sizeof(double) * nc * 6;
    CK(walloc(w, &w->crhs, nc));
    CK(walloc(w, &w->cx, nc));
    CK(walloc(w, &w->cr, nc));
    CK(walloc(w, &w->cp, nc));
    CK(walloc(w, &w->cAp, nc));
    CK(walloc(w, &w->cz, nc));
    CK(walloc(w, &w->cscal, size_t(c.B) * kNS));
    CK(walloc(w, &w->cpartial, size_t(c.B) * kRedBlocks * 2));
  }
  return cudaSuccess;
}

// Plain CG on the coarsest degree in FP64 to relative tolerance coarse_tol,
// starting from x = 0. Host-driven, convergence is checked every `chk` steps
// and converged right-hand sides stay frozen on the device in between; in a
// captured solve the loop is a device-side WHILE node checked every pass.
cudaError_t coarse_cg(Ctx& c, int degree, const double* rhs, double* x, int& iters_out) {
  Workspace* w = c.w;
  const int B = c.B;
  const int64_t n = int64_t(c.m->K) * npd(degree);
  const size_t nt = size_t(n) * B;
  const dim3 g = vgrid(n, B);
  const double tol = c.o->coarse_tol;
  CK(cudaMemsetAsync(x, 0, nt * sizeof(double), c.st));
  CK(cudaMemcpyAsync(w->cr, rhs, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  k_init_scal<<<1, 64, 0, c.st>>>(B, w->cscal, tol * tol); note_launch();
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, rhs, rhs, w->cpartial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_INIT_BB, w->cscal, w->cpartial); note_launch();
  k_init_check<<<B, kRedThreads, 0, c.st>>>(w->cscal, w->cpartial); note_launch();  // r = b: r.r = b.b
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_INIT_RZ, w->cscal, w->cpartial); note_launch();
  k_update_p<<<g, kRedThreads, 0, c.st>>>(n, w->cscal, w->cr, w->cp, 1); note_launch();
  auto pass = [&]() -> cudaError_t {
    CK(launch_apply(c.m, degree, DG_F64, B, c.lambda, w->cp, w->cAp, c.st));
    k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->cp, w->cAp, w->cpartial); note_launch();
    k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_ALPHA, w->cscal, w->cpartial); note_launch();
    k_update_xr<<<g, kRedThreads, 0, c.st>>>(n, w->cscal, x, w->cr, w->cp, w->cAp, nullptr, w->cpartial); note_launch();
    k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_RR, w->cscal, w->cpartial); note_launch();
    k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->cr, w->cr, w->cpartial); note_launch();
    k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_BETA, w->cscal, w->cpartial); note_launch();
    k_update_p<<<g, kRedThreads, 0, c.st>>>(n, w->cscal, w->cr, w->cp, 0); note_launch();
    return cudaSuccess;
  };
  if (c.g) {
    cudaGraphConditionalHandle hw = 0;
    CK(cond_handle(c, &hw));
    k_loop_head<<<1, 32, 0, c.st>>>(w->cscal, B, w->gctr, G_COARSE, c.o->coarse_max_iter, hw); note_launch();
    CK(cond_open(c, hw, cudaGraphCondTypeWhile));
    CK(pass());
    k_loop_tail<<<1, 32, 0, c.st>>>(w->cscal, B, w->gctr, G_COARSE, G_COARSE_TOTAL, c.o->coarse_max_iter,
                                    body_kernels(c), hw, 0, 0); note_launch();
    CK(cond_close(c));
    iters_out = 0;  // counted on the device
    return cudaGetLastError();
  }
  const int chk = 8;
  int it = 0;
  for (; it < c.o->coarse_max_iter;) {
    CK(pass());
    ++it;
    if (it % chk == 0 || it == c.o->coarse_max_iter) {
      CK(cudaMemcpyAsync(w->h_scal, w->cscal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, c.st));
      CK(cudaStreamSynchronize(c.st));
      bool any = false;
      for (int b = 0; b < B; ++b) any = any || w->h_scal[b * kNS + S_ACTIVE] != 0.0;
      if (!any) break;
    }
  }
  iters_out = it;
  return cudaGetLastError();
}

// The algebraic multigrid of the coarsest degree for this batch and lambda
// (built on the host from the probed matrix; never while a solve is captured).
cudaError_t ensure_amg(Ctx& c, int degree) {
  Workspace* w = c.w;
  char key[96];
  std::snprintf(key, sizeof key, "%d/%.17g/%d", degree, c.lambda, c.B);
  if (w->amg && w->amg_key == key) return cudaSuccess;
  if (c.g) return cudaErrorStreamCaptureUnsupported;
  amg_free(w->amg);
  w->amg = nullptr;
  CK(amg_build(c.m, degree, c.lambda, c.B, &w->amg, c.st));
  w->amg_key = key;
  ++w->amg_gen;
  return cudaSuccess;
}

// CG on the coarsest degree preconditioned by one AMG V-cycle per iteration,
// to relative tolerance coarse_tol from x = 0 (host check every iteration, or
// a device-side WHILE node in a captured solve).
cudaError_t coarse_pcg_amg(Ctx& c, int degree, const double* rhs, double* x, int& iters_out) {
  Workspace* w = c.w;
  const int B = c.B;
  CK(ensure_amg(c, degree));
  const int64_t n = int64_t(c.m->K) * npd(degree);
  const size_t nt = size_t(n) * B;
  const dim3 g = vgrid(n, B);
  CK(cudaMemsetAsync(x, 0, nt * sizeof(double), c.st));
  CK(cudaMemcpyAsync(w->cr, rhs, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  k_init_scal<<<1, 64, 0, c.st>>>(B, w->cscal, c.o->coarse_tol * c.o->coarse_tol); note_launch();
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, rhs, rhs, w->cpartial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_INIT_BB, w->cscal, w->cpartial); note_launch();
  k_init_check<<<B, kRedThreads, 0, c.st>>>(w->cscal, w->cpartial); note_launch();
  CK(amg_vcycle(w->amg, w->cr, w->cz, c.st));
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->cr, w->cz, w->cpartial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_INIT_RZ, w->cscal, w->cpartial); note_launch();
  k_update_p<<<g, kRedThreads, 0, c.st>>>(n, w->cscal, w->cz, w->cp, 1); note_launch();
  auto half1 = [&]() -> cudaError_t {
    CK(amg_apply_fine(w->amg, w->cp, w->cAp, c.st));  // the probed matrix is this degree's operator
    k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->cp, w->cAp, w->cpartial); note_launch();
    k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_ALPHA, w->cscal, w->cpartial); note_launch();
    k_update_xr<<<g, kRedThreads, 0, c.st>>>(n, w->cscal, x, w->cr, w->cp, w->cAp, nullptr, w->cpartial);
    note_launch();
    k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_RR, w->cscal, w->cpartial); note_launch();
    return cudaSuccess;
  };
  auto half2 = [&]() -> cudaError_t {
    CK(amg_vcycle(w->amg, w->cr, w->cz, c.st));
    k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->cr, w->cz, w->cpartial); note_launch();
    k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_BETA, w->cscal, w->cpartial); note_launch();
    k_update_p<<<g, kRedThreads, 0, c.st>>>(n, w->cscal, w->cz, w->cp, 0); note_launch();
    return cudaSuccess;
  };
  if (c.g) {
    cudaGraphConditionalHandle hw = 0, hi = 0;
    CK(cond_handle(c, &hw));
    k_loop_head<<<1, 32, 0, c.st>>>(w->cscal, B, w->gctr, G_COARSE, c.o->coarse_max_iter, hw); note_launch();
    CK(cond_open(c, hw, cudaGraphCondTypeWhile));
    CK(half1());
    CK(cond_handle(c, &hi));
    k_loop_tail<<<1, 32, 0, c.st>>>(w->cscal, B, w->gctr, G_COARSE, G_COARSE_TOTAL, c.o->coarse_max_iter,
                                    body_kernels(c), hw, hi, 1); note_launch();
    CK(cond_open(c, hi, cudaGraphCondTypeIf));
    CK(half2());
    k_count<<<1, 32, 0, c.st>>>(w->gctr, body_kernels(c)); note_launch();
    CK(cond_close(c));
    CK(cond_close(c));
    iters_out = 0;
    return cudaGetLastError();
  }
  int it = 0;
  for (; it < c.o->coarse_max_iter;) {
    CK(half1());
    ++it;
    CK(cudaMemcpyAsync(w->h_scal, w->cscal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    bool any = false;
    for (int b = 0; b < B; ++b) any = any || w->h_scal[b * kNS + S_ACTIVE] != 0.0;
    if (!any || it >= c.o->coarse_max_iter) break;  // no further pass: no preconditioning for it
    CK(half2());
  }
  iters_out = it;
  return cudaGetLastError();
}

template <typename T>
std::vector<LevelVecs<T>>& levels(Workspace* w);
template <>
std::vector<LevelVecs<float>>& levels<float>(Workspace* w) { return w->lv32; }
template <>
std::vector<LevelVecs<double>>& levels<double>(Workspace* w) { return w->lv64; }

template <typename T>
const T* transfer_ptr(dg_mesh* m, int Nf, int Nc);
template <>
const float* transfer_ptr<float>(dg_mesh* m, int Nf, int Nc) { return m->transfer[std::make_pair(Nf, Nc)].P32; }
template <>
const double* transfer_ptr<double>(dg_mesh* m, int Nf, int Nc) { return m->transfer[std::make_pair(Nf, Nc)].P64; }

template <typename T>
constexpr dg_prec prec_of() { return std::is_same<T, double>::value ? DG_F64 : DG_F32; }

// Chebyshev smoothing of the given degree on level l.
template <typename T>
cudaError_t chebyshev(Ctx& c, int l, bool zero_x) {
  LevelVecs<T>& v = levels<T>(c.w)[l];
  const int deg = c.o->degrees[l];
  const int64_t n = int64_t(c.m->K) * npd(deg);
  const int64_t nt = n * c.B;
  const double rho = c.w->rho[l];
  const double lmin = rho / 10.0, lmax = 1.1 * rho;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rk = 1.0 / sigma;
  if (!zero_x) CK(launch_apply(c.m, deg, prec_of<T>(), c.B, c.lambda, v.x, v.Ad, c.st));
  // res = rhs (- A x), d = D^{-1} res / theta, x (+)= d
  k_cheb_first<T><<<egrid(nt), 256, 0, c.st>>>(n, nt, v.dinv, v.rhs, zero_x ? nullptr : v.Ad, v.res, v.d, v.x,
                                                T(1.0 / theta)); note_launch();
  for (int k = 1; k < c.o->cheb_degree; ++k) {
    CK(launch_apply(c.m, deg, prec_of<T>(), c.B, c.lambda, v.d, v.Ad, c.st));
    const double rnew = 1.0 / (2.0 * sigma - rk);
    k_cheb_step<T><<<egrid(nt), 256, 0, c.st>>>(n, nt, v.dinv, v.Ad, v.res, v.d, v.x, T(rnew * rk), T(2.0 * rnew / delta)); note_launch();
    rk = rnew;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t vcycle(Ctx& c, int l, int& coarse_iters) {
  std::vector<LevelVecs<T>>& lv = levels<T>(c.w);
  const int L = c.o->nlevels;
  const int deg = c.o->degrees[l];
  const int64_t n = int64_t(c.m->K) * npd(deg);
  const int64_t nt = n * c.B;
  if (l == L - 1) {
    // coarsest degree: CG in FP64 whatever the level precision
    int it = 0;
    auto solve = [&](const double* r, double* xo) {
      return c.o->coarse_amg ? coarse_pcg_amg(c, deg, r, xo, it) : coarse_cg(c, deg, r, xo, it);
    };
    if (std::is_same<T, double>::value) {
      CK(solve(reinterpret_cast<const double*>(lv[l].rhs), reinterpret_cast<double*>(lv[l].x)));
    } else {
      k_convert<double, T><<<egrid(nt), 256, 0, c.st>>>(nt, lv[l].rhs, c.w->crhs); note_launch();
      CK(solve(c.w->crhs, c.w->cx));
      k_convert<T, double><<<egrid(nt), 256, 0, c.st>>>(nt, c.w->cx, lv[l].x); note_launch();
    }
    coarse_iters += it;
    return cudaGetLastError();
  }
  LevelVecs<T>& v = lv[l];
  // pre-smoothing from x = 0, then res = rhs - A x
  CK(chebyshev<T>(c, l, true));
  CK(launch_apply(c.m, deg, prec_of<T>(), c.B, c.lambda, v.d, v.Ad, c.st));
  // restrict res - A d, recurse, prolong
  const int degc = c.o->degrees[l + 1];
  const int Npf = npd(deg), Npc = npd(degc);
  const int64_t nE = int64_t(c.m->K) * c.B;
  const T* P = transfer_ptr<T>(c.m, deg, degc);
  k_sub_restrict<T><<<int((nE * Npc + 255) / 256), 256, 0, c.st>>>(Npf, Npc, nE, P, v.res, v.Ad, lv[l + 1].rhs);
  note_launch();
  CK(vcycle<T>(c, l + 1, coarse_iters));
  k_prolong<T><<<int((nE * Npf + 255) / 256), 256, 0, c.st>>>(Npf, Npc, nE, P, lv[l + 1].x, v.x); note_launch();
  // post-smoothing
  CK(chebyshev<T>(c, l, false));
  return cudaGetLastError();
}

// Largest eigenvalue of D^{-1}A on level l by power iteration from a seeded
// random start (normalised on the host; setup cost only).
template <typename T>
cudaError_t power_rho(Ctx& c, int l, double& rho) {
  LevelVecs<T>& v = levels<T>(c.w)[l];
  const int deg = c.o->degrees[l];
  const int64_t n = int64_t(c.m->K) * npd(deg);
  std::vector<T> h(n);
  std::mt19937_64 rng(12345 + deg);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (auto& e : h) e = T(nd(rng));
  CK(cudaMemcpyAsync(v.d, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, c.st));
  const dim3 g = vgrid(n, 1);
  std::vector<double> hp(kRedBlocks * 2);
  auto norm = [&](const T* a, double& out) -> cudaError_t {
    k_dot<T, T><<<g, kRedThreads, 0, c.st>>>(n, a, a, c.w->partial); note_launch();
    CK(cudaMemcpyAsync(hp.data(), c.w->partial, sizeof(double) * kRedBlocks * 2, cudaMemcpyDeviceToHost, c.st));
    CK(cudaStreamSynchronize(c.st));
    double s = 0.0;
    for (unsigned k = 0; k < g.x; ++k) s += hp[2 * k];
    out = std::sqrt(s);
    return cudaSuccess;
  };
  double nv = 1.0, lam = 0.0;
  CK(norm(v.d, nv));
  for (int it = 0; it < c.o->power_steps; ++it) {
    k_scaled_copy<T><<<egrid(n), 256, 0, c.st>>>(n, T(1.0 / nv), v.d, v.x); note_launch();  // x = d / ||d||
    CK(launch_apply(c.m, deg, prec_of<T>(), 1, c.lambda, v.x, v.Ad, c.st));
    k_scale<T, T><<<egrid(n), 256, 0, c.st>>>(n, n, v.dinv, v.Ad, v.d); note_launch();    // d = D^{-1} A x
    CK(norm(v.d, nv));
    lam = nv;
  }
  rho = lam;
  return cudaGetLastError();
}

cudaError_t setup_pmg(Ctx& c, std::string& key) {
  Workspace* w = c.w;
  const dg_solver_opts* o = c.o;
  char buf[64];
  std::snprintf(buf, sizeof buf, "%.17g/%d/%d", c.lambda, o->power_steps, o->mixed);
  key = buf;
  if (w->dinv_key == key && !w->rho.empty()) return cudaSuccess;
  w->rho.assign(o->nlevels, 0.0);
  for (int l = 0; l < o->nlevels; ++l) {
    const int deg = o->degrees[l];
    const int64_t n = int64_t(c.m->K) * npd(deg);
    if (o->mixed) {
      CK(launch_diagonal(c.m, deg, DG_F32, c.lambda, w->lv32[l].dinv, c.st));
      k_recip<float><<<egrid(n), 256, 0, c.st>>>(n, w->lv32[l].dinv); note_launch();
      if (l + 1 < o->nlevels) CK(power_rho<float>(c, l, w->rho[l]));
    } else {
      CK(launch_diagonal(c.m, deg, DG_F64, c.lambda, w->lv64[l].dinv, c.st));
      k_recip<double><<<egrid(n), 256, 0, c.st>>>(n, w->lv64[l].dinv); note_launch();
      if (l + 1 < o->nlevels) CK(power_rho<double>(c, l, w->rho[l]));
    }
  }
  w->dinv_key = key;
  return cudaGetLastError();
}

// z = M^{-1} r for the outer iteration
cudaError_t precondition(Ctx& c, int& coarse_iters) {
  Workspace* w = c.w;
  const int64_t n = int64_t(c.m->K) * npd(c.m->N);
  const int64_t nt = n * c.B;
  switch (c.o->precond) {
    case DG_PREC_NONE:
      CK(cudaMemcpyAsync(w->z, w->r, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
      break;
    case DG_PREC_JACOBI:
      k_scale<double, double><<<egrid(nt), 256, 0, c.st>>>(n, nt, w->dinv, w->r, w->z); note_launch();
      break;
    case DG_PREC_INVMASS: {
      const int Np = npd(c.m->N);
      const double* Minv = reinterpret_cast<const double*>(c.m->ops64[c.m->N].buf) + (ops_count(c.m->N) - size_t(Np) * Np);
      k_invmass<<<int((nt + 255) / 256), 256, 0, c.st>>>(Np, c.m->K, c.B, c.m->geo64, Minv, c.lambda, w->r, w->z); note_launch();
      break;
    }
    case DG_PREC_AMG:
      CK(amg_vcycle(w->amg, w->r, w->z, c.st));
      break;
    case DG_PREC_PMG:
      if (c.o->mixed) {
        k_convert<float, double><<<egrid(nt), 256, 0, c.st>>>(nt, w->r, w->lv32[0].rhs); note_launch();
        CK(vcycle<float>(c, 0, coarse_iters));
        k_convert<double, float><<<egrid(nt), 256, 0, c.st>>>(nt, w->lv32[0].x, w->z); note_launch();
      } else {
        CK(cudaMemcpyAsync(w->lv64[0].rhs, w->r, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
        CK(vcycle<double>(c, 0, coarse_iters));
        CK(cudaMemcpyAsync(w->z, w->lv64[0].x, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
      }
      break;
  }
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------ outer iteration
// Start: scalars, r = b - A x, z = M^{-1} r, r.z, p = z.
cudaError_t pcg_start(Ctx& c, const double* b, double* x, int& coarse_iters) {
  Workspace* w = c.w;
  const int B = c.B;
  const int64_t n = int64_t(c.m->K) * npd(c.m->N);
  const int64_t nt = n * B;
  const dim3 g = vgrid(n, B);
  k_init_scal<<<1, 64, 0, c.st>>>(B, w->scal, c.o->tol * c.o->tol); note_launch();
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, b, b, w->partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_INIT_BB, w->scal, w->partial); note_launch();
  CK(launch_apply(c.m, c.m->N, DG_F64, B, c.lambda, x, w->Ap, c.st));
  k_sub<double><<<egrid(nt), 256, 0, c.st>>>(nt, b, w->Ap, w->r); note_launch();
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->r, w->r, w->partial); note_launch();
  k_init_check<<<B, kRedThreads, 0, c.st>>>(w->scal, w->partial); note_launch();
  CK(precondition(c, coarse_iters));
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->r, w->z, w->partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_INIT_RZ, w->scal, w->partial); note_launch();
  k_update_p<<<g, kRedThreads, 0, c.st>>>(n, w->scal, w->z, w->p, 1); note_launch();
  return cudaGetLastError();
}

// First half of a pass: A p, alpha, x += alpha p, r -= alpha A p, r.r (convergence).
cudaError_t pcg_half1(Ctx& c, double* x, bool flexible) {
  Workspace* w = c.w;
  const int B = c.B;
  const int64_t n = int64_t(c.m->K) * npd(c.m->N);
  const dim3 g = vgrid(n, B);
  CK(launch_apply(c.m, c.m->N, DG_F64, B, c.lambda, w->p, w->Ap, c.st));
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->p, w->Ap, w->partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_ALPHA, w->scal, w->partial); note_launch();
  k_update_xr<<<g, kRedThreads, 0, c.st>>>(n, w->scal, x, w->r, w->p, w->Ap, flexible ? w->z : nullptr, w->partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(FIN_RR, w->scal, w->partial); note_launch();
  return cudaGetLastError();
}

// Second half: z = M^{-1} r, beta, p = z + beta p.
cudaError_t pcg_half2(Ctx& c, bool flexible, int& coarse_iters) {
  Workspace* w = c.w;
  const int B = c.B;
  const int64_t n = int64_t(c.m->K) * npd(c.m->N);
  const dim3 g = vgrid(n, B);
  CK(precondition(c, coarse_iters));
  k_dot<<<g, kRedThreads, 0, c.st>>>(n, w->r, w->z, w->partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, c.st>>>(flexible ? FIN_BETA_FLEX : FIN_BETA, w->scal, w->partial); note_launch();
  k_update_p<<<g, kRedThreads, 0, c.st>>>(n, w->scal, w->z, w->p, 0); note_launch();
  return cudaGetLastError();
}

// Host-driven loop: the residual check reads the scalars back every `chk` passes.
cudaError_t pcg_eager(Ctx& c, const double* b, double* x, int& it, int& coarse_iters) {
  Workspace* w = c.w;
  const dg_solver_opts* o = c.o;
  const int B = c.B;
  const bool flexible = o->precond == DG_PREC_PMG || o->precond == DG_PREC_AMG;
  CK(cudaEventRecord(w->ev0, c.st));
  CK(pcg_start(c, b, x, coarse_iters));
  CK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  bool any = false;
  for (int bb = 0; bb < B; ++bb) any = any || w->h_scal[bb * kNS + S_ACTIVE] != 0.0;
  it = 0;
  const int chk = flexible ? 1 : 4;
  while (any && it < o->max_iter) {
    CK(pcg_half1(c, x, flexible));
    ++it;
    if (it % chk == 0 || it == o->max_iter) {
      CK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, c.st));
      CK(cudaStreamSynchronize(c.st));
      any = false;
      for (int bb = 0; bb < B; ++bb) any = any || w->h_scal[bb * kNS + S_ACTIVE] != 0.0;
      if (!any) break;
    }
    if (it >= o->max_iter) break;  // no further pass: no preconditioning for it
    CK(pcg_half2(c, flexible, coarse_iters));
  }
  CK(cudaEventRecord(w->ev1, c.st));
  return cudaSuccess;
}

// Every (degree, precision) the solve applies, once on zeroed scratch, so that
// all lazily sized buffers and uploaded operators exist before the capture
// (allocations are not captured).
cudaError_t warm_applies(Ctx& c) {
  Workspace* w = c.w;
  const dg_solver_opts* o = c.o;
  const size_t nt = size_t(c.m->K) * npd(c.m->N) * c.B;
  CK(cudaMemsetAsync(w->p, 0, nt * sizeof(double), c.st));
  CK(launch_apply(c.m, c.m->N, DG_F64, c.B, c.lambda, w->p, w->Ap, c.st));
  if (o->precond != DG_PREC_PMG) return cudaGetLastError();
  const int L = o->nlevels;
  for (int l = 0; l + 1 < L; ++l) {
    const size_t nl = size_t(c.m->K) * npd(o->degrees[l]) * c.B;
    if (o->mixed) {
      CK(cudaMemsetAsync(w->lv32[l].d, 0, nl * sizeof(float), c.st));
      CK(launch_apply(c.m, o->degrees[l], DG_F32, c.B, c.lambda, w->lv32[l].d, w->lv32[l].Ad, c.st));
    } else {
      CK(cudaMemsetAsync(w->lv64[l].d, 0, nl * sizeof(double), c.st));
      CK(launch_apply(c.m, o->degrees[l], DG_F64, c.B, c.lambda, w->lv64[l].d, w->lv64[l].Ad, c.st));
    }
  }
  if (!o->coarse_amg) {
    const size_t nc = size_t(c.m->K) * npd(o->degrees[L - 1]) * c.B;
    CK(cudaMemsetAsync(w->cp, 0, nc * sizeof(double), c.st));
    CK(launch_apply(c.m, o->degrees[L - 1], DG_F64, c.B, c.lambda, w->cp, w->cAp, c.st));
  }
  return cudaGetLastError();
}

// Everything a captured graph has baked in: batch, lambda, options, the
// scratch and AMG buffers it addresses, the apply kernels chosen, and the
// smoother bounds.
std::string graph_key(const Ctx& c) {
  const dg_solver_opts* o = c.o;
  char buf[400];
  std::snprintf(buf, sizeof buf, "%d|%.17g|%.17g|%d|%d|%d|%d|%.17g|%d|%d|%d|%d|%llu|%llu|%llu|%s|", c.B, c.lambda,
                o->tol, o->max_iter, o->precond, o->nlevels, o->cheb_degree, o->coarse_tol, o->coarse_max_iter,
                o->mixed, o->power_steps, o->coarse_amg, (unsigned long long)c.m->scratch_gen,
                (unsigned long long)c.m->kern_gen, (unsigned long long)c.w->amg_gen, c.w->dinv_key.c_str());
  std::string k = buf;
  for (int l = 0; l < o->nlevels && l < 8; ++l) k += std::to_string(o->degrees[l]) + ",";
  return k;
}

// The captured solve: counters reset, start, then
//   WHILE (active and passes < max_iter) { first half; tail; IF (active) { second half } }
cudaError_t capture_body(Ctx& c) {
  Workspace* w = c.w;
  const bool flexible = c.o->precond == DG_PREC_PMG || c.o->precond == DG_PREC_AMG;
  int unused = 0;
  CK(cudaMemsetAsync(w->gctr, 0, sizeof(unsigned long long) * G_NCTR, c.st));
  CK(pcg_start(c, w->gb, w->gx, unused));
  cudaGraphConditionalHandle hw = 0, hi = 0;
  CK(cond_handle(c, &hw));
  k_loop_head<<<1, 32, 0, c.st>>>(w->scal, c.B, w->gctr, G_OUTER, c.o->max_iter, hw); note_launch();
  CK(cond_open(c, hw, cudaGraphCondTypeWhile));
  CK(pcg_half1(c, w->gx, flexible));
  CK(cond_handle(c, &hi));
  k_loop_tail<<<1, 32, 0, c.st>>>(w->scal, c.B, w->gctr, G_OUTER, -1, c.o->max_iter, body_kernels(c), hw, hi, 1);
  note_launch();
  CK(cond_open(c, hi, cudaGraphCondTypeIf));
  CK(pcg_half2(c, flexible, unused));
  k_count<<<1, 32, 0, c.st>>>(w->gctr, body_kernels(c)); note_launch();
  CK(cond_close(c));
  CK(cond_close(c));
  return cudaGetLastError();
}

cudaError_t capture_solve(Ctx& c, const std::string& key) {
  Workspace* w = c.w;
  if (w->gexec) {
    cudaGraphExecDestroy(w->gexec);
    w->gexec = nullptr;
    w->gkey.clear();
  }
  GraphState G;
  Ctx cc = c;
  cc.g = &G;
  cc.st = w->cap[0];
  const uint64_t n0 = launch_count();
  CK(cudaStreamBeginCapture(cc.st, cudaStreamCaptureModeRelaxed));
  cudaError_t e = capture_body(cc);
  // close whatever a failure left open, innermost first
  while (!G.frames.empty()) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(cc.st, &dummy);
    cc.st = G.frames.back().outer;
    G.frames.pop_back();
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cc.st, &graph);
  const uint64_t total = launch_count() - n0;
  add_launches(-int64_t(total));  // counted when they run
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) {
    w->g_top = total - G.root_nested;
    e = cudaGraphInstantiate(&w->gexec, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    w->gexec = nullptr;
    return e;
  }
  w->gkey = key;
  return cudaSuccess;
}

// Captured loop: stage b and x, replay the graph, read the scalars back once.
cudaError_t pcg_graph(Ctx& c, const double* b, double* x, int& it, int& coarse_iters) {
  Workspace* w = c.w;
  const size_t nt = size_t(c.m->K) * npd(c.m->N) * c.B;
  if (!w->gb) {
    CK(walloc(w, &w->gb, nt));
    CK(walloc(w, &w->gx, nt));
    CK(walloc(w, &w->gctr, size_t(G_NCTR)));
    CK(cudaMallocHost(&w->h_gctr, sizeof(unsigned long long) * G_NCTR));
    for (cudaStream_t& s : w->cap) CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  }
  if (!w->gexec || w->gkey != graph_key(c)) {
    CK(warm_applies(c));
    CK(cudaStreamSynchronize(c.st));
    CK(capture_solve(c, graph_key(c)));
  }
  CK(cudaEventRecord(w->ev0, c.st));
  CK(cudaMemcpyAsync(w->gb, b, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  CK(cudaMemcpyAsync(w->gx, x, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  CK(cudaGraphLaunch(w->gexec, c.st));
  CK(cudaMemcpyAsync(x, w->gx, nt * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
  CK(cudaEventRecord(w->ev1, c.st));
  add_launches(int64_t(w->g_top));
  CK(cudaMemcpyAsync(w->h_gctr, w->gctr, sizeof(unsigned long long) * G_NCTR, cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  add_launches(int64_t(w->h_gctr[G_KERNELS]));
  it = int(w->h_gctr[G_OUTER]);
  coarse_iters = int(w->h_gctr[G_COARSE_TOTAL]);
  return cudaSuccess;
}

// Outer (flexible) PCG. Returns a cudaError_t; solver status in `status`.
cudaError_t pcg_run(Ctx& c, const double* b, double* x, dg_solve_info* info, dg_status& status) {
  CK(setup_workspace(c));
  c.w = c.m->ws;
  Workspace* w = c.w;
  const dg_solver_opts* o = c.o;
  const int B = c.B;
  const int64_t n = int64_t(c.m->K) * npd(c.m->N);
  std::string key;
  if (o->precond == DG_PREC_JACOBI) {
    char buf[48];
    std::snprintf(buf, sizeof buf, "jac/%.17g", c.lambda);
    if (w->dinv_key != buf) {
      CK(launch_diagonal(c.m, c.m->N, DG_F64, c.lambda, w->dinv, c.st));
      k_recip<double><<<egrid(n), 256, 0, c.st>>>(n, w->dinv); note_launch();
      w->dinv_key = buf;
    }
  } else if (o->precond == DG_PREC_PMG) {
    CK(setup_pmg(c, key));
    if (o->coarse_amg) CK(ensure_amg(c, o->degrees[o->nlevels - 1]));
  } else if (o->precond == DG_PREC_AMG) {
    CK(ensure_amg(c, c.m->N));
  }
  int it = 0, coarse_iters = 0;
  if (o->graph) CK(pcg_graph(c, b, x, it, coarse_iters));
  else CK(pcg_eager(c, b, x, it, coarse_iters));
  CK(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, w->ev0, w->ev1));
  status = DG_OK;
  for (int bb = 0; bb < B; ++bb) {
    const double* s = w->h_scal + bb * kNS;
    if (s[S_BREAK] != 0.0) status = DG_ERR_BREAKDOWN;
    else if (s[S_ACTIVE] != 0.0 && status == DG_OK) status = DG_ERR_NOT_CONVERGED;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int bb = 0; bb < B; ++bb) {
      info->iters[bb] = int(w->h_scal[bb * kNS + S_ITERS]);
      info->relres[bb] = w->h_scal[bb * kNS + S_RELRES];
    }
    info->total_iters = it;
    info->ms = ms;
    info->coarse_iters = coarse_iters;
    if (o->precond == DG_PREC_PMG) info->precond_bytes = double(w->pmg_bytes + (o->coarse_amg ? amg_bytes(w->amg) : 0));
    if (o->precond == DG_PREC_AMG) info->precond_bytes = double(amg_bytes(w->amg));
  }
  return cudaSuccess;
}

}  // namespace dgx

using namespace dgx;

extern "C" {

void dg_solver_opts_default(dg_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->max_iter = 1000;
  o->precond = DG_PREC_JACOBI;
  o->nlevels = 0;
  o->cheb_degree = 2;
  o->coarse_tol = 1e-2;
  o->coarse_max_iter = 500;
  o->mixed = 1;
  o->power_steps = 20;
  o->coarse_amg = 0;
  o->graph = 1;
}

dg_status dg_pcg_solve(dg_mesh* m, const dg_solver_opts* o, int B, double lambda, const double* b, double* x,
                       dg_solve_info* info, void* stream) {
  if (!m || !o || !b || !x) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (B < 1 || B > DG_MAX_BATCH) { set_error("batch must be in 1..64"); return DG_ERR_ARG; }
  if (!(o->tol > 0.0) || o->max_iter < 0) { set_error("tol must be > 0 and max_iter >= 0"); return DG_ERR_ARG; }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  if (o->precond < DG_PREC_NONE || o->precond > DG_PREC_AMG) { set_error("unknown preconditioner"); return DG_ERR_ARG; }
  if (o->precond == DG_PREC_INVMASS && !(lambda > 0)) { set_error("inverse-mass preconditioner needs lambda > 0"); return DG_ERR_ARG; }
  if (o->precond == DG_PREC_PMG) {
    if (o->nlevels < 2 || o->nlevels > 8 || o->degrees[0] != m->N) {
      set_error("p-multigrid needs 2..8 levels starting at the mesh degree");
      return DG_ERR_ARG;
    }
    for (int l = 1; l < o->nlevels; ++l)
      if (o->degrees[l] >= o->degrees[l - 1] || o->degrees[l] < 1) {
        set_error("p-multigrid degrees must strictly decrease to >= 1");
        return DG_ERR_ARG;
      }
    if (o->cheb_degree < 1 || o->power_steps < 1 || !(o->coarse_tol > 0) || o->coarse_max_iter < 1) {
      set_error("bad multigrid smoother/coarse options");
      return DG_ERR_ARG;
    }
  }
  try {
    Ctx c{m, o, B, lambda, (cudaStream_t)stream, m->ws};
    dg_status st = DG_OK;
    g_fail_where[0] = 0;
    cudaError_t e = pcg_run(c, b, x, info, st);
    if (e != cudaSuccess) {
      set_error(std::string("dg_pcg_solve: ") + cudaGetErrorString(e) + " at " + g_fail_where);
      return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    }
    if (st == DG_ERR_NOT_CONVERGED) set_error("dg_pcg_solve: max_iter reached before tol");
    if (st == DG_ERR_BREAKDOWN) set_error("dg_pcg_solve: non-positive or non-finite p^T A p or residual");
    return st;
  } catch (const std::exception& ex) {
    set_error(ex.what());
    return DG_ERR_ARG;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free Jacobi-PCG.
//
// Some callers cannot allocate device memory while they run: code that hands
// every byte of the GPU to its own caching allocator or memory pool, code that
// must not hit cudaMalloc's implicit device synchronisation in a time-critical
// loop, or hosts that treat an allocation failure in the middle of a
// simulation as fatal. For them the library keeps a fixed scratch array in
// device memory (a file-scope __device__ array: every GPU that loads the
// library holds it until the process exits) and solves from it without any
// allocation. The mesh itself is still created once, up front, by
// dg_mesh_setup.
namespace dgx {

constexpr size_t kStaticScratchDoubles = size_t(1) << 22;  // 32 MiB per device
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];
static double* g_static_scratch_ptr[64] = {};  // device address, per device ordinal

static size_t align32(size_t n) { return (n + 31) & ~size_t(31); }  // 256-byte steps

// Words of the fixed array one call uses: r, z, p, Ap, the Jacobi inverse, the
// per-right-hand-side scalars and reduction partials, and the apply kernel's
// scratch: the gradient rows of the mma.sync tensor kernels (2 Np per element,
// 3 Np with lambda != 0) or the tcgen05 kernel's rows and face data.
size_t static_scratch_need(const dg_mesh* m, int kernel, int B, bool helm) {
  const int64_t n = int64_t(m->K) * npd(m->N);
  const size_t apply = kernel == DG_KERNEL_TC64 ? tc64_scratch_words(m->N, int64_t(B) * m->K, helm)
                                                : size_t(n) * B * (helm ? 3 : 2) + 1;
  return 4 * align32(size_t(n) * B) + align32(size_t(n)) + align32(size_t(B) * kNS) +
         align32(size_t(B) * kRedBlocks * 2) + align32(apply);
}

}  // namespace dgx

extern "C" dg_status dg_pcg_jacobi_solve_static(const dg_mesh* mc, int B, double lambda, double tol, int max_iter,
                                                const double* b, double* x, dg_solve_info* info, void* stream) {
  using namespace dgx;
  if (!mc || !b || !x) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (B < 1 || B > DG_MAX_BATCH) { set_error("batch must be in 1..64"); return DG_ERR_ARG; }
  if (!(tol > 0.0) || max_iter < 0) { set_error("tol must be > 0 and max_iter >= 0"); return DG_ERR_ARG; }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  const int64_t n = int64_t(m->K) * npd(m->N);
  int kf = m->kern[m->N][0][lambda != 0.0 ? 1 : 0];
  if (kf == DG_KERNEL_AUTO) kf = default_kernel(m->N, true);
  const size_t need = static_scratch_need(m, kf, B, lambda != 0.0);
  if (need > kStaticScratchDoubles) {
    set_error("dg_pcg_jacobi_solve_static: problem needs " + std::to_string(need) +
              " scratch doubles, the static array holds " + std::to_string(kStaticScratchDoubles) +
              " (at B = 1 and degree 8 with the default kernel, K must stay below about 9,200 triangles "
              "for lambda = 0 and 8,400 otherwise)");
    return DG_ERR_ARG;
  }
  if (!m->ops64[m->N].buf) { set_error("mesh operators missing"); return DG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess || dev < 0 || dev >= 64) {
    set_error(std::string("dg_pcg_jacobi_solve_static: cudaGetDevice: ") + cudaGetErrorString(ce));
    return DG_ERR_CUDA;
  }
  // the tensor-core apply's operator slices are built by dg_mesh_setup on the
  // mesh's device; building them here would allocate
  if (((kf == DG_KERNEL_TENSOR || kf == DG_KERNEL_TENSOR_PIPE) && !tensor_ops_ready(m->N, true)) ||
      (kf == DG_KERNEL_TC64 && !tc64_ops_ready(m->N))) {
    set_error("dg_pcg_jacobi_solve_static: the current device is not the one the mesh was set up on");
    return DG_ERR_ARG;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    if (!g_static_scratch_ptr[dev]) {  // one-time set-up on this device (before any stream capture)
      void* sp = nullptr;
      ce = cudaGetSymbolAddress(&sp, g_static_scratch);
      if (ce != cudaSuccess) {
        set_error(std::string("dg_pcg_jacobi_solve_static: cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
        return DG_ERR_CUDA;
      }
      g_static_scratch_ptr[dev] = static_cast<double*>(sp);
    }
    base = g_static_scratch_ptr[dev];
  }
  const size_t nt = size_t(n) * B;
  double* r = base;
  double* z = r + align32(nt);
  double* p = z + align32(nt);
  double* Ap = p + align32(nt);
  double* dinv = Ap + align32(nt);
  double* scal = dinv + align32(size_t(n));
  double* partial = scal + align32(size_t(B) * kNS);
  double* c1 = partial + align32(size_t(B) * kRedBlocks * 2);  // the apply kernel's scratch
  const dim3 g = vgrid(n, B);
#define SCK(expr)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error(std::string("dg_pcg_jacobi_solve_static: ") + cudaGetErrorString(e_));     \
      return DG_ERR_CUDA;                                                                  \
    }                                                                                      \
  } while (0)
  // every scratch word read below is written first in this call, except the
  // per-right-hand-side scalars, which k_init_scal clears
  SCK(launch_diagonal(m, m->N, DG_F64, lambda, dinv, st));
  k_recip<double><<<egrid(n), 256, 0, st>>>(n, dinv); note_launch();
  k_init_scal<<<1, 64, 0, st>>>(B, scal, tol * tol); note_launch();
  k_dot<<<g, kRedThreads, 0, st>>>(n, b, b, partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, st>>>(FIN_INIT_BB, scal, partial); note_launch();
  SCK(launch_apply(m, m->N, DG_F64, B, lambda, x, Ap, st, c1));
  k_sub<double><<<egrid(nt), 256, 0, st>>>(nt, b, Ap, r); note_launch();
  k_dot<<<g, kRedThreads, 0, st>>>(n, r, r, partial); note_launch();
  k_init_check<<<B, kRedThreads, 0, st>>>(scal, partial); note_launch();
  k_scale<double, double><<<egrid(nt), 256, 0, st>>>(n, nt, dinv, r, z); note_launch();
  k_dot<<<g, kRedThreads, 0, st>>>(n, r, z, partial); note_launch();
  k_finalize<<<B, kRedThreads, 0, st>>>(FIN_INIT_RZ, scal, partial); note_launch();
  k_update_p<<<g, kRedThreads, 0, st>>>(n, scal, z, p, 1); note_launch();
  double hs[DG_MAX_BATCH * kNS];
  SCK(cudaMemcpyAsync(hs, scal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  bool any = false;
  for (int k = 0; k < B; ++k) any = any || hs[k * kNS + S_ACTIVE] != 0.0;
  int it = 0;
  while (any && it < max_iter) {
    SCK(launch_apply(m, m->N, DG_F64, B, lambda, p, Ap, st, c1));
    k_dot<<<g, kRedThreads, 0, st>>>(n, p, Ap, partial); note_launch();
    k_finalize<<<B, kRedThreads, 0, st>>>(FIN_ALPHA, scal, partial); note_launch();
    k_update_xr<<<g, kRedThreads, 0, st>>>(n, scal, x, r, p, Ap, nullptr, partial); note_launch();
    k_finalize<<<B, kRedThreads, 0, st>>>(FIN_RR, scal, partial); note_launch();
    ++it;
    if (it % 4 == 0 || it == max_iter) {
      SCK(cudaMemcpyAsync(hs, scal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, st));
      SCK(cudaStreamSynchronize(st));
      any = false;
      for (int k = 0; k < B; ++k) any = any || hs[k * kNS + S_ACTIVE] != 0.0;
      if (!any) break;
    }
    k_scale<double, double><<<egrid(nt), 256, 0, st>>>(n, nt, dinv, r, z); note_launch();
    k_dot<<<g, kRedThreads, 0, st>>>(n, r, z, partial); note_launch();
    k_finalize<<<B, kRedThreads, 0, st>>>(FIN_BETA, scal, partial); note_launch();
    k_update_p<<<g, kRedThreads, 0, st>>>(n, scal, z, p, 0); note_launch();
  }
  SCK(cudaMemcpyAsync(hs, scal, sizeof(double) * B * kNS, cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
#undef SCK
  dg_status status = DG_OK;
  for (int k = 0; k < B; ++k) {
    if (hs[k * kNS + S_BREAK] != 0.0) status = DG_ERR_BREAKDOWN;
    else if (hs[k * kNS + S_ACTIVE] != 0.0 && status == DG_OK) status = DG_ERR_NOT_CONVERGED;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int k = 0; k < B; ++k) {
      info->iters[k] = int(hs[k * kNS + S_ITERS]);
      info->relres[k] = hs[k * kNS + S_RELRES];
    }
    info->total_iters = it;
    info->ms = 0.f;
  }
  if (status == DG_ERR_NOT_CONVERGED) set_error("dg_pcg_jacobi_solve_static: max_iter reached before tol");
  if (status == DG_ERR_BREAKDOWN) set_error("dg_pcg_jacobi_solve_static: Krylov breakdown");
  return status;
}
