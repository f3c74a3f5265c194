// SIPDG apply in FP32 as two register-blocked small GEMMs per element tile
// (included once per degree GA_N).
//
// The bilinear form of Eq. ellipticOp1 in the grouping of Eq. ellipticOp3
// (volume gradient through Dr/Ds, face jumps and averages with the penalty,
// lift through the face mass) is, for a tile of E elements stored as columns:
//
//   C1 (2Np x E)  = [Dr; Ds] U                        reference gradient
//   Y             = [ G.C1 (wr; ws) ; nr F2 ; ns F2 ; F1 ; (lambda J U) ]
//   Au (Np x E)   = [Br Bs | Dr_f^T Ds_f^T | E_f | M] Y
//
// where F1 = sJ Mf(-{n.grad u} - tau [u]) and F2 = 1/2 sJ Mf [u] live on the
// 3(N+1) face nodes, Dr_f / Ds_f are the face-node rows of Dr / Ds (the
// transposed term 1/2 (n.grad l_i, [u])), E_f scatters a face-node value to its
// volume node, Br = Dr^T M, Bs = Ds^T M. Both products run from shared memory
// with register tiles of TI rows x 4 elements per thread, so one operator load
// and one data load feed 4*TI multiply-adds.
//
// The neighbour coupling uses the face buffer written by face_prep: each
// element's own face-node values and outward normal derivatives (a third small
// GEMM with only the face-node rows of Dr, Ds). The operator kernel reads the
// neighbour's pair, reversed along the face and with the derivative's sign
// flipped (opposite normals).
#include "dg_internal.h"

#ifndef GA_N
#error "define GA_N before including apply_gemm.cuh"
#endif

namespace dgx {
namespace GA_NS {

constexpr int N = GA_N;
constexpr int Np = (N + 1) * (N + 2) / 2;
constexpr int Nfp = N + 1;
constexpr int NFN = 3 * Nfp;
constexpr int THREADS = 256;
constexpr int E = 64;                                    // elements per tile
constexpr int TE = 4;                                    // elements per thread tile
constexpr int ET = E / TE;                               // element tiles
constexpr int IT = THREADS / ET;                         // row tiles
constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
constexpr int TI1 = cdiv(2 * Np, IT);                    // rows per thread, gradient GEMM
constexpr int R1 = TI1 * IT;                             // padded rows of [Dr; Ds]
constexpr int TIF = cdiv(2 * NFN, IT);                   // rows per thread, face-prep GEMM
constexpr int RF = TIF * IT;
constexpr int TI3 = cdiv(Np, IT);                        // rows per thread, output GEMM
constexpr int R3 = TI3 * IT;                             // padded output rows
constexpr int al4c(int n) { return (n + 3) & ~3; }
constexpr int TP1 = al4c(TI1), TPF = al4c(TIF), TP3 = al4c(TI3);   // tile rows padded to float4
constexpr int RA1 = IT * TP1, RAF = IT * TPF, RA3 = IT * TP3;       // stored rows per k
constexpr int KP = 2 * Np + 3 * NFN;                     // depth of the output GEMM (Poisson)
constexpr int KH = KP + Np;                              // ... with the screening term
constexpr int LDO = E + 1;                               // output staging stride (conflict-free)

// shared-memory layout (floats); every region starts on a 16-byte boundary
constexpr int al4(int n) { return (n + 3) & ~3; }
constexpr int oOA = 0;                                   // [Np][IT][TP1] [Dr;Ds] by row tile
constexpr int oOB = al4(oOA + Np * RA1);                 // [KH][IT][TP3] output operator by row tile
constexpr int oMF = al4(oOB + KH * RA3);                 // [Nfp][Nfp] face mass
constexpr int oU = al4(oMF + Nfp * Nfp);                 // [Np][E]
constexpr int oY = al4(oU + Np * E);                     // [KH][E]: rows 0..2Np-1 hold C1, then Y
constexpr int oJ = al4(oY + KH * E);                     // [NFN][E] jumps
constexpr int oAV = al4(oJ + NFN * E);                   // [NFN][E] averages
constexpr int oG = al4(oAV + NFN * E);                   // [16][E] per-element geometry
constexpr int oO = al4(oG + E * 16);                     // [Np][LDO] output staging
constexpr int oRaw = al4(oO + Np * LDO);                 // [12][E] raw geometry / connectivity
constexpr int nApply = oRaw + E * 12;
constexpr int oFA = 0;                                   // face_prep: [Np][IT][TPF] face-node rows
constexpr int oFU = al4(oFA + Np * RAF);                 // [Np][E]
constexpr int oFC = al4(oFU + Np * E);                   // [RF][E]
constexpr int oFG = al4(oFC + RF * E);                   // [12][E] raw geometry
constexpr int nPrep = oFG + E * 12;
static_assert(E % TE == 0 && THREADS % ET == 0, "tile shape");
static_assert(R1 >= 2 * Np && RF >= 2 * NFN && R3 >= Np, "padded operators cover all rows");

__host__ __device__ constexpr int row_start(int row) { return row * (N + 1) - row * (row - 1) / 2; }
__host__ __device__ constexpr int fnode(int f, int j) {
  return f == 0 ? j : (f == 1 ? row_start(j) + (N - j) : row_start(N - j));
}

__device__ __forceinline__ void face_vec(float rx, float sx, float ry, float sy, int f, float& gx, float& gy) {
  if (f == 0) { gx = -sx; gy = -sy; }
  else if (f == 1) { gx = rx + sx; gy = ry + sy; }
  else { gx = -rx; gy = -ry; }
}

// C[r][e] (+)= sum_k A[k][r] X[k][e] for the thread's TI x 4 tile (rows
// r = ti*TI + t). A: operator stored per k as IT row tiles of TP (>= TI, a
// multiple of 4) entries, so the thread's TI entries are TP/4 aligned float4
// loads; X: [K][E] tile data, one float4 per k.
template <int TI, int TP>
__device__ __forceinline__ void mma_tile(const float* __restrict__ A, const float* __restrict__ X, int K, int ti,
                                         int e0, float (&acc)[TI][TE]) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 x = *reinterpret_cast<const float4*>(X + k * E + e0);
    const float4* a4 = reinterpret_cast<const float4*>(A + (k * IT + ti) * TP);
    float av[TP];
#pragma unroll
    for (int v = 0; v < TP / 4; ++v) {
      const float4 t4 = a4[v];
      av[4 * v + 0] = t4.x;
      av[4 * v + 1] = t4.y;
      av[4 * v + 2] = t4.z;
      av[4 * v + 3] = t4.w;
    }
#pragma unroll
    for (int t = 0; t < TI; ++t) {
      acc[t][0] = fmaf(av[t], x.x, acc[t][0]);
      acc[t][1] = fmaf(av[t], x.y, acc[t][1]);
      acc[t][2] = fmaf(av[t], x.z, acc[t][2]);
      acc[t][3] = fmaf(av[t], x.w, acc[t][3]);
    }
  }
}

// Per-thread register prefetch of a tile: nodal values (as U[m][e] items),
// geometry, connectivity and the per-face inverse length scale. Issued for the
// next tile while the current one computes, committed to shared memory after.
constexpr int PU = cdiv(Np * E, THREADS);
constexpr int PFI = cdiv(NFN * E, THREADS);

struct Prefetch {
  float u[PU];
  float4 g;
  int c[3];
  float ih[3];
};

__device__ __forceinline__ void issue(Prefetch& p, const float* __restrict__ u, const float* __restrict__ geo,
                                      const int32_t* __restrict__ conn, const float* __restrict__ ih, int64_t K,
                                      int64_t w, int64_t nwork, int64_t ntiles) {
  if (w >= nwork) return;
  const int b = int(w / ntiles);
  const int64_t eb = (w - int64_t(b) * ntiles) * E;
  const int ne = int((K - eb) < E ? (K - eb) : E);
  const float* src = u + (size_t(b) * K + eb) * Np;
#pragma unroll
  for (int r = 0; r < PU; ++r) {
    const int idx = threadIdx.x + r * THREADS;
    const int m = idx / E, e = idx - m * E;
    p.u[r] = (idx < Np * E && e < ne) ? __ldg(src + size_t(e) * Np + m) : 0.f;
  }
  const int t = threadIdx.x;
  if (t < ne) {
    p.g = __ldg(reinterpret_cast<const float4*>(geo) + eb + t);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      p.c[f] = __ldg(conn + 3 * (eb + t) + f);
      p.ih[f] = ih ? __ldg(ih + 3 * (eb + t) + f) : 0.f;
    }
  } else {
    p.g = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      p.c[f] = -3;
      p.ih[f] = 0.f;
    }
  }
}

// raw per-element record in shared memory, field-major [RAW][E]:
// rx sx ry sy | c0 c1 c2 | ih0 ih1 ih2
constexpr int RAW = 12;

__device__ __forceinline__ void commit(const Prefetch& p, float* U, float* Raw) {
#pragma unroll
  for (int r = 0; r < PU; ++r) {
    const int idx = threadIdx.x + r * THREADS;
    if (idx < Np * E) U[idx] = p.u[r];
  }
  const int t = threadIdx.x;
  if (t < E) {
    Raw[0 * E + t] = p.g.x;
    Raw[1 * E + t] = p.g.y;
    Raw[2 * E + t] = p.g.z;
    Raw[3 * E + t] = p.g.w;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      Raw[(4 + f) * E + t] = __int_as_float(p.c[f]);
      Raw[(7 + f) * E + t] = p.ih[f];
    }
  }
}

__global__ void __launch_bounds__(THREADS) face_prep_g(int64_t K, int B, const float* __restrict__ geo,
                                                       const int32_t* __restrict__ conn,
                                                       const float* __restrict__ ops,
                                                       const float* __restrict__ u, float2* __restrict__ face) {
  extern __shared__ __align__(16) float smg[];
  float* FA = smg + oFA;
  float* U = smg + oFU;
  float* C = smg + oFC;
  float* Raw = smg + oFG;
  for (int idx = threadIdx.x; idx < Np * RAF; idx += THREADS) FA[idx] = ops[idx];
  const int ti = threadIdx.x / ET, te = threadIdx.x - ti * ET;
  const int64_t ntiles = (K + E - 1) / E;
  const int64_t nwork = ntiles * B;
  Prefetch pf;
  issue(pf, u, geo, conn, nullptr, K, blockIdx.x, nwork, ntiles);
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int b = int(w / ntiles);
    const int64_t eb = (w - int64_t(b) * ntiles) * E;
    const int ne = int((K - eb) < E ? (K - eb) : E);
    __syncthreads();
    commit(pf, U, Raw);
    __syncthreads();
    issue(pf, u, geo, conn, nullptr, K, w + gridDim.x, nwork, ntiles);
    float acc[TIF][TE] = {};
    mma_tile<TIF, TPF>(FA, U, Np, ti, te * TE, acc);
#pragma unroll
    for (int t = 0; t < TIF; ++t)
#pragma unroll
      for (int c = 0; c < TE; ++c) C[(ti * TIF + t) * E + te * TE + c] = acc[t][c];
    __syncthreads();
    float2* fo = face + (size_t(b) * K + eb) * NFN;
    for (int idx = threadIdx.x; idx < ne * NFN; idx += THREADS) {
      const int e = idx / NFN, q = idx - e * NFN, f = q / Nfp, j = q - f * Nfp;
      const float rx = Raw[e], sx = Raw[E + e], ry = Raw[2 * E + e], sy = Raw[3 * E + e];
      float gx, gy;
      face_vec(rx, sx, ry, sy, f, gx, gy);
      const float gn = sqrtf(gx * gx + gy * gy);
      const float nx = gx / gn, ny = gy / gn;
      const float d = (nx * rx + ny * ry) * C[q * E + e] + (nx * sx + ny * sy) * C[(NFN + q) * E + e];
      fo[idx] = make_float2(U[fnode(f, j) * E + e], d);
    }
  }
}

template <bool HELM>
__global__ void __launch_bounds__(THREADS, 1) apply_g(int64_t K, int B, const float* __restrict__ geo,
                                                   const int32_t* __restrict__ conn, const float* __restrict__ ihf,
                                                   const float* __restrict__ ops, const float* __restrict__ u,
                                                   const float2* __restrict__ face, float lambda,
                                                   float* __restrict__ Au) {
  extern __shared__ __align__(16) float smg[];
  float* OA = smg + oOA;
  float* OB = smg + oOB;
  float* MF = smg + oMF;
  float* U = smg + oU;
  float* Y = smg + oY;
  float* Jm = smg + oJ;
  float* Av = smg + oAV;
  float* Gs = smg + oG;
  float* O = smg + oO;
  float* Raw = smg + oRaw;
  constexpr int KD = HELM ? KH : KP;
  constexpr float cpen = float((N + 1) * (N + 2)) / 2.0f;
  for (int idx = threadIdx.x; idx < Np * RA1; idx += THREADS) OA[idx] = ops[Np * RAF + idx];
  for (int idx = threadIdx.x; idx < KD * RA3; idx += THREADS) OB[idx] = ops[Np * RAF + Np * RA1 + idx];
  for (int idx = threadIdx.x; idx < Nfp * Nfp; idx += THREADS)
    MF[idx] = ops[Np * RAF + Np * RA1 + KH * RA3 + idx];
  const int ti = threadIdx.x / ET, te = threadIdx.x - ti * ET;
  const int64_t ntiles = (K + E - 1) / E;
  const int64_t nwork = ntiles * B;
  Prefetch pf;
  issue(pf, u, geo, conn, ihf, K, blockIdx.x, nwork, ntiles);
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int b = int(w / ntiles);
    const int64_t eb = (w - int64_t(b) * ntiles) * E;
    const int ne = int((K - eb) < E ? (K - eb) : E);
    __syncthreads();
    commit(pf, U, Raw);
    __syncthreads();
    issue(pf, u, geo, conn, ihf, K, w + gridDim.x, nwork, ntiles);
    // neighbour face data for this tile: gathers issued before the gradient GEMM
    const float2* fb = face + size_t(b) * K * NFN;
    float2 nbv[PFI];
#pragma unroll
    for (int r = 0; r < PFI; ++r) {
      const int idx = threadIdx.x + r * THREADS;
      const int q = idx / E, e = idx - q * E;
      nbv[r] = make_float2(0.f, 0.f);
      if (idx < NFN * E && e < ne) {
        const int f = q / Nfp, j = q - f * Nfp;
        const int c = __float_as_int(Raw[(4 + f) * E + e]);
        if (c >= 0) nbv[r] = __ldg(fb + size_t(c >> 2) * NFN + (c & 3) * Nfp + (Nfp - 1 - j));
      }
    }
    // per-element geometry, field-major [16][E]: Grr Grs Gss J | per face (nr ns sJ tau)
    for (int e = threadIdx.x; e < E; e += THREADS) {
      if (e >= ne) {
        for (int k = 0; k < 16; ++k) Gs[k * E + e] = 0.f;
        continue;
      }
      const float rx = Raw[e], sx = Raw[E + e], ry = Raw[2 * E + e], sy = Raw[3 * E + e];
      const float J = 1.0f / (rx * sy - ry * sx);
      Gs[0 * E + e] = J * (rx * rx + ry * ry);
      Gs[1 * E + e] = J * (rx * sx + ry * sy);
      Gs[2 * E + e] = J * (sx * sx + sy * sy);
      Gs[3 * E + e] = J;
      for (int f = 0; f < 3; ++f) {
        float gx, gy;
        face_vec(rx, sx, ry, sy, f, gx, gy);
        const float gn = sqrtf(gx * gx + gy * gy);
        const float nx = gx / gn, ny = gy / gn;
        Gs[(4 + 4 * f + 0) * E + e] = nx * rx + ny * ry;
        Gs[(4 + 4 * f + 1) * E + e] = nx * sx + ny * sy;
        Gs[(4 + 4 * f + 2) * E + e] = J * gn;
        Gs[(4 + 4 * f + 3) * E + e] = cpen * Raw[(7 + f) * E + e];
      }
    }
    // C1 = [Dr; Ds] U  -> Y rows 0 .. 2Np-1 (ur, us)
    {
      float acc[TI1][TE] = {};
      mma_tile<TI1, TP1>(OA, U, Np, ti, te * TE, acc);
#pragma unroll
      for (int t = 0; t < TI1; ++t) {
        const int r = ti * TI1 + t;
        if (r < 2 * Np) *reinterpret_cast<float4*>(Y + r * E + te * TE) =
            make_float4(acc[t][0], acc[t][1], acc[t][2], acc[t][3]);
      }
    }
    __syncthreads();
    // jumps and averages at the face nodes (needs ur, us before they become wr, ws)
#pragma unroll
    for (int r = 0; r < PFI; ++r) {
      const int idx = threadIdx.x + r * THREADS;
      if (idx >= NFN * E) break;
      const int q = idx / E, e = idx - q * E;
      const int f = q / Nfp, j = q - f * Nfp, k = fnode(f, j);
      float jm = 0.f, av = 0.f;
      if (e < ne) {
        const float* g = Gs + (4 + 4 * f) * E + e;
        const float um = U[k * E + e];
        const float dnm = g[0] * Y[k * E + e] + g[E] * Y[(Np + k) * E + e];
        const int c = __float_as_int(Raw[(4 + f) * E + e]);
        if (c >= 0) {
          jm = nbv[r].x - um;
          av = 0.5f * (dnm - nbv[r].y);
        } else if (c == -2) {
          jm = -2.0f * um;
          av = dnm;
        }
      }
      Jm[idx] = jm;
      Av[idx] = av;
    }
    __syncthreads();
    // Y rows: wr, ws (in place), nr F2, ns F2, F1, lambda J u
    for (int idx = threadIdx.x; idx < Np * E; idx += THREADS) {
      const int i = idx / E, e = idx - i * E;
      const float* g = Gs + e;
      const float ur = Y[i * E + e], us = Y[(Np + i) * E + e];
      Y[i * E + e] = g[0] * ur + g[E] * us;
      Y[(Np + i) * E + e] = g[E] * ur + g[2 * E] * us;
      if (HELM) Y[(KP + i) * E + e] = lambda * g[3 * E] * U[i * E + e];
    }
    for (int idx = threadIdx.x; idx < NFN * E; idx += THREADS) {
      const int q = idx / E, e = idx - q * E;
      const int f = q / Nfp, j = q - f * Nfp;
      const float* g = Gs + (4 + 4 * f) * E + e;
      const float tau = g[3 * E], sJ = g[2 * E];
      float m1 = 0.f, m2 = 0.f;
#pragma unroll
      for (int l = 0; l < Nfp; ++l) {
        const float mf = MF[j * Nfp + l];
        const float jl = Jm[(f * Nfp + l) * E + e];
        m1 = fmaf(mf, Av[(f * Nfp + l) * E + e] + tau * jl, m1);
        m2 = fmaf(mf, jl, m2);
      }
      const float f2 = 0.5f * sJ * m2;
      Y[(2 * Np + q) * E + e] = g[0] * f2;
      Y[(2 * Np + NFN + q) * E + e] = g[E] * f2;
      Y[(2 * Np + 2 * NFN + q) * E + e] = -sJ * m1;
    }
    __syncthreads();
    // Au = OB Y
    {
      float acc[TI3][TE] = {};
      mma_tile<TI3, TP3>(OB, Y, KD, ti, te * TE, acc);
#pragma unroll
      for (int t = 0; t < TI3; ++t) {
        const int r = ti * TI3 + t;
        if (r < Np)
#pragma unroll
          for (int c = 0; c < TE; ++c) O[r * LDO + te * TE + c] = acc[t][c];
      }
    }
    __syncthreads();
    float* dst = Au + (size_t(b) * K + eb) * Np;
    for (int idx = threadIdx.x; idx < ne * Np; idx += THREADS) {
      const int e = idx / Np, i = idx - e * Np;
      dst[idx] = O[i * LDO + e];
    }
  }
}

// Host: operator buffer [face-prep rows | [Dr;Ds] | output operator | Mf], all
// column-major with zero-padded rows.
std::vector<float> build_ops(const RefElem& R) {
  std::vector<float> h(size_t(Np) * RAF + size_t(Np) * RA1 + size_t(KH) * RA3 + Nfp * Nfp, 0.f);
  float* FA = h.data();
  float* OA = FA + size_t(Np) * RAF;
  float* OB = OA + size_t(Np) * RA1;
  float* MF = OB + size_t(KH) * RA3;
  // entry (k, row) of an operator stored by row tiles of TI rows padded to TP
  auto at = [](float* A, int TI, int TP, int k, int row) -> float& {
    return A[(k * IT + row / TI) * TP + row % TI];
  };
  for (int m = 0; m < Np; ++m)
    for (int q = 0; q < NFN; ++q) {
      const int k = fnode(q / Nfp, q % Nfp);
      at(FA, TIF, TPF, m, q) = float(R.Dr[size_t(k) * Np + m]);
      at(FA, TIF, TPF, m, NFN + q) = float(R.Ds[size_t(k) * Np + m]);
    }
  for (int m = 0; m < Np; ++m)
    for (int i = 0; i < Np; ++i) {
      at(OA, TI1, TP1, m, i) = float(R.Dr[size_t(i) * Np + m]);
      at(OA, TI1, TP1, m, Np + i) = float(R.Ds[size_t(i) * Np + m]);
    }
  for (int i = 0; i < Np; ++i) {
    for (int m = 0; m < Np; ++m) {
      at(OB, TI3, TP3, m, i) = float(R.Br[size_t(i) * Np + m]);
      at(OB, TI3, TP3, Np + m, i) = float(R.Bs[size_t(i) * Np + m]);
      at(OB, TI3, TP3, KP + m, i) = float(R.M[size_t(i) * Np + m]);
    }
    for (int q = 0; q < NFN; ++q) {
      const int k = fnode(q / Nfp, q % Nfp);
      at(OB, TI3, TP3, 2 * Np + q, i) = float(R.Dr[size_t(k) * Np + i]);
      at(OB, TI3, TP3, 2 * Np + NFN + q, i) = float(R.Ds[size_t(k) * Np + i]);
      at(OB, TI3, TP3, 2 * Np + 2 * NFN + q, i) = (k == i) ? 1.f : 0.f;
    }
  }
  for (int j = 0; j < Nfp * Nfp; ++j) MF[j] = float(R.Mf[j]);
  return h;
}

struct Cfg {
  float* ops = nullptr;
  int grid_prep = 0, grid_p = 0, grid_h = 0;
};

cudaError_t launch(const dg_mesh* m, int B, double lambda, const float* u, float* Au, float2* face,
                   cudaStream_t st) {
  static Cfg cfg[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  Cfg& c = cfg[dev];
  constexpr size_t smP = sizeof(float) * nPrep;
  constexpr size_t smA = sizeof(float) * nApply;
  std::unique_lock<std::mutex> lk(table_mutex());
  if (!c.ops) {
    const RefElem R = m->ref[N].N ? m->ref[N] : build_reference(N);
    const std::vector<float> h = build_ops(R);
    float* d = nullptr;
    e = cudaMalloc(&d, h.size() * sizeof(float));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    int sms = 0, a = 0, p = 0, hh = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(face_prep_g, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smP));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(apply_g<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smA));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(apply_g<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smA));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, face_prep_g, THREADS, smP);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, apply_g<false>, THREADS, smA);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&hh, apply_g<true>, THREADS, smA);
    if (e != cudaSuccess) return e;
    c.grid_prep = sms * (a > 0 ? a : 1);
    c.grid_p = sms * (p > 0 ? p : 1);
    c.grid_h = sms * (hh > 0 ? hh : 1);
    c.ops = d;
  }
  lk.unlock();
  const int64_t work = ((m->K + E - 1) / E) * B;
  auto clampg = [work](int g) { return int(work < g ? work : g); };
  face_prep_g<<<clampg(c.grid_prep), THREADS, smP, st>>>(m->K, B, m->geo32, m->conn, c.ops, u, face);
  note_launch();
  if (lambda != 0.0) {
    apply_g<true><<<clampg(c.grid_h), THREADS, smA, st>>>(m->K, B, m->geo32, m->conn, m->ih32, c.ops, u, face,
                                                          float(lambda), Au);
  } else {
    apply_g<false><<<clampg(c.grid_p), THREADS, smA, st>>>(m->K, B, m->geo32, m->conn, m->ih32, c.ops, u, face,
                                                           0.f, Au);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace GA_NS
}  // namespace dgx
