// SIPDG apply in FP32 on the Blackwell tensor cores (tcgen05, tensor memory,
// bulk copies), the operator of Eq. ellipticOp3 written as two dense products
// per element (as in apply_tensor.cu):
//   C1 = [Dr; Ds] u                         (gradient product, + M u for Helmholtz)
//   Au = OB Y (+ lambda J M u)              (output product)
// with Y = [wr, ws | 1/2 nr sJ [u], 1/2 ns sJ [u], -sJ ({n.grad u} + tau [u])]
// the pointwise stage of Section 5.2 (wr = Grr ur + Grs us, ws = Grs ur + Gss us,
// jumps and averages at the face nodes, penalty of Eq. PenaltyParameter) and
// OB = [Br Bs | Dr_f^T Mf Ds_f^T Mf | E_f Mf] the transposed derivative and
// lift operators with the face mass folded in.
//
// Precision: FP32-level. Every operand is split into two FP16 pieces (hi and
// the FP16 rounding of the remainder, 22 significant bits) after scaling by a
// power of two that keeps it in FP16 range: operator rows on the host, each
// element's data row on the device. The products hi*hi + hi*lo + lo*hi are
// accumulated in FP32 in tensor memory; the dropped lo*lo term and the
// representation error are near 2^-21 of |A||x|.
//
// Two kernels per apply:
//  * tc_face: the gradient product restricted to the face-node rows; writes
//    every element's face traces and outward normal derivatives (u, n.grad u)
//    at its face nodes, [B][K][3][N+1] float2, which the neighbours read.
//  * tc_apply: one 128-element tile per step: bulk copy of the tile's u rows
//    into shared memory (the next tile's copy in flight meanwhile), FP16
//    pieces of u into tensor memory, gradient product, the pointwise stage
//    written as FP16 pieces of Y into tensor memory, output product, epilogue
//    through shared memory to coalesced stores. Four threads per element
//    (512 threads, warps w, w+4, w+8, w+12 share the element's tensor-memory
//    lane): two take the volume columns of half the nodes each, two take the
//    face columns. Operator pieces stay in shared memory for the whole launch.
// One thread issues the MMAs (M = 128 elements, A from tensor memory, B from
// shared memory); completion reaches the other threads through mbarriers
// whose waits are bounded (a timeout sets an error flag, read by
// dg_tensor_timeouts, and ends the kernel).
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dg_internal.h"
#include "tc05.cuh"

namespace dgx {
namespace {

constexpr int kTile = 128;  // elements per tile = MMA rows = tensor-memory lanes

constexpr int rup16(int x) { return (x + 15) / 16 * 16; }
constexpr int rup8(int x) { return (x + 7) / 8 * 8; }
constexpr int rup128(int x) { return (x + 127) / 128 * 128; }

template <int N>
struct Tc {
  static constexpr int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  static constexpr int K1 = rup16(Np);       // depth of the gradient product
  static constexpr int N1 = rup16(3 * Np);   // rows [Dr; Ds; M]
  static constexpr int NP1 = rup16(2 * Np);  // rows the Poisson form uses
  static constexpr int NF = rup16(2 * NFN);  // face kernel: [Dr; Ds] rows of the face-node entries
  static constexpr int V0 = (Np + 1) / 2;    // nodes of volume half 0 (half 1 has Np - V0)
  static constexpr int VL = rup8(V0);        // tensor-memory columns loaded per volume half
  static constexpr int VB = rup16(2 * V0);   // Y columns of one volume half (wr at 0.., ws at V0..)
  static constexpr int FB2 = rup16(6 * Nfp);  // Y columns of faces 0 and 1
  static constexpr int FB3 = rup16(3 * Nfp);  // Y columns of face 2
  static constexpr int KY = 2 * VB + FB2 + FB3;
  static constexpr int N2 = rup16(Np);  // output rows
  static constexpr int RQ = N2 / 4;     // output rows per thread of an element
  static constexpr int YMAX = VB > FB2 ? VB : FB2;
  // tensor-memory columns of tc_apply
  static constexpr int oA1 = 0, oD1 = K1, oA2 = oD1 + N1, oD2 = oA2 + KY, TCOLS = oD2 + N2;
  static_assert(TCOLS <= 512, "tensor memory");
  // operator image (bytes): tc_apply part [B1 hi | B1 lo | B2 hi | B2 lo | isc1 | isc2],
  // tc_face part [BF hi | BF lo | iscF]
  static constexpr int szB1 = N1 * K1 * 2, szB2 = N2 * KY * 2, szBF = NF * K1 * 2;
  static constexpr int opsA = 2 * szB1 + 2 * szB2 + 4 * (N1 + N2);  // a multiple of 16
  static constexpr int opsF = 2 * szBF + 4 * NF;
  static_assert(opsA % 16 == 0 && opsF % 16 == 0, "bulk copy sizes");
  static constexpr int utile = kTile * Np * 4;  // bytes of one FP32 u tile
  // shared memory of tc_apply
  static constexpr int smA_ut = rup128(opsA);
  static constexpr int smA_pmax = smA_ut + 2 * utile;
  static constexpr int smA_bar = smA_pmax + 6 * kTile * 4;
  static constexpr int smA = smA_bar + 8 * 8;
  // shared memory of tc_face
  static constexpr int smF_ut = rup128(opsF);
  static constexpr int smF_stg = smF_ut + 2 * utile;       // [kTile][NFN] float2 face data
  static constexpr int smF_bar = smF_stg + rup128(kTile * NFN * 8);
  static constexpr int smF = smF_bar + 8 * 8;
};

__device__ int g_tc05_err;

__device__ __forceinline__ int tile_len(int64_t nE, int64_t e0) { return nE - e0 < kTile ? int(nE - e0) : kTile; }

__device__ __forceinline__ int fnode(int N, int f, int j) {
  auto rs = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

// FP16 pieces of a pair of scaled values: hi = fp16(x), lo = fp16(x - hi);
// k even in the low half of the 32-bit column, k odd in the high half
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Scale exponent for a row whose largest magnitude is mx: 2^s mx < 2^14 (and
// FP16 range). Clamped to 127, so rows below about 1e-34 keep fewer bits.
__device__ __forceinline__ int scale_exp(float mx) {
  const int em = tc::exp_of(mx);
  return em == -200 ? 0 : min(14 - em, 127);
}
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((127 + s) << 23); }  // s in [-126, 127]

// one bulk copy of the element rows [e0, e0 + ne) of u into a tile buffer, armed on
// `bar`; bytes beyond the last multiple of 16 are left to plain loads (fix_tail)
__device__ __forceinline__ void issue_tile(const float* u, int Np, int64_t e0, int ne, float* dst, uint64_t* bar) {
  const uint32_t bytes = uint32_t(ne) * uint32_t(Np) * 4u;
  const uint32_t bulk = bytes & ~15u;
  tc::mbar_expect_tx(bar, bulk);
  if (bulk) tc::bulk_g2s(dst, u + e0 * Np, bulk, bar);
}
__device__ __forceinline__ void fix_tail(const float* u, int Np, int64_t e0, int ne, float* dst) {
  const int n = ne * Np, b = n & ~3;
  for (int i = b + int(threadIdx.x); i < n; i += blockDim.x) dst[i] = u[e0 * Np + i];
}

// -------------------------------------------------------------------------------
// Face data: FN[be][f][j] = (u, n.grad u) at face node j of face f (counter-clockwise),
// with the element's own outward normal. One thread per element; the tile's
// face data go through shared memory to coalesced stores.
template <int N>
__global__ void __launch_bounds__(kTile) tc_face(int64_t K, int64_t nE, const float* __restrict__ gx,
                                                 const float* __restrict__ u, const uint8_t* __restrict__ opsF,
                                                 float2* __restrict__ FN) {
  using S = Tc<N>;
  constexpr int Np = S::Np, Nfp = S::Nfp, NFN = S::NFN, K1 = S::K1, NF = S::NF;
  extern __shared__ __align__(128) uint8_t sm[];
  const uint8_t* sBF = sm;
  const float* iscF = reinterpret_cast<const float*>(sm + 2 * S::szBF);
  float* ut = reinterpret_cast<float*>(sm + S::smF_ut);
  float2* stg = reinterpret_cast<float2*>(sm + S::smF_stg);  // [kTile][NFN]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::smF_bar);  // op, u0, u1, mma
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 4);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t lanebase = uint32_t(warp * 32) << 16;
  const int64_t ntiles = (nE + kTile - 1) / kTile;
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(bars + i, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(slot, 128);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = *slot;
  if (tid == 0) {
    tc::mbar_expect_tx(bars, S::opsF);
    tc::bulk_g2s(sm, opsF, S::opsF, bars);
    if (int64_t(blockIdx.x) < ntiles) {
      const int64_t e0 = int64_t(blockIdx.x) * kTile;
      issue_tile(u, Np, e0, tile_len(nE, e0), ut, bars + 1);
    }
  }
  if (!tc::mbar_wait(bars, 0)) *abort_flag = 1;
  constexpr uint32_t idesc = tc::idesc_f16(128, NF, false);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    const int64_t e0 = tile * kTile;
    const int ne = tile_len(nE, e0);
    float* cur = ut + buf * (kTile * Np);
    const int e = tid;
    const bool live = e < ne;
    const int64_t el = (e0 + e) % K;
    // the face normals, loaded while the tile and the products are in flight
    float nrm[6];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      nrm[2 * f] = live ? __ldg(gx + 16 * el + 4 + 4 * f) : 0.f;
      nrm[2 * f + 1] = live ? __ldg(gx + 16 * el + 5 + 4 * f) : 0.f;
    }
    if (!tc::mbar_wait(bars + 1 + buf, (it >> 1) & 1)) *abort_flag = 1;
    if (tid == 0 && tile + gridDim.x < ntiles) {
      const int64_t e1 = (tile + gridDim.x) * kTile;
      issue_tile(u, Np, e1, tile_len(nE, e1), ut + (buf ^ 1) * (kTile * Np), bars + 2 - buf);
    }
    if (ne < kTile) fix_tail(u, Np, e0, ne, cur);
    __syncthreads();
    if (*abort_flag) break;
    const float* urow = cur + e * Np;
    // FP16 pieces of the element's scaled u row into tensor memory
    float mx = 0.f;
    if (live)
      for (int k = 0; k < Np; ++k) mx = fmaxf(mx, fabsf(urow[k]));
    const int s1 = scale_exp(mx);
    const float f1 = pow2f(s1);
#pragma unroll
    for (int c0 = 0; c0 < K1 / 2; c0 += 8) {
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = 2 * (c0 + c);
        const float a = (live && k < Np) ? urow[k] * f1 : 0.f;
        const float b = (live && k + 1 < Np) ? urow[k + 1] * f1 : 0.f;
        split_pair(a, b, hi[c], lo[c]);
      }
      tc::tmem_st8(tb + lanebase + c0, hi);
      tc::tmem_st8(tb + lanebase + K1 / 2 + c0, lo);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      uint32_t acc = 0;
#pragma unroll
      for (int ks = 0; ks < K1 / 16; ++ks) {
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {  // (hi, hi), (hi, lo), (lo, hi)
          const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
          const uint64_t bd = tc::smem_desc(tc::smem_addr(sBF) + pb * S::szBF + ks * 256, 128, (K1 / 8) * 128);
          tc::mma_ts(tb + K1, tb + pa * (K1 / 2) + ks * 8, bd, idesc, acc);
          acc = 1;
        }
      }
      tc::mma_commit(bars + 3);
    }
    if (!tc::mbar_wait(bars + 3, it & 1)) *abort_flag = 1;
    tc::fence_after();
    // outward normal derivatives at the face nodes from the face rows of D
    uint32_t d[NF];
#pragma unroll
    for (int c0 = 0; c0 < NF; c0 += 8) {
      uint32_t v[8];
      tc::tmem_ld8(tb + lanebase + K1 + c0, v);
#pragma unroll
      for (int c = 0; c < 8; ++c) d[c0 + c] = v[c];
    }
    tc::tmem_wait_ld();
    if (live) {
      const float isc = tc::ldexp2(1.0f, -s1);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
#pragma unroll
        for (int j = 0; j < Nfp; ++j) {
          const int rr = f * Nfp + j;
          const float dr = __uint_as_float(d[rr]) * iscF[rr];
          const float ds = __uint_as_float(d[NFN + rr]) * iscF[NFN + rr];
          stg[e * NFN + rr] = make_float2(urow[fnode(N, f, j)], (nrm[2 * f] * dr + nrm[2 * f + 1] * ds) * isc);
        }
      }
    }
    __syncthreads();
    {
      const int n = ne * NFN;  // float2 entries of the tile, contiguous in FN
      float2* dst = FN + e0 * NFN;
      if ((n & 1) == 0 && ((e0 * NFN) & 1) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(stg);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int i = tid; i < n / 2; i += kTile) d4[i] = s4[i];
      } else {
        for (int i = tid; i < n; i += kTile) dst[i] = stg[i];
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  }
  if (*abort_flag && tid == 0) atomicExch(&g_tc05_err, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tb, 128);
}

// -------------------------------------------------------------------------------
// The face columns of one face f for the element: Y[base + j], Y[base + Nfp + j],
// Y[base + 2 Nfp + j] from the element's own gradient at the face nodes (dr, ds:
// tensor-memory words), its trace, and the neighbour's face data p.
template <int N, int BASE, int YN>
__device__ __forceinline__ void face_columns(float (&y)[YN], const uint32_t (&dr)[N + 1], const uint32_t (&ds)[N + 1],
                                             const float2 (&p)[N + 1], int f, int code, const float* g,
                                             const float* urow, const float* isc1, float iu, float cpen) {
  constexpr int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1;
  const float nr = __ldg(g + 4 + 4 * f), ns = __ldg(g + 5 + 4 * f), sJ = __ldg(g + 6 + 4 * f);
  const float tau = cpen * __ldg(g + 7 + 4 * f);
#pragma unroll
  for (int j = 0; j < Nfp; ++j) {
    const int kf = fnode(N, f, j);
    const float um = urow[kf];
    const float dnm = (nr * (__uint_as_float(dr[j]) * isc1[kf]) + ns * (__uint_as_float(ds[j]) * isc1[Np + kf])) * iu;
    float jm = 0.f, av = 0.f;
    if (code >= 0) {
      jm = p[j].x - um;
      av = 0.5f * (dnm - p[j].y);
    } else if (code == -2) {  // Dirichlet
      jm = -2.f * um;
      av = dnm;
    }
    const float hs = 0.5f * sJ * jm;
    y[BASE + j] = nr * hs;
    y[BASE + Nfp + j] = ns * hs;
    y[BASE + 2 * Nfp + j] = -sJ * (av + tau * jm);
  }
}

template <int N>
__device__ __forceinline__ void load_face(uint32_t tb, uint32_t lanebase, int oD1, int f, uint32_t (&dr)[N + 1],
                                          uint32_t (&ds)[N + 1]) {
  constexpr int Np = (N + 1) * (N + 2) / 2;
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const int kf = fnode(N, f, j);
    tc::tmem_ld1(tb + lanebase + oD1 + kf, dr[j]);
    tc::tmem_ld1(tb + lanebase + oD1 + Np + kf, ds[j]);
  }
}

// neighbour's face data across face f in the element's own node order
template <int N>
__device__ __forceinline__ void load_nb(const float2* FN, int64_t boff, int code, bool live, float2 (&p)[N + 1]) {
  constexpr int Nfp = N + 1, NFN = 3 * Nfp;
  if (live && code >= 0) {
    const float2* fnb = FN + (boff + (code >> 2)) * NFN + (code & 3) * Nfp;
#pragma unroll
    for (int j = 0; j < Nfp; ++j) p[j] = __ldg(fnb + (Nfp - 1 - j));
  } else {
#pragma unroll
    for (int j = 0; j < Nfp; ++j) p[j] = make_float2(0.f, 0.f);
  }
}

// FP16 pieces of Y columns [0, L) of this quarter into tensor memory at
// column offset c (of piece hi; piece lo KY/2 further)
template <int L, int YN>
__device__ __forceinline__ void store_y(const float (&y)[YN], float f2, uint32_t addr, uint32_t lo_off) {
#pragma unroll
  for (int c0 = 0; c0 < L / 2; c0 += 8) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) split_pair(y[2 * (c0 + c)] * f2, y[2 * (c0 + c) + 1] * f2, hi[c], lo[c]);
    tc::tmem_st8(addr + c0, hi);
    tc::tmem_st8(addr + lo_off + c0, lo);
  }
}

template <int L, int YN>
__device__ __forceinline__ float absmax(const float (&y)[YN]) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < L; ++j) m = fmaxf(m, fabsf(y[j]));
  return m;
}

// The whole apply of one tile per step (see the file comment).
template <int N, bool HELM>
__global__ void __launch_bounds__(512, 1) tc_apply(int64_t K, int64_t nE, const float* __restrict__ gx,
                                                   const int32_t* __restrict__ conn,
                                                   const float2* __restrict__ FN, const float* __restrict__ u,
                                                   const uint8_t* __restrict__ opsA, float lambda,
                                                   float* __restrict__ out) {
  using S = Tc<N>;
  constexpr int Np = S::Np, Nfp = S::Nfp, K1 = S::K1, KY = S::KY, V0 = S::V0, VB = S::VB;
  extern __shared__ __align__(128) uint8_t sm[];
  const uint8_t* sB1 = sm;
  const uint8_t* sB2 = sm + 2 * S::szB1;
  const float* isc1 = reinterpret_cast<const float*>(sm + 2 * S::szB1 + 2 * S::szB2);
  const float* isc2 = isc1 + S::N1;
  float* ut = reinterpret_cast<float*>(sm + S::smA_ut);
  float* pmax = reinterpret_cast<float*>(sm + S::smA_pmax);  // [4][kTile] partial maxima
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::smA_bar);  // op, u0, u1, mma1, mma2
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 5);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = (warp & 3) * 32 + lane;  // element of the tile (tensor-memory lane)
  const int q = warp >> 2;               // the element's quarter of the work
  const uint32_t lanebase = uint32_t((warp & 3) * 32) << 16;
  const int64_t ntiles = (nE + kTile - 1) / kTile;
  const float cpen = float((N + 1) * (N + 2)) * 0.5f;
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) tc::mbar_init(bars + i, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = *slot;
  if (tid == 0) {
    tc::mbar_expect_tx(bars, S::opsA);
    tc::bulk_g2s(sm, opsA, S::opsA, bars);
    if (int64_t(blockIdx.x) < ntiles) {
      const int64_t e0 = int64_t(blockIdx.x) * kTile;
      issue_tile(u, Np, e0, tile_len(nE, e0), ut, bars + 1);
    }
  }
  if (!tc::mbar_wait(bars, 0)) *abort_flag = 1;
  constexpr uint32_t idesc1 = tc::idesc_f16(128, HELM ? S::N1 : S::NP1, false);
  constexpr uint32_t idesc2 = tc::idesc_f16(128, S::N2, false);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int buf = it & 1;
    const int64_t e0 = tile * kTile;
    const int ne = tile_len(nE, e0);
    float* cur = ut + buf * (kTile * Np);
    const bool live = e < ne;
    const int64_t be = e0 + e;
    const int64_t el = be % K;  // element of the mesh (first right-hand side: no division)
    const int64_t boff = be - el;
    const float* g = gx + 16 * el;
    // neighbour data of the face quarters, requested before anything waits
    int code0 = -1, code1 = -1;
    float2 p0[Nfp], p1[Nfp];
    if (q >= 2) {
      const int f0 = q == 2 ? 0 : 2;
      code0 = live ? __ldg(conn + 3 * el + f0) : -1;
      if (q == 2) code1 = live ? __ldg(conn + 3 * el + 1) : -1;
      load_nb<N>(FN, boff, code0, live, p0);
      load_nb<N>(FN, boff, code1, live && q == 2, p1);
    }
    if (!tc::mbar_wait(bars + 1 + buf, (it >> 1) & 1)) *abort_flag = 1;
    if (tid == 0 && tile + gridDim.x < ntiles) {
      const int64_t e1 = (tile + gridDim.x) * kTile;
      issue_tile(u, Np, e1, tile_len(nE, e1), ut + (buf ^ 1) * (kTile * Np), bars + 2 - buf);
    }
    if (ne < kTile) fix_tail(u, Np, e0, ne, cur);
    __syncthreads();
    if (*abort_flag) break;
    const float* urow = cur + e * Np;

    // ---- FP16 pieces of u (scaled per element) into tensor memory: quarter q
    //      takes k in [16q, 16q + 16)
    float xv[16];
    {
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = 16 * q + j;
        xv[j] = (live && k < Np) ? urow[k] : 0.f;
        mx = fmaxf(mx, fabsf(xv[j]));
      }
      pmax[q * kTile + e] = mx;
    }
    __syncthreads();
    const int s1 = scale_exp(fmaxf(fmaxf(pmax[e], pmax[kTile + e]), fmaxf(pmax[2 * kTile + e], pmax[3 * kTile + e])));
    if (16 * q < K1) {
      const float f1 = pow2f(s1);
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) split_pair(xv[2 * c] * f1, xv[2 * c + 1] * f1, hi[c], lo[c]);
      tc::tmem_st8(tb + lanebase + S::oA1 + 8 * q, hi);
      tc::tmem_st8(tb + lanebase + S::oA1 + K1 / 2 + 8 * q, lo);
      tc::tmem_wait_st();
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      uint32_t acc = 0;
#pragma unroll
      for (int ks = 0; ks < K1 / 16; ++ks) {
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
          const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
          const uint64_t bd = tc::smem_desc(tc::smem_addr(sB1) + pb * S::szB1 + ks * 256, 128, (K1 / 8) * 128);
          tc::mma_ts(tb + S::oD1, tb + S::oA1 + pa * (K1 / 2) + ks * 8, bd, idesc1, acc);
          acc = 1;
        }
      }
      tc::mma_commit(bars + 3);
    }
    if (!tc::mbar_wait(bars + 3, it & 1)) *abort_flag = 1;
    tc::fence_after();
    const float iu = tc::ldexp2(1.0f, -s1);  // D1 column c holds C1[c] 2^{s1} / isc1[c]

    // ---- the pointwise stage: this quarter's Y columns in registers
    float y[S::YMAX];
#pragma unroll
    for (int j = 0; j < S::YMAX; ++j) y[j] = 0.f;
    float mx;
    if (q < 2) {
      // volume columns of nodes [n0, n0 + len): wr at [0, len), ws at [V0, V0 + len)
      const int n0 = q * V0;
      uint32_t dr[S::VL], ds[S::VL];
#pragma unroll
      for (int c0 = 0; c0 < S::VL; c0 += 8) {
        uint32_t v[8], w[8];
        tc::tmem_ld8(tb + lanebase + S::oD1 + n0 + c0, v);
        tc::tmem_ld8(tb + lanebase + S::oD1 + Np + n0 + c0, w);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          dr[c0 + c] = v[c];
          ds[c0 + c] = w[c];
        }
      }
      tc::tmem_wait_ld();
      if (live) {
        const float grr = __ldg(g + 1), grs = __ldg(g + 2), gss = __ldg(g + 3);
        const int len = q == 0 ? V0 : Np - V0;
#pragma unroll
        for (int j = 0; j < V0; ++j) {
          if (j < len) {
            const float ur = __uint_as_float(dr[j]) * isc1[n0 + j] * iu;
            const float us = __uint_as_float(ds[j]) * isc1[Np + n0 + j] * iu;
            y[j] = grr * ur + grs * us;
            y[V0 + j] = grs * ur + gss * us;
          }
        }
      }
      mx = absmax<VB>(y);
    } else if (q == 2) {
      uint32_t dr0[Nfp], ds0[Nfp], dr1[Nfp], ds1[Nfp];
      load_face<N>(tb, lanebase, S::oD1, 0, dr0, ds0);
      load_face<N>(tb, lanebase, S::oD1, 1, dr1, ds1);
      tc::tmem_wait_ld();
      if (live) {
        face_columns<N, 0>(y, dr0, ds0, p0, 0, code0, g, urow, isc1, iu, cpen);
        face_columns<N, 3 * Nfp>(y, dr1, ds1, p1, 1, code1, g, urow, isc1, iu, cpen);
      }
      mx = absmax<S::FB2>(y);
    } else {
      uint32_t dr0[Nfp], ds0[Nfp];
      load_face<N>(tb, lanebase, S::oD1, 2, dr0, ds0);
      tc::tmem_wait_ld();
      if (live) face_columns<N, 0>(y, dr0, ds0, p0, 2, code0, g, urow, isc1, iu, cpen);
      mx = absmax<S::FB3>(y);
    }
    uint32_t mv[S::RQ];  // Helmholtz: M u rows of this quarter's outputs
    if (HELM) {
#pragma unroll
      for (int c0 = 0; c0 < S::RQ; c0 += 4) {
        uint32_t v[4];
        tc::tmem_ld4(tb + lanebase + S::oD1 + 2 * Np + q * S::RQ + c0, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) mv[c0 + c] = v[c];
      }
      tc::tmem_wait_ld();
    }
    pmax[q * kTile + e] = mx;
    __syncthreads();
    const int s2 = scale_exp(fmaxf(fmaxf(pmax[e], pmax[kTile + e]), fmaxf(pmax[2 * kTile + e], pmax[3 * kTile + e])));
    {
      const float f2 = pow2f(s2);
      const uint32_t a2 = tb + lanebase + S::oA2;
      if (q < 2) store_y<VB>(y, f2, a2 + q * (VB / 2), KY / 2);
      else if (q == 2) store_y<S::FB2>(y, f2, a2 + VB, KY / 2);
      else store_y<S::FB3>(y, f2, a2 + VB + S::FB2 / 2, KY / 2);
      tc::tmem_wait_st();
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      uint32_t acc = 0;
#pragma unroll 1
      for (int ks = 0; ks < KY / 16; ++ks) {
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
          const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
          const uint64_t bd = tc::smem_desc(tc::smem_addr(sB2) + pb * S::szB2 + ks * 256, 128, (KY / 8) * 128);
          tc::mma_ts(tb + S::oD2, tb + S::oA2 + pa * (KY / 2) + ks * 8, bd, idesc2, acc);
          acc = 1;
        }
      }
      tc::mma_commit(bars + 4);
    }
    if (!tc::mbar_wait(bars + 4, it & 1)) *abort_flag = 1;
    tc::fence_after();

    // ---- epilogue: rows [q RQ, q RQ + RQ) of the element's output
    {
      constexpr int RQ = S::RQ;
      uint32_t dv[RQ];
#pragma unroll
      for (int c0 = 0; c0 < RQ; c0 += 4) {
        uint32_t v[4];
        tc::tmem_ld4(tb + lanebase + S::oD2 + q * RQ + c0, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) dv[c0 + c] = v[c];
      }
      tc::tmem_wait_ld();
      float* stg = cur;  // the tile's u rows are no longer needed (every read of them
                         // precedes the barriers since the pointwise stage)
      if (live) {
        const float iy = tc::ldexp2(1.0f, -s2);
        const float lj = HELM ? lambda * __ldg(g) : 0.f;
#pragma unroll
        for (int c = 0; c < RQ; ++c) {
          const int r = q * RQ + c;
          if (r < Np) {
            float o = __uint_as_float(dv[c]) * isc2[r] * iy;
            if (HELM) o += lj * (__uint_as_float(mv[c]) * isc1[2 * Np + r] * iu);
            stg[e * Np + r] = o;
          }
        }
      }
      __syncthreads();
      const int n = ne * Np;
      float* dst = out + e0 * Np;
      if (ne == kTile) {
        const float4* s4 = reinterpret_cast<const float4*>(stg);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int i = tid; i < n / 4; i += 512) d4[i] = s4[i];
      } else {
        for (int i = tid; i < n; i += 512) dst[i] = stg[i];
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  }
  if (*abort_flag && tid == 0) atomicExch(&g_tc05_err, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ------------------------------------------------------------------------- host side
// FP16 bits of a float (round to nearest even)
uint16_t half_bits(float f) {
  const __half h = __float2half_rn(f);
  __half_raw r = h;
  return r.x;
}
float half_value(uint16_t b) {
  __half_raw r;
  r.x = b;
  return __half2float(__half(r));
}

// Rows x Kd matrix A (row-major, FP64) into two FP16 pieces in the canonical
// no-swizzle K-major layout of an Rp x Kp operand, each row scaled by 2^{e_r}
// so that its largest entry is below 2^14; isc[r] = 2^{-e_r}.
void put_operator(uint8_t* img, const std::vector<double>& A, int rows, int Kd, int Rp, int Kp, float* isc) {
  const size_t piece = size_t(Rp) * Kp * 2;
  const uint32_t SBO = uint32_t(Kp / 8) * 128;
  for (int r = 0; r < Rp; ++r) {
    double mx = 0.0;
    if (r < rows)
      for (int k = 0; k < Kd; ++k) mx = std::max(mx, std::fabs(A[size_t(r) * Kd + k]));
    int ex = 0;
    if (mx > 0.0) std::frexp(mx, &ex);  // mx < 2^ex
    const int er = mx > 0.0 ? 14 - ex : 0;
    isc[r] = float(std::ldexp(1.0, -er));
    for (int k = 0; k < Kp; ++k) {
      const double v = (r < rows && k < Kd) ? std::ldexp(A[size_t(r) * Kd + k], er) : 0.0;
      const uint16_t h = half_bits(float(v));
      const uint16_t l = half_bits(float(v - double(half_value(h))));
      const size_t off = size_t(r / 8) * SBO + size_t(k / 8) * 128 + size_t(r % 8) * 16 + size_t(k % 8) * 2;
      std::memcpy(img + off, &h, 2);
      std::memcpy(img + piece + off, &l, 2);
    }
  }
}

struct TcOps {
  uint8_t* opsA = nullptr;  // tc_apply part
  uint8_t* opsF = nullptr;  // tc_face part
};
TcOps g_tc[64][kMaxN + 1];  // [device][degree]

template <int N>
cudaError_t build_tc_ops(const RefElem& R, TcOps& o) {
  using S = Tc<N>;
  constexpr int Np = S::Np, Nfp = S::Nfp, NFN = S::NFN;
  // [Dr; Ds; M]
  std::vector<double> A1(size_t(3 * Np) * Np);
  for (int i = 0; i < Np * Np; ++i) {
    A1[i] = R.Dr[i];
    A1[Np * Np + i] = R.Ds[i];
    A1[2 * Np * Np + i] = R.M[i];
  }
  // OB in the Y column order of tc_apply
  std::vector<double> B(size_t(Np) * S::KY, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int h = 0; h < 2; ++h) {
      const int n0 = h * S::V0, len = h == 0 ? S::V0 : Np - S::V0;
      for (int j = 0; j < len; ++j) {
        B[size_t(i) * S::KY + h * S::VB + j] = R.Br[size_t(i) * Np + n0 + j];
        B[size_t(i) * S::KY + h * S::VB + S::V0 + j] = R.Bs[size_t(i) * Np + n0 + j];
      }
    }
    for (int f = 0; f < 3; ++f) {
      const int gb = 2 * S::VB + (f < 2 ? f * 3 * Nfp : S::FB2);
      for (int l = 0; l < Nfp; ++l) {
        double dr = 0.0, ds = 0.0, ef = 0.0;
        for (int j = 0; j < Nfp; ++j) {
          const int k = face_node(N, f, j);
          const double mf = R.Mf[size_t(j) * Nfp + l];
          dr += R.Dr[size_t(k) * Np + i] * mf;
          ds += R.Ds[size_t(k) * Np + i] * mf;
          if (k == i) ef += mf;
        }
        B[size_t(i) * S::KY + gb + l] = dr;
        B[size_t(i) * S::KY + gb + Nfp + l] = ds;
        B[size_t(i) * S::KY + gb + 2 * Nfp + l] = ef;
      }
    }
  }
  // face rows of [Dr; Ds]
  std::vector<double> F(size_t(2 * NFN) * Np);
  for (int f = 0; f < 3; ++f)
    for (int j = 0; j < Nfp; ++j) {
      const int k = face_node(N, f, j);
      for (int m = 0; m < Np; ++m) {
        F[size_t(f * Nfp + j) * Np + m] = R.Dr[size_t(k) * Np + m];
        F[size_t(NFN + f * Nfp + j) * Np + m] = R.Ds[size_t(k) * Np + m];
      }
    }
  std::vector<uint8_t> ia(S::opsA, 0), iff(S::opsF, 0);
  float* isc1 = reinterpret_cast<float*>(ia.data() + 2 * S::szB1 + 2 * S::szB2);
  put_operator(ia.data(), A1, 3 * Np, Np, S::N1, S::K1, isc1);
  put_operator(ia.data() + 2 * S::szB1, B, Np, S::KY, S::N2, S::KY, isc1 + S::N1);
  put_operator(iff.data(), F, 2 * NFN, Np, S::NF, S::K1, reinterpret_cast<float*>(iff.data() + 2 * S::szBF));
  cudaError_t e = cudaMalloc(&o.opsA, ia.size());
  if (e == cudaSuccess) e = cudaMemcpy(o.opsA, ia.data(), ia.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&o.opsF, iff.size());
  if (e == cudaSuccess) e = cudaMemcpy(o.opsF, iff.data(), iff.size(), cudaMemcpyHostToDevice);
  return e;
}

template <int N>
cudaError_t launch_n(dg_mesh* m, int B, double lambda, const float* u, float* Au, cudaStream_t st) {
  using S = Tc<N>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  static int grid_face[64], grid_apply[64];
  TcOps* ops = nullptr;
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    TcOps& o = g_tc[dev][N];
    if (!o.opsA) {
      const RefElem R = m->ref[N].N ? m->ref[N] : build_reference(N);
      TcOps built;
      e = build_tc_ops<N>(R, built);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(tc_face<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::smF);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_apply<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::smA);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_apply<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::smA);
      int sms = 0, smem_sm = 0;
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      if (e != cudaSuccess) return e;
      // face CTAs per SM: by shared memory (1 KB reserved per CTA) and tensor
      // memory (128 of 512 columns each)
      const int per = std::max(1, std::min(4, smem_sm / (S::smF + 1024)));
      grid_face[dev] = sms * per;
      grid_apply[dev] = sms;
      o = built;
    }
    ops = &o;
  }
  const int64_t nE = int64_t(B) * m->K;
  const size_t need = size_t(nE) * 3 * (N + 1);
  if (m->face32_cap < need) {
    cudaFree(m->face32);
    m->face32 = nullptr;
    m->face32_cap = 0;
    e = cudaMalloc(&m->face32, need * sizeof(float2));
    if (e == cudaSuccess) e = poison(m->face32, need * sizeof(float2), POISON_APPLY);
    if (e != cudaSuccess) return e;
    m->face32_cap = need;
    ++m->scratch_gen;
  }
  const int64_t ntiles = (nE + kTile - 1) / kTile;
  const unsigned gf = unsigned(std::min<int64_t>(ntiles, grid_face[dev]));
  const unsigned ga = unsigned(std::min<int64_t>(ntiles, grid_apply[dev]));
  tc_face<N><<<gf, kTile, S::smF, st>>>(m->K, nE, m->geox32, u, ops->opsF, m->face32);
  note_launch();
  if (lambda != 0.0)
    tc_apply<N, true><<<ga, 512, S::smA, st>>>(m->K, nE, m->geox32, m->conn, m->face32, u, ops->opsA, float(lambda),
                                               Au);
  else
    tc_apply<N, false><<<ga, 512, S::smA, st>>>(m->K, nE, m->geox32, m->conn, m->face32, u, ops->opsA, 0.f, Au);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool tc05_usable(const void* u, const void* Au) {
  return (reinterpret_cast<uintptr_t>(u) & 15u) == 0 && (reinterpret_cast<uintptr_t>(Au) & 15u) == 0;
}

cudaError_t launch_apply_tc05(dg_mesh* m, int degree, int B, double lambda, const float* u, float* Au,
                              cudaStream_t st) {
  if (B < 1) return cudaSuccess;
  switch (degree) {
    case 1: return launch_n<1>(m, B, lambda, u, Au, st);
    case 2: return launch_n<2>(m, B, lambda, u, Au, st);
    case 3: return launch_n<3>(m, B, lambda, u, Au, st);
    case 4: return launch_n<4>(m, B, lambda, u, Au, st);
    case 5: return launch_n<5>(m, B, lambda, u, Au, st);
    case 6: return launch_n<6>(m, B, lambda, u, Au, st);
    case 7: return launch_n<7>(m, B, lambda, u, Au, st);
    case 8: return launch_n<8>(m, B, lambda, u, Au, st);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
// One warp waits on an mbarrier phase that nothing completes (count 1, no
// arrival), with the bounded wait of the kernels above; *gave_up = 1 when the
// wait ran out, and the timeout is counted in g_tc05_err.
__global__ void wait_selftest(uint64_t limit_ns, int* gave_up) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_init_fence();
  }
  __syncwarp();
  const bool ok = tc::mbar_wait(&bar, 0, limit_ns);
  if (threadIdx.x == 0) {
    *gave_up = ok ? 0 : 1;
    if (!ok) atomicAdd(&g_tc05_err, 1);
  }
}
}  // namespace

cudaError_t launch_wait_selftest(double seconds, int* gave_up_dev, cudaStream_t st) {
  wait_selftest<<<1, 32, 0, st>>>(uint64_t(seconds * 1e9), gave_up_dev);
  note_launch();
  return cudaGetLastError();
}

cudaError_t tc05_error(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc05_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc05_err, &zero, sizeof(int));
  return e;
}

}  // namespace dgx
