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
  static constexpr int E2 = (NFN + 1) / 2;   // face-node entries of face quarter 0 (quarter 1: NFN - E2)
  static constexpr int FQ = rup16(3 * E2);   // Y columns of one face quarter (3 per entry)
  static constexpr int KYV = 2 * VB, KYF = 2 * FQ;  // depths of the volume and face output products
  static constexpr int N2 = rup16(Np);  // output rows
  static constexpr int RQ = N2 / 4;     // output rows per thread of an element
  static constexpr int KQ = K1 / 2;     // u values per volume quarter in the gradient product's input
  // tensor-memory columns of tc_apply
  static constexpr int oA1 = 0, oD1 = K1, oAV = oD1 + N1, oAF = oAV + KYV, oDV = oAF + KYF, oDF = oDV + N2,
                       TCOLS = oDF + N2;
  static_assert(TCOLS <= 512, "tensor memory");
  static_assert(KQ % 8 == 0 || KQ % 4 == 0, "volume quarter input columns");
  // operator image (bytes): tc_apply part [B1 hi | B1 lo | BV hi | BV lo | BF2 hi | BF2 lo |
  // isc1 | iscV | iscF2], tc_face part [BF hi | BF lo | iscF]
  static constexpr int szB1 = N1 * K1 * 2, szBV = N2 * KYV * 2, szBF2 = N2 * KYF * 2, szBF = NF * K1 * 2;
  static constexpr int opsA = 2 * szB1 + 2 * szBV + 2 * szBF2 + 4 * (N1 + 2 * N2);  // a multiple of 16
  static constexpr int opsF = 2 * szBF + 4 * NF;
  static_assert(opsA % 16 == 0 && opsF % 16 == 0, "bulk copy sizes");
  static constexpr int utile = kTile * Np * 4;  // bytes of one FP32 u tile
  // shared memory of tc_apply
  static constexpr int smA_ut = rup128(opsA);
  static constexpr int smA_pmax = smA_ut + 2 * utile;
  static constexpr int smA_bar = smA_pmax + 4 * kTile * 4;
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
// Face data: FN[f (N+1) + j][be] = (u, n.grad u) at face node j of face f
// (counter-clockwise), with the element's own outward normal; column-major with
// leading dimension ldc (a multiple of 32), so that the apply kernel's threads,
// one element each, read their own entries coalesced. One thread per element;
// the tile's face data go through shared memory to coalesced stores.
template <int N>
__global__ void __launch_bounds__(kTile) tc_face(int64_t K, int64_t nE, const float* __restrict__ gx,
                                                 const float* __restrict__ u, const uint8_t* __restrict__ opsF,
                                                 float2* __restrict__ FN, int64_t ldc) {
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
    const int64_t el = e0 + e < K ? e0 + e : (e0 + e) % K;
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
    // column by column: a warp writes 32 consecutive elements of one entry
    for (int i = warp; i < NFN; i += kTile / 32)
      for (int le = tid & 31; le < ne; le += 32) FN[int64_t(i) * ldc + e0 + le] = stg[le * NFN + i];
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
__device__ __forceinline__ void named_sync(int id) { asm volatile("bar.sync %0, 256;\n" ::"r"(id) : "memory"); }

__device__ __forceinline__ void tmem_st4(uint32_t a, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(a), "r"(v0), "r"(v1), "r"(v2),
               "r"(v3)
               : "memory");
}

// FP16 pieces of Y columns [0, L) (scaled by f2) into tensor memory at column
// `addr` (piece hi) and addr + lo_off (piece lo)
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

// The face columns of the face-node entries [I0, I1) (entry i = f Nfp + j):
// per entry [1/2 nr sJ [u], 1/2 ns sJ [u], -sJ ({n.grad u} + tau [u])] from the
// element's own face data (trace, outward normal derivative) and its
// neighbour's across face f, both read from the face kernel's output.
template <int N, int I0, int I1, int YN>
__device__ __forceinline__ void face_quarter(float (&y)[YN], const float2* __restrict__ FN, int64_t ldc, const float* g,
                                             const int32_t* __restrict__ conn, int64_t be, int64_t el, int64_t boff,
                                             float cpen) {
  constexpr int Nfp = N + 1, NFN = 3 * Nfp;
  constexpr int FA = I0 / Nfp, FB = (I1 - 1) / Nfp;  // faces the entries touch
  float nr[3], ns[3], sJ[3], tau[3];
  int code[3];
  const float2* nb[3];
#pragma unroll
  for (int f = FA; f <= FB; ++f) {
    nr[f] = __ldg(g + 4 + 4 * f);
    ns[f] = __ldg(g + 5 + 4 * f);
    sJ[f] = __ldg(g + 6 + 4 * f);
    tau[f] = cpen * __ldg(g + 7 + 4 * f);
    code[f] = __ldg(conn + 3 * el + f);
    nb[f] = code[f] >= 0 ? FN + int64_t((code[f] & 3) * Nfp) * ldc + (boff + (code[f] >> 2)) : FN;
  }
  float2 own[I1 - I0], oth[I1 - I0];
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    const int f = i / Nfp, j = i - f * Nfp;
    own[i - I0] = __ldg(FN + int64_t(i) * ldc + be);
    oth[i - I0] = code[f] >= 0 ? __ldg(nb[f] + int64_t(Nfp - 1 - j) * ldc) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    const int f = i / Nfp;
    const float um = own[i - I0].x, dnm = own[i - I0].y;
    float jm = 0.f, av = 0.f;
    if (code[f] >= 0) {
      jm = oth[i - I0].x - um;
      av = 0.5f * (dnm - oth[i - I0].y);
    } else if (code[f] == -2) {  // Dirichlet
      jm = -2.f * um;
      av = dnm;
    }
    const float hs = 0.5f * sJ[f] * jm;
    y[3 * (i - I0)] = nr[f] * hs;
    y[3 * (i - I0) + 1] = ns[f] * hs;
    y[3 * (i - I0) + 2] = -sJ[f] * (av + tau[f] * jm);
  }
}

// The whole apply of one tile per step (see the file comment). Warps 0-7
// (volume pair: quarters 0 and 1 of every element) build the gradient
// product's input, read its result and form the volume columns; warps 8-15
// (face pair: quarters 2 and 3) form the face columns from the face kernel's
// output without waiting for the gradient product. The output product is two
// accumulators, volume and face columns, each with its own scale, so each
// pair issues its own products as soon as its columns are in tensor memory.
template <int N, bool HELM>
__global__ void __launch_bounds__(512, 1) tc_apply(int64_t K, int64_t nE, const float* __restrict__ gx,
                                                   const int32_t* __restrict__ conn,
                                                   const float2* __restrict__ FN, int64_t ldc,
                                                   const float* __restrict__ u, const uint8_t* __restrict__ opsA,
                                                   float lambda, float* __restrict__ out) {
  using S = Tc<N>;
  constexpr int Np = S::Np, K1 = S::K1, V0 = S::V0, VB = S::VB, FQ = S::FQ, KQ = S::KQ;
  extern __shared__ __align__(128) uint8_t sm[];
  const uint8_t* sB1 = sm;
  const uint8_t* sBV = sm + 2 * S::szB1;
  const uint8_t* sBF = sBV + 2 * S::szBV;
  const float* isc1 = reinterpret_cast<const float*>(sBF + 2 * S::szBF2);
  const float* iscV = isc1 + S::N1;
  const float* iscF = iscV + S::N2;
  float* ut = reinterpret_cast<float*>(sm + S::smA_ut);
  float* pmax = reinterpret_cast<float*>(sm + S::smA_pmax);  // [4][kTile] partial maxima
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::smA_bar);  // op, u0, u1, mma1, mmaV, mmaF
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 6);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = (warp & 3) * 32 + lane;  // element of the tile (tensor-memory lane)
  const int q = warp >> 2;               // the element's quarter of the work
  const uint32_t lanebase = uint32_t((warp & 3) * 32) << 16;
  const int64_t ntiles = (nE + kTile - 1) / kTile;
  const float cpen = float((N + 1) * (N + 2)) * 0.5f;
  if (tid == 0) {
    for (int i = 0; i < 6; ++i) tc::mbar_init(bars + i, 1);
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
    const int64_t el = be < K ? be : be % K;  // element of the mesh (first right-hand side: no division)
    const int64_t boff = be - el;
    const float* g = gx + 16 * el;
    float s_own = 0.f;  // 2^{-s} of this pair's Y scale, for the epilogue
    float iu_own = 0.f;  // 2^{-s1} of the gradient product's input scale (volume pair)
    int s1 = 0;
    if (q < 2) {
      // ================= volume pair
      if (!tc::mbar_wait(bars + 1 + buf, (it >> 1) & 1)) *abort_flag = 1;
      if (tid == 0 && tile + gridDim.x < ntiles) {
        const int64_t e1 = (tile + gridDim.x) * kTile;
        issue_tile(u, Np, e1, tile_len(nE, e1), ut + (buf ^ 1) * (kTile * Np), bars + 2 - buf);
      }
      if (ne < kTile) {
        const int n = ne * Np, b = n & ~3;
        for (int i = b + tid; i < n; i += 256) cur[i] = u[e0 * Np + i];
      }
      const float* urow = cur + e * Np;
      named_sync(1);  // tail of a ragged tile in place
      // FP16 pieces of u (scaled per element): quarter q takes k in [q KQ, q KQ + KQ)
      float xv[KQ];
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < KQ; ++j) {
        const int k = q * KQ + j;
        xv[j] = (live && k < Np) ? urow[k] : 0.f;
        mx = fmaxf(mx, fabsf(xv[j]));
      }
      pmax[q * kTile + e] = mx;
      named_sync(1);
      s1 = scale_exp(fmaxf(pmax[e], pmax[kTile + e]));
      {
        const float f1 = pow2f(s1);
#pragma unroll
        for (int c0 = 0; c0 < KQ / 2; c0 += 4) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) split_pair(xv[2 * (c0 + c)] * f1, xv[2 * (c0 + c) + 1] * f1, hi[c], lo[c]);
          tmem_st4(tb + lanebase + S::oA1 + q * (KQ / 2) + c0, hi[0], hi[1], hi[2], hi[3]);
          tmem_st4(tb + lanebase + S::oA1 + K1 / 2 + q * (KQ / 2) + c0, lo[0], lo[1], lo[2], lo[3]);
        }
        tc::tmem_wait_st();
      }
      tc::fence_before();
      named_sync(1);
      if (tid == 0) {
        tc::fence_after();
        uint32_t acc = 0;
#pragma unroll
        for (int ks = 0; ks < K1 / 16; ++ks) {
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {  // (hi, hi), (hi, lo), (lo, hi)
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
      iu_own = iu;
      // volume columns of nodes [n0, n0 + len): wr at [0, len), ws at [V0, V0 + len)
      float y[VB];
#pragma unroll
      for (int j = 0; j < VB; ++j) y[j] = 0.f;
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
      pmax[q * kTile + e] = absmax<VB>(y);
      named_sync(1);
      const int sv = scale_exp(fmaxf(pmax[e], pmax[kTile + e]));
      s_own = tc::ldexp2(1.0f, -sv);
      store_y<VB>(y, pow2f(sv), tb + lanebase + S::oAV + q * (VB / 2), S::KYV / 2);
      tc::tmem_wait_st();
      tc::fence_before();
      named_sync(1);
      if (tid == 0) {
        tc::fence_after();
        uint32_t acc = 0;
#pragma unroll
        for (int ks = 0; ks < S::KYV / 16; ++ks) {
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
            const uint64_t bd =
                tc::smem_desc(tc::smem_addr(sBV) + pb * S::szBV + ks * 256, 128, (S::KYV / 8) * 128);
            tc::mma_ts(tb + S::oDV, tb + S::oAV + pa * (S::KYV / 2) + ks * 8, bd, idesc2, acc);
            acc = 1;
          }
        }
        tc::mma_commit(bars + 4);
      }
    } else {
      // ================= face pair
      const int qf = q - 2;
      float y[FQ];
#pragma unroll
      for (int j = 0; j < FQ; ++j) y[j] = 0.f;
      if (live) {
        if (qf == 0) face_quarter<N, 0, S::E2>(y, FN, ldc, g, conn, be, el, boff, cpen);
        else face_quarter<N, S::E2, S::NFN>(y, FN, ldc, g, conn, be, el, boff, cpen);
      }
      pmax[q * kTile + e] = absmax<FQ>(y);
      named_sync(2);
      const int sf = scale_exp(fmaxf(pmax[2 * kTile + e], pmax[3 * kTile + e]));
      s_own = tc::ldexp2(1.0f, -sf);
      store_y<FQ>(y, pow2f(sf), tb + lanebase + S::oAF + qf * (FQ / 2), S::KYF / 2);
      tc::tmem_wait_st();
      tc::fence_before();
      named_sync(2);
      if (tid == 256) {
        tc::fence_after();
        uint32_t acc = 0;
#pragma unroll
        for (int ks = 0; ks < S::KYF / 16; ++ks) {
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            const int pa = pr == 2 ? 1 : 0, pb = pr == 1 ? 1 : 0;
            const uint64_t bd =
                tc::smem_desc(tc::smem_addr(sBF) + pb * S::szBF2 + ks * 256, 128, (S::KYF / 8) * 128);
            tc::mma_ts(tb + S::oDF, tb + S::oAF + pa * (S::KYF / 2) + ks * 8, bd, idesc2, acc);
            acc = 1;
          }
        }
        tc::mma_commit(bars + 5);
      }
    }
    // ---- epilogue: both output products done; rows [q RQ, q RQ + RQ)
    // the other pair's scale comes through shared memory
    float* sscale = pmax;  // [3][kTile]: the pairs' 2^{-s} and 2^{-s1}; pmax is free again
    __syncthreads();       // every pair has read its partial maxima
    if (q == 0) {
      sscale[e] = s_own;
      sscale[2 * kTile + e] = iu_own;
    }
    if (q == 2) sscale[kTile + e] = s_own;
    const bool okv = tc::mbar_wait(bars + 4, it & 1);
    const bool okf = tc::mbar_wait(bars + 5, it & 1);
    if (!okv || !okf) *abort_flag = 1;
    tc::fence_after();
    __syncthreads();
    {
      constexpr int RQ = S::RQ;
      uint32_t dv[RQ], df[RQ], mv[RQ];
#pragma unroll
      for (int c0 = 0; c0 < RQ; c0 += 4) {
        uint32_t v[4], w[4];
        tc::tmem_ld4(tb + lanebase + S::oDV + q * RQ + c0, v);
        tc::tmem_ld4(tb + lanebase + S::oDF + q * RQ + c0, w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          dv[c0 + c] = v[c];
          df[c0 + c] = w[c];
        }
        if (HELM) {
          tc::tmem_ld4(tb + lanebase + S::oD1 + 2 * Np + q * RQ + c0, v);
#pragma unroll
          for (int c = 0; c < 4; ++c) mv[c0 + c] = v[c];
        }
      }
      tc::tmem_wait_ld();
      float* stg = cur;  // the tile's u rows are no longer needed
      if (live) {
        const float iyv = sscale[e], iyf = sscale[kTile + e], iu = sscale[2 * kTile + e];
        const float lj = HELM ? lambda * __ldg(g) : 0.f;
#pragma unroll
        for (int c = 0; c < RQ; ++c) {
          const int r = q * RQ + c;
          if (r < Np) {
            float o = __uint_as_float(dv[c]) * iscV[r] * iyv + __uint_as_float(df[c]) * iscF[r] * iyf;
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
    if (*abort_flag) break;
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
  // OB split into its volume columns (Y order of the volume pair) and its
  // face columns (Y order of the face pair: per face-node entry i = f Nfp + l,
  // [Dr_f^T Mf, Ds_f^T Mf, E_f Mf] column l of face f)
  std::vector<double> BV(size_t(Np) * S::KYV, 0.0), BF2(size_t(Np) * S::KYF, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int h = 0; h < 2; ++h) {
      const int n0 = h * S::V0, len = h == 0 ? S::V0 : Np - S::V0;
      for (int j = 0; j < len; ++j) {
        BV[size_t(i) * S::KYV + h * S::VB + j] = R.Br[size_t(i) * Np + n0 + j];
        BV[size_t(i) * S::KYV + h * S::VB + S::V0 + j] = R.Bs[size_t(i) * Np + n0 + j];
      }
    }
    for (int f = 0; f < 3; ++f)
      for (int l = 0; l < Nfp; ++l) {
        double dr = 0.0, ds = 0.0, ef = 0.0;
        for (int j = 0; j < Nfp; ++j) {
          const int k = face_node(N, f, j);
          const double mf = R.Mf[size_t(j) * Nfp + l];
          dr += R.Dr[size_t(k) * Np + i] * mf;
          ds += R.Ds[size_t(k) * Np + i] * mf;
          if (k == i) ef += mf;
        }
        const int ent = f * Nfp + l;
        const int col = ent < S::E2 ? 3 * ent : S::FQ + 3 * (ent - S::E2);
        BF2[size_t(i) * S::KYF + col] = dr;
        BF2[size_t(i) * S::KYF + col + 1] = ds;
        BF2[size_t(i) * S::KYF + col + 2] = ef;
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
  float* isc1 = reinterpret_cast<float*>(ia.data() + 2 * S::szB1 + 2 * S::szBV + 2 * S::szBF2);
  put_operator(ia.data(), A1, 3 * Np, Np, S::N1, S::K1, isc1);
  put_operator(ia.data() + 2 * S::szB1, BV, Np, S::KYV, S::N2, S::KYV, isc1 + S::N1);
  put_operator(ia.data() + 2 * S::szB1 + 2 * S::szBV, BF2, Np, S::KYF, S::N2, S::KYF, isc1 + S::N1 + S::N2);
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
  const int64_t ldc = (nE + 31) & ~int64_t(31);
  const size_t need = size_t(ldc) * 3 * (N + 1);
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
  tc_face<N><<<gf, kTile, S::smF, st>>>(m->K, nE, m->geox32, u, ops->opsF, m->face32, ldc);
  note_launch();
  if (lambda != 0.0)
    tc_apply<N, true><<<ga, 512, S::smA, st>>>(m->K, nE, m->geox32, m->conn, m->face32, ldc, u, ops->opsA,
                                               float(lambda), Au);
  else
    tc_apply<N, false><<<ga, 512, S::smA, st>>>(m->K, nE, m->geox32, m->conn, m->face32, ldc, u, ops->opsA, 0.f, Au);
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
