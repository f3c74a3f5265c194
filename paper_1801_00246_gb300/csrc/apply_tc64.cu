// SIPDG apply in FP64 on the Blackwell tensor cores (tcgen05), without the
// FP64 pipe (GB300 runs FP64 arithmetic at 1/64 of its FP32 rate).
//
// The operator of Eq. ellipticOp3 as the two dense products of apply_tensor.cu,
//   C1 = [Dr; Ds] u                 and   Au = OB Y,
// Y = [wr, ws | 1/2 nr sJ [u], 1/2 ns sJ [u], -sJ ({n.grad u} + tau [u]) (| lambda J u)]
// (OB = [Br Bs | Dr_f^T Mf  Ds_f^T Mf | E_f Mf (| M)]: the Helmholtz term enters
// as extra columns of Y and rows of OB), in three kernels:
//  * tc64_gemm: out[row] = A X[row] for 128 rows per tile, exact to FP64
//    accuracy by integer slicing (the error-free splitting of Ozaki et al.,
//    Numer. Algorithms 59, 2012): every operator row scaled by a power of two
//    and cut into 8 signed 7-bit slices on the host, every data row the same
//    way on the device (integer operations on the double's bits); the 36 slice
//    products with i + j <= 7 run as tcgen05.mma (BF16 operands from shared
//    memory, FP32 accumulators in tensor memory, one accumulator per slice
//    exponent i + j: integer sums below 2^24 for K <= 224 and up to 4 products,
//    exact); the accumulators are recombined by Horner's rule in float-float
//    and rebuilt as doubles from the exponent bits. Data slices are written by
//    the threads into a double-buffered shared-memory chunk (32 columns) while
//    the previous chunk's products run; operator blocks (48 rows x 32 columns,
//    8 slices) arrive by bulk copy.
//  * the gradient product C1 = [Dr; Ds] u (rows interleaved, so one thread
//    holds ur and us of a node; the rows of M follow for Helmholtz) writes C1,
//    M u, every element's face data (u, n.grad u at its face nodes) and
//    exponent bounds per row;
//  * the output product Au = OB Y (+ lambda J M u) forms each data chunk of Y
//    while slicing it: the metric terms wr, ws, and the jumps, averages and
//    penalty of Eq. PenaltyParameter against the neighbours' face data, in
//    float-float on the FP32 pipe (Y never reaches memory).
// Accuracy: relative error near 2^-44 of |A||u| (the slicing's), as the mma.sync path.
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_internal.h"
#include "tc05.cuh"

namespace dgx {
namespace {

constexpr int kT = 128;                      // rows per tile (MMA M)
constexpr int kKC = 32;                      // data columns per chunk
constexpr int kNC = 48;                      // output columns per pass (MMA N)
constexpr int kSl = 8;                       // slices of 7 bits
constexpr int kABytes = kSl * kT * kKC * 2;  // one data chunk, 8 slices: 64 KB
constexpr int kBBytes = kSl * kNC * kKC * 2; // one operator block, 8 slices: 24 KB
constexpr int kASlice = kT * kKC * 2, kBSlice = kNC * kKC * 2;
constexpr int kSmem = 2 * kABytes + 2 * kBBytes + 4 * kT * 4 + 12 * 8;

__device__ int g_tc64_err;

// exponent e with |v| < 2^e (-1100 for zero)
__device__ __forceinline__ int exp_bound64(double v) {
  const int E = int((__double_as_longlong(v) >> 52) & 0x7ff);
  return E == 0 ? -1100 : E - 1022;
}

// |v| 2^{56 - E} as a 56-bit integer (|v| < 2^E) and its sign
__device__ __forceinline__ uint64_t fixed56(double v, int E, uint32_t& sgn) {
  const unsigned long long b = __double_as_longlong(v);
  const int Eb = int((b >> 52) & 0x7ff);
  sgn = uint32_t(b >> 63);
  if (Eb == 0) return 0ull;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = Eb - 1075 + 56 - E;  // <= 3 whenever |v| < 2^E
  if (sh >= 0) return sh < 11 ? (m << sh) : 0ull;
  return sh > -63 ? (m >> (-sh)) : 0ull;
}
// BF16 bits of slice j (7 bits of I below bit 56 - 7j) with the sign
__device__ __forceinline__ uint32_t slice_bits(uint64_t I, int j, uint32_t sgn) {
  const uint32_t x = uint32_t(I >> (49 - 7 * j)) & 127u;
  const float f = __uint_as_float(0x4B000000u | x) - 8388608.0f;  // exactly x
  return (__float_as_uint(f) >> 16) | (sgn << 15);
}

// exact double of (h + l) 2^sc for a float-float pair with |l| small against h
__device__ __forceinline__ double ff_to_double(float h, float l, int sc) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
  const uint32_t uh = __float_as_uint(h), ul = __float_as_uint(l);
  const int eh = int((uh >> 23) & 0xffu), el = int((ul >> 23) & 0xffu);
  if (eh == 0) return 0.0;
  long long M = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;  // h in a 53-bit frame
  if (el != 0) {
    const int sh = 29 - (eh - el);
    const long long ml = (long long)((ul & 0x7fffffu) | 0x800000u);
    long long Ml = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> (-sh)) : 0ll);
    if ((uh ^ ul) >> 31) Ml = -Ml;
    M += Ml;
  }
  int e = eh;
  if (M >= (1ll << 53)) {
    M >>= 1;
    ++e;
  } else if (M < (1ll << 52)) {
    M <<= 1;
    --e;
  }
  const unsigned long long bits = ((unsigned long long)(uh >> 31) << 63) |
                                  ((unsigned long long)(e - 127 + 1023 + sc) << 52) |
                                  ((unsigned long long)M & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// ------------------------------------------------------------------ float-float
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ff_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return ff{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const float s = __fadd_rn(x.h, y.h);
  const float bb = __fsub_rn(s, x.h);
  float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(y.h, bb));
  e = __fadd_rn(e, __fadd_rn(x.l, y.l));
  return ff_renorm(s, e);
}
__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.h, -x.l}; }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return ff_renorm(p, e);
}
__device__ __forceinline__ ff ff_pow2(ff x, float p2) { return ff{x.h * p2, x.l * p2}; }  // exact scaling

// x 2^{-R} as float-float (top 47 bits of the double; parts below the FP32
// range of the scaled value, far below the largest input, flush to zero)
__device__ __forceinline__ ff d2ff(double x, int R) {
  const unsigned long long b = __double_as_longlong(x);
  const int Eb = int((b >> 52) & 0x7ff);
  const int e = Eb - 1023 - R;
  if (Eb == 0 || e < -125) return ff{0.f, 0.f};
  const uint32_t sgn = uint32_t(b >> 63) << 31;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float h = __uint_as_float(sgn | (uint32_t(min(e, 127) + 127) << 23) | uint32_t(m >> 29));
  const uint32_t r23 = uint32_t(m >> 6) & 0x7fffffu;  // the next 23 bits
  const int el = e - 46;
  float l = 0.f;
  if (el >= -126 && r23) {
    l = (__uint_as_float(0x4B000000u | r23) - 8388608.0f) * __uint_as_float(uint32_t(el + 127) << 23);
    l = __uint_as_float(__float_as_uint(l) | sgn);
  }
  return ff{h, l};
}

// ------------------------------------------------------------------ the GEMM
__device__ __forceinline__ int fnode(int N, int f, int j) {
  auto rs = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

// Horner's rule over the 8 slice sums of one output column: (h, l) with
// h + l = sum_s acc_s 2^{-7 s} (float-float)
__device__ __forceinline__ ff horner8(const uint32_t (&acc)[kSl][4], int c) {
  float h = __uint_as_float(acc[kSl - 1][c]), l = 0.f;
#pragma unroll
  for (int s = kSl - 2; s >= 0; --s) {
    const float a = __uint_as_float(acc[s][c]);
    const float hs = h * 0.0078125f, ls = l * 0.0078125f;
    const float sum = __fadd_rn(a, hs);
    const float bb = __fsub_rn(sum, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(hs, bb));
    h = sum;
    l = __fadd_rn(ls, err);
  }
  return ff_renorm(h, l);
}

// |x| 2^{56 - E} (x = h + l, a float-float pair with |x| < 2^E) as a 56-bit
// integer, and the sign of x
__device__ __forceinline__ uint64_t fixed56_ff(ff x, int E, uint32_t& sgn) {
  const uint32_t uh = __float_as_uint(x.h), ul = __float_as_uint(x.l);
  const int eh = int((uh >> 23) & 0xffu), el = int((ul >> 23) & 0xffu);
  if (eh == 0) {  // h zero (or below the normal range): the value is negligible
    sgn = 0;
    return 0ull;
  }
  sgn = uh >> 31;
  auto part = [E](uint32_t u, int eb) -> long long {  // |part| 2^{56 - E}
    const long long m = (long long)((u & 0x7fffffu) | 0x800000u);
    const int sh = eb - 150 + 56 - E;
    if (sh >= 0) return sh < 40 ? (m << sh) : 0ll;
    return sh > -40 ? (m >> (-sh)) : 0ll;
  };
  long long I = part(uh, eh);
  if (el != 0) {
    const long long L = part(ul, el);
    I += ((uh ^ ul) >> 31) ? -L : L;
  }
  return I > 0 ? (uint64_t)I : 0ull;
}

// Arguments of the apply's two products.
struct ApplyArgs {
  int N;
  int64_t K;
  const double* gx;        // derived geometry, 16 FP64 words per element
  const int32_t* conn;     // face connectivity
  double* C1;              // [rows][2 Np]: (ur, us) per node, interleaved
  double* Mu;              // [rows][Np]: M u (Helmholtz), or null
  double2* FN;             // [rows][3 (N+1)]: (u, n.grad u) at the face nodes
  int* exc;                // [rows]: exponent bound of the row's C1 values
  int* exfn;               // [rows]: exponent bound of the row's face data
  double lambda;
  int VK;                  // columns of the volume part of Y (2 Np rounded up to 32)
};

// out[r][c] = sum_k A[c][k] X[r][k] for r < rows, c < M, k < Kd (A sliced in
// blocks of kNC rows x kKC columns: block (nc, kc) at (nc KCH + kc) kBBytes).
//
// Warp-specialised pipeline over a stream of data chunks (tile, output pass
// nc, column chunk kc), chunk g using shared-memory buffer g & 1:
//  * warps 0-15 (four threads per row of the 128-row tile) fix each row's
//    scale exponent, slice chunk g into buffer g & 1 once the products of
//    chunk g - 2 have released it (mbarrier `empty`), signal `full`, and after
//    a pass's last chunk wait for its accumulators (`acc_full`), drain them
//    and release them (`acc_empty`);
//  * warp 16 loads operator block g by bulk copy, waits for `full`, issues the
//    36 slice products per 16 columns from one lane and commits to `empty`
//    (and to `acc_full` after a pass's last chunk); before a pass's first
//    chunk it waits until the previous pass has been drained.
// No CTA-wide barrier in the steady state; every wait is bounded in time.
//
// MODE 0: X is a plain FP64 matrix (rows of length Kd, stride ldx); out FP64.
// MODE 1 (the apply's gradient product): X = u, A = [Dr; Ds] with rows
//   interleaved (column 2n = ur at node n, 2n + 1 = us) and, for Helmholtz,
//   the rows of M after them; the epilogue writes C1, M u, the face data and
//   the rows' exponent bounds instead of `out`.
// MODE 2 (the apply's output product): the data row is Y = [wr_n, ws_n per
//   node | per face-node entry 1/2 nr sJ [u], 1/2 ns sJ [u],
//   -sJ ({n.grad u} + tau [u]), 0], formed while slicing, in float-float on the
//   FP32 pipe, from C1, the face data of the element and its neighbours and the
//   geometry (Y never reaches memory); the epilogue adds lambda J M u.
constexpr int kSlicers = 512;  // threads of warps 0-15
template <int MODE>
__global__ void __launch_bounds__(kSlicers + 32, 1) tc64_gemm(int64_t rows, int M, int Kd, int NCH, int KCH,
                                                              const double* __restrict__ X, int64_t ldx, int vec2,
                                                              const uint8_t* __restrict__ Bops,
                                                              const int* __restrict__ ea, double* __restrict__ out,
                                                              int64_t ldo, ApplyArgs ap) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA = sm;                        // [2][8 slices][128 rows][32] canonical
  uint8_t* sB = sm + 2 * kABytes;          // [2][8 slices][48 rows][32] canonical
  int* pmax = reinterpret_cast<int*>(sB + 2 * kBBytes);  // [4][kT]
  // full[2], empty[2], bfull[2], acc_full, acc_empty
  uint64_t* bars = reinterpret_cast<uint64_t*>(pmax + 4 * kT);
  uint64_t *full = bars, *empty = bars + 2, *bfull = bars + 4, *acc_full = bars + 6, *acc_empty = bars + 7;
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 8);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (rows + kT - 1) / kT;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(full + i, kSlicers / 32);  // one arrival per slicing warp
      tc::mbar_init(empty + i, 1);             // the products' commit
      tc::mbar_init(bfull + i, 1);             // the bulk copy
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, kSlicers / 32);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = *slot;
  constexpr uint32_t idesc = tc::idesc_f16(128, kNC, true);

  if (warp == kSlicers / 32) {
    // ================= products
    uint32_t g = 0, pass = 0;
    const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sA), 128, (kKC / 8) * 128);
    const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sB), 128, (kKC / 8) * 128);
    for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
      for (int nc = 0; nc < NCH; ++nc, ++pass) {
        // the accumulators are free once the previous pass has been drained
        if (pass > 0 && !tc::mbar_wait(acc_empty, (pass - 1) & 1u)) *abort_flag = 1;
        tc::fence_after();
        for (int kc = 0; kc < KCH; ++kc, ++g) {
          const uint32_t b = g & 1u;
          // the operator stage is free once chunk g - 2's products completed
          if (g >= 2 && !tc::mbar_wait(empty + b, ((g - 2) >> 1) & 1u)) *abort_flag = 1;
          if (lane == 0) {
            tc::mbar_expect_tx(bfull + b, kBBytes);
            tc::bulk_g2s(sB + b * kBBytes, Bops + size_t(nc * KCH + kc) * kBBytes, kBBytes, bfull + b);
          }
          __syncwarp();
          if (!tc::mbar_wait(full + b, (g >> 1) & 1u)) *abort_flag = 1;
          if (!tc::mbar_wait(bfull + b, (g >> 1) & 1u)) *abort_flag = 1;
          tc::fence_after();
          if (lane == 0) {
            const uint64_t ab = adesc0 + ((b * kABytes) >> 4), bb = bdesc0 + ((b * kBBytes) >> 4);
            uint32_t started = kc > 0 ? 0xffu : 0u;
#pragma unroll
            for (int ks = 0; ks < kKC / 16; ++ks)
#pragma unroll
              for (int i = 0; i < kSl; ++i)
#pragma unroll
                for (int j = 0; j < kSl - i; ++j) {
                  const int s = i + j;
                  tc::mma_ss(tb + s * kNC, ab + ((j * kASlice + ks * 256) >> 4), bb + ((i * kBSlice + ks * 256) >> 4),
                             idesc, (started >> s) & 1u);
                  started |= 1u << s;
                }
            tc::mma_commit(empty + b);
            if (kc == KCH - 1) tc::mma_commit(acc_full);
          }
          __syncwarp();
        }
      }
    }
  } else {
    // ================= slicing and epilogue
    const int e = (warp & 3) * 32 + lane;
    const int q = warp >> 2;
    const uint32_t lanebase = uint32_t((warp & 3) * 32) << 16;
    uint32_t g = 0, pass = 0;
    const int N = ap.N, Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
    auto load8 = [&](const double* xr, bool live, int k0, int kd, double (&v)[8]) {
      if (live && vec2 && k0 + 8 <= kd) {
        const double2* p2 = reinterpret_cast<const double2*>(xr + k0);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const double2 w = __ldg(p2 + t);
          v[2 * t] = w.x;
          v[2 * t + 1] = w.y;
        }
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (live && k0 + t < kd) ? __ldg(xr + k0 + t) : 0.0;
      }
    };
    auto store_slices = [&](const uint64_t (&I)[8], const uint32_t (&sg)[8], uint32_t b) {
      uint8_t* dst = sA + b * kABytes + (e >> 3) * 512 + q * 128 + (e & 7) * 16;
#pragma unroll
      for (int j = 0; j < kSl; ++j) {
        uint4 w;
        w.x = slice_bits(I[0], j, sg[0]) | (slice_bits(I[1], j, sg[1]) << 16);
        w.y = slice_bits(I[2], j, sg[2]) | (slice_bits(I[3], j, sg[3]) << 16);
        w.z = slice_bits(I[4], j, sg[4]) | (slice_bits(I[5], j, sg[5]) << 16);
        w.w = slice_bits(I[6], j, sg[6]) | (slice_bits(I[7], j, sg[7]) << 16);
        *reinterpret_cast<uint4*>(dst + j * kASlice) = w;
      }
    };
    for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
      const int64_t row = tile * kT + e;
      const bool live = row < rows;
      const int64_t el = MODE == 0 ? 0 : (live ? row : 0) % ap.K;
      const int64_t boff = (live ? row : 0) - el;
      const double* xr = X + (live ? row : 0) * ldx;
      const double* gg = MODE == 0 ? nullptr : ap.gx + 16 * el;
      // ---- the row's scale exponent E (|data| < 2^E) and, MODE 2, the input reference R
      int E = 0, R = 0;
      int codes[3] = {-1, -1, -1};
      if (MODE == 2) {
        // inputs scaled by 2^-R, R bounding C1 and the face data of the element and
        // its neighbours (so scaled values stay in the FP32 range); E from the row's
        // largest |Y| (relative to 2^R), found by a float pre-pass over this thread's
        // columns (float estimates within 2^-20 of Y: a margin factor covers them)
        int r = live ? max(__ldg(ap.exc + row), __ldg(ap.exfn + row)) : -1100;
        if (live) {
#pragma unroll
          for (int f = 0; f < 3; ++f) {
            codes[f] = __ldg(ap.conn + 3 * el + f);
            if (codes[f] >= 0) r = max(r, __ldg(ap.exfn + boff + (codes[f] >> 2)));
          }
        }
        R = r == -1100 ? 0 : r;
        float ymax = 0.f;
        if (live) {
          const float grr = d2ff(__ldg(gg + 1), 0).h, grs = d2ff(__ldg(gg + 2), 0).h, gss = d2ff(__ldg(gg + 3), 0).h;
          const float cp = float((N + 1) * (N + 2)) * 0.5f;
          for (int kc = 0; kc < KCH; ++kc) {
            const int c0 = kc * kKC + 8 * q;
            if (c0 < ap.VK) {
              double v[8];
              load8(ap.C1 + row * 2 * Np, live, c0, 2 * Np, v);
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const float ur = d2ff(v[2 * t], R).h, us = d2ff(v[2 * t + 1], R).h;
                ymax = fmaxf(ymax, fmaxf(fabsf(grr * ur + grs * us), fabsf(grs * ur + gss * us)));
              }
            } else {
              const int i0 = (c0 - ap.VK) >> 2;
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const int i = i0 + t;
                if (i < NFN) {
                  const int f = i / Nfp, j = i - f * Nfp;
                  const int code = codes[f];
                  const double2 own = __ldg(ap.FN + row * NFN + i);
                  const float um = d2ff(own.x, R).h, dnm = d2ff(own.y, R).h;
                  float jm = 0.f, av = 0.f;
                  if (code >= 0) {
                    const double2 oth = __ldg(ap.FN + (boff + (code >> 2)) * NFN + (code & 3) * Nfp + (Nfp - 1 - j));
                    jm = d2ff(oth.x, R).h - um;
                    av = 0.5f * (dnm - d2ff(oth.y, R).h);
                  } else if (code == -2) {
                    jm = -2.f * um;
                    av = dnm;
                  }
                  const double* gf = gg + 4 + 4 * f;
                  const float nr = d2ff(__ldg(gf), 0).h, ns = d2ff(__ldg(gf + 1), 0).h, sJ = d2ff(__ldg(gf + 2), 0).h;
                  const float tau = cp * d2ff(__ldg(gf + 3), 0).h;
                  const float hs = 0.5f * sJ * jm;
                  ymax = fmaxf(ymax, fmaxf(fmaxf(fabsf(nr * hs), fabsf(ns * hs)), fabsf(sJ * (av + tau * jm))));
                }
              }
            }
          }
        }
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");  // pmax free (previous tile read it)
        reinterpret_cast<float*>(pmax)[q * kT + e] = ymax;
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        const float* pf = reinterpret_cast<const float*>(pmax);
        const float mx = fmaxf(fmaxf(pf[e], pf[kT + e]), fmaxf(pf[2 * kT + e], pf[3 * kT + e]));
        E = mx > 0.f ? tc::exp_of(mx * 1.0001f) : 0;  // |Y| 2^-R < 2^E
      } else {
        int em = -1100;
        if (live) {
          double v[2][8];
          for (int kc = 0; kc < KCH; kc += 2) {
            load8(xr, live, kc * kKC + 8 * q, Kd, v[0]);
            load8(xr, live && kc + 1 < KCH, (kc + 1) * kKC + 8 * q, Kd, v[1]);
#pragma unroll
            for (int t = 0; t < 8; ++t) em = max(em, max(exp_bound64(v[0][t]), exp_bound64(v[1][t])));
          }
        }
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");  // pmax free (previous tile read it)
        pmax[q * kT + e] = em;
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        E = max(max(pmax[e], pmax[kT + e]), max(pmax[2 * kT + e], pmax[3 * kT + e]));
        if (E == -1100) E = 0;
      }
      ff gmx[3];  // MODE 2: Grr, Grs, Gss as float-float
      if (MODE == 2) {
#pragma unroll
        for (int t = 0; t < 3; ++t) gmx[t] = live ? d2ff(__ldg(gg + 1 + t), 0) : ff{0.f, 0.f};
      }
      double vn[8];  // MODE 0/1: the next chunk's values, loaded one chunk ahead
      if (MODE != 2) load8(xr, live, 8 * q, Kd, vn);
      int mexc = -1100, mexf = -1100;  // MODE 1: exponent bounds of the C1 values and face data written
      for (int nc = 0; nc < NCH; ++nc, ++pass) {
        for (int kc = 0; kc < KCH; ++kc, ++g) {
          const uint32_t b = g & 1u;
          uint64_t I[8];
          uint32_t sg[8];
          const int c0 = kc * kKC + 8 * q;  // this thread's 8 data columns
          if (MODE != 2) {
            double v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = vn[t];
            {  // request the next chunk of this row (the next pass starts again at chunk 0)
              const int kn = kc + 1 < KCH ? kc + 1 : 0;
              if (kc + 1 < KCH || nc + 1 < NCH) load8(xr, live, kn * kKC + 8 * q, Kd, vn);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) I[t] = fixed56(v[t], E, sg[t]);
          } else {
            ff y[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) y[t] = ff{0.f, 0.f};
            if (live && c0 < ap.VK) {
              // volume: nodes c0/2 .. c0/2 + 3, (wr, ws) each
              double v[8];
              load8(ap.C1 + row * 2 * Np, live, c0, 2 * Np, v);
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const ff ur = d2ff(v[2 * t], R), us = d2ff(v[2 * t + 1], R);
                y[2 * t] = ff_add(ff_mul(gmx[0], ur), ff_mul(gmx[1], us));
                y[2 * t + 1] = ff_add(ff_mul(gmx[1], ur), ff_mul(gmx[2], us));
              }
            } else if (live) {
              // faces: entries i0, i0 + 1 (four columns each: a, b, c, 0)
              const int i0 = (c0 - ap.VK) >> 2;
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const int i = i0 + t;
                if (i < NFN) {
                  const int f = i / Nfp, j = i - f * Nfp;
                  const int code = codes[f];
                  const double2 own = __ldg(ap.FN + row * NFN + i);
                  const ff um = d2ff(own.x, R), dnm = d2ff(own.y, R);
                  ff jm{0.f, 0.f}, av{0.f, 0.f};
                  if (code >= 0) {
                    const double2 oth = __ldg(ap.FN + (boff + (code >> 2)) * NFN + (code & 3) * Nfp + (Nfp - 1 - j));
                    jm = ff_sub(d2ff(oth.x, R), um);
                    av = ff_pow2(ff_sub(dnm, d2ff(oth.y, R)), 0.5f);
                  } else if (code == -2) {  // Dirichlet
                    jm = ff_pow2(um, -2.0f);
                    av = dnm;
                  }
                  const double* gf = gg + 4 + 4 * f;
                  const ff nr = d2ff(__ldg(gf), 0), ns = d2ff(__ldg(gf + 1), 0), sJ = d2ff(__ldg(gf + 2), 0);
                  const ff tau = ff_mul(ff{float((N + 1) * (N + 2)) * 0.5f, 0.f}, d2ff(__ldg(gf + 3), 0));
                  const ff hs = ff_pow2(ff_mul(sJ, jm), 0.5f);
                  y[4 * t] = ff_mul(nr, hs);
                  y[4 * t + 1] = ff_mul(ns, hs);
                  y[4 * t + 2] = ff_neg(ff_mul(sJ, ff_add(av, ff_mul(tau, jm))));
                }
              }
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) I[t] = fixed56_ff(y[t], E, sg[t]);
          }
          // buffer b is free once chunk g - 2's products completed
          if (g >= 2 && !tc::mbar_wait(empty + b, ((g - 2) >> 1) & 1u)) *abort_flag = 1;
          store_slices(I, sg, b);
          tc::fence_async_smem();
          __syncwarp();
          if (lane == 0) asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(
                                          tc::smem_addr(full + b))
                                      : "memory");
        }
        // drain: output columns [12q, 12q + 12) of this pass
        if (!tc::mbar_wait(acc_full, pass & 1u)) *abort_flag = 1;
        tc::fence_after();
#pragma unroll 1
        for (int p = 0; p < 3; ++p) {
          const int cl = 12 * q + 4 * p;
          uint32_t acc[kSl][4];
#pragma unroll
          for (int s = 0; s < kSl; ++s) {
            uint32_t vv[4];
            tc::tmem_ld4(tb + lanebase + s * kNC + cl, vv);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[s][c] = vv[c];
          }
          tc::tmem_wait_ld();
          if (p == 2) {  // the accumulators are read: release them to the next pass
            tc::fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(
                                            tc::smem_addr(acc_empty))
                                        : "memory");
          }
          if (MODE == 0 || MODE == 2) {
            const int Eo = MODE == 2 ? E + R : E;  // the data row's scale
            float lj_h = 0.f, lj_l = 0.f;
            if (MODE == 2 && ap.Mu && live) {
              const ff lj = ff_mul(d2ff(ap.lambda, 0), d2ff(__ldg(gg), 0));
              lj_h = lj.h;
              lj_l = lj.l;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int col = nc * kNC + cl + c;
              if (live && col < M) {
                // value = 2^{ea + E - 14} sum_s acc_s 2^{-7 s}
                const ff hl = horner8(acc, c);
                const int sc = __ldg(ea + col) + Eo - 14;
                double o;
                if (MODE == 2 && ap.Mu) {  // + lambda J (M u) in float-float at the product's scale
                  const double mu = __ldg(ap.Mu + row * Np + col);
                  const ff t = ff_mul(ff{lj_h, lj_l}, d2ff(mu, sc));
                  const ff sum = ff_add(hl, t);
                  o = ff_to_double(sum.h, sum.l, sc);
                } else {
                  o = ff_to_double(hl.h, hl.l, sc);
                }
                out[row * ldo + col] = o;
              }
            }
          } else {
            // MODE 1: columns (2n, 2n + 1) = (ur, us) of node n; columns from 2 Np: M u
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
              const int col = nc * kNC + cl + c;
              if (!live || col >= M) continue;
              if (col >= 2 * Np) {  // Helmholtz rows: M u
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                  if (col + t < M) {
                    const ff hl = horner8(acc, c + t);
                    ap.Mu[row * Np + col + t - 2 * Np] = ff_to_double(hl.h, hl.l, __ldg(ea + col + t) + E - 14);
                  }
                }
                continue;
              }
              const int n = col >> 1;
              const int er = __ldg(ea + col), es = __ldg(ea + col + 1);
              const int ec = max(er, es);
              ff ur = horner8(acc, c), us = horner8(acc, c + 1);
              const double dur = ff_to_double(ur.h, ur.l, er + E - 14), dus = ff_to_double(us.h, us.l, es + E - 14);
              ap.C1[row * 2 * Np + col] = dur;
              ap.C1[row * 2 * Np + col + 1] = dus;
              mexc = max(mexc, max(exp_bound64(dur), exp_bound64(dus)));
              // face data at the face nodes this node is (a corner belongs to two faces)
              int rrow = 0;
              while (n >= (rrow + 1) * (N + 1) - (rrow + 1) * rrow / 2) ++rrow;  // n's row of constant s
              const int rs0 = rrow * (N + 1) - rrow * (rrow - 1) / 2, len = N + 1 - rrow;
              int fa = -1, ja = 0, fb = -1, jb = 0;
              if (rrow == 0) fa = 0, ja = n;                  // face 0, j = n
              if (n == rs0 + len - 1) {                       // face 1, j = row
                if (fa < 0) fa = 1, ja = rrow;
                else fb = 1, jb = rrow;
              }
              if (n == rs0 && fb < 0) {                       // face 2, j = N - row
                if (fa < 0) fa = 2, ja = N - rrow;
                else fb = 2, jb = N - rrow;
              }
              if (fa >= 0) {
                ur = ff_pow2(ur, __uint_as_float(uint32_t(127 + er - ec) << 23));
                us = ff_pow2(us, __uint_as_float(uint32_t(127 + es - ec) << 23));
                const int S = ec + E - 14;
                const double un = __ldg(X + row * ldx + n);
                const double* g2 = ap.gx + 16 * (row % ap.K);
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                  const int f = t == 0 ? fa : fb, j = t == 0 ? ja : jb;
                  if (f >= 0) {
                    const ff nr = d2ff(__ldg(g2 + 4 + 4 * f), 0), ns = d2ff(__ldg(g2 + 5 + 4 * f), 0);
                    const ff dn = ff_add(ff_mul(nr, ur), ff_mul(ns, us));
                    const double ddn = ff_to_double(dn.h, dn.l, S);
                    ap.FN[row * NFN + f * Nfp + j] = make_double2(un, ddn);
                    mexf = max(mexf, max(exp_bound64(un), exp_bound64(ddn)));
                  }
                }
              }
            }
          }
        }
      }
      if (MODE == 1) {  // the rows' exponent bounds of C1 and of the face data
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        pmax[q * kT + e] = mexc;
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        const int xc = max(max(pmax[e], pmax[kT + e]), max(pmax[2 * kT + e], pmax[3 * kT + e]));
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        pmax[q * kT + e] = mexf;
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        const int xf = max(max(pmax[e], pmax[kT + e]), max(pmax[2 * kT + e], pmax[3 * kT + e]));
        if (q == 0 && live) {
          ap.exc[row] = xc;
          ap.exfn[row] = xf;
        }
      }
    }
  }
  if (*abort_flag && tid == 0) atomicExch(&g_tc64_err, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ------------------------------------------------------------------ host side
int row_exp(const double* row, int K) {
  double mx = 0.0;
  for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(row[k]));
  if (mx == 0.0) return 0;
  int e = 0;
  std::frexp(mx, &e);  // mx < 2^e
  return e;
}

uint16_t bf16_int(int x) {  // exact for |x| <= 256
  const float f = float(x);
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return uint16_t(b >> 16);
}

}  // namespace

// A (M x K, row-major FP64) into the block layout of tc64_gemm.
cudaError_t tc64_op_create(const std::vector<double>& A, int M, int K, Tc64Op* op) {
  op->M = M;
  op->K = K;
  op->NCH = (M + kNC - 1) / kNC;
  op->KCH = (K + kKC - 1) / kKC;
  if (K > 224) return cudaErrorInvalidValue;  // longer sums would leave the FP32 group sums inexact
  std::vector<uint8_t> img(size_t(op->NCH) * op->KCH * kBBytes, 0);
  std::vector<int> ea(size_t(op->NCH) * kNC, 0);
  for (int r = 0; r < M; ++r) {
    const int er = row_exp(&A[size_t(r) * K], K);
    ea[r] = er;
    for (int k = 0; k < K; ++k) {
      const double v = A[size_t(r) * K + k];
      if (v == 0.0 || !std::isfinite(v)) continue;
      int e2 = 0;
      const double fr = std::frexp(std::fabs(v), &e2);
      const int sh = e2 + 56 - er;
      if (sh <= 0) continue;
      const unsigned long long I = (unsigned long long)std::ldexp(fr, sh);
      const int sgn = v < 0 ? -1 : 1;
      const int nc = r / kNC, rl = r % kNC, kc = k / kKC, kl = k % kKC;
      uint8_t* blk = img.data() + size_t(nc * op->KCH + kc) * kBBytes;
      const size_t off = size_t(rl / 8) * ((kKC / 8) * 128) + size_t(kl / 8) * 128 + size_t(rl % 8) * 16 + size_t(kl % 8) * 2;
      for (int i = 0; i < kSl; ++i) {
        const int x = sgn * int((I >> (49 - 7 * i)) & 127ull);
        const uint16_t b = bf16_int(x);
        std::memcpy(blk + size_t(i) * kBSlice + off, &b, 2);
      }
    }
  }
  cudaError_t e = cudaMalloc(&op->blocks, img.size());
  if (e == cudaSuccess) e = cudaMemcpy(op->blocks, img.data(), img.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&op->ea, ea.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(op->ea, ea.data(), ea.size() * sizeof(int), cudaMemcpyHostToDevice);
  return e;
}

void tc64_op_free(Tc64Op* op) {
  cudaFree(op->blocks);
  cudaFree(op->ea);
  op->blocks = nullptr;
  op->ea = nullptr;
}

namespace {
template <int MODE>
cudaError_t gemm_launch(const Tc64Op& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                        const ApplyArgs& ap, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int grid[64];
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    if (!grid[dev & 63]) {
      e = cudaFuncSetAttribute(tc64_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(tc64_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(tc64_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
      int sms = 0;
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      grid[dev & 63] = sms;  // one CTA per SM (all of tensor memory, most of shared memory)
    }
  }
  const double* vx = MODE == 2 ? ap.C1 : X;  // the rows read with paired loads
  const int64_t vld = MODE == 2 ? 2 * ((ap.N + 1) * (ap.N + 2) / 2) : ldx;
  const int vec2 = (vld % 2 == 0 && (reinterpret_cast<uintptr_t>(vx) & 15u) == 0) ? 1 : 0;
  const int64_t tiles = (rows + kT - 1) / kT;
  const unsigned g = unsigned(std::min<int64_t>(tiles, grid[dev & 63]));
  tc64_gemm<MODE><<<g, kSlicers + 32, kSmem, st>>>(rows, op.M, op.K, op.NCH, op.KCH, X, ldx, vec2, op.blocks, op.ea, out,
                                                   ldo, ap);
  note_launch();
  return cudaGetLastError();
}
}  // namespace

cudaError_t tc64_gemm_launch(const Tc64Op& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                             cudaStream_t st) {
  return gemm_launch<0>(op, rows, X, ldx, out, ldo, ApplyArgs{}, st);
}

namespace {
struct Tc64Apply {
  Tc64Op grad, gradh;  // [Dr; Ds] with rows interleaved (Dr row n, Ds row n, ...), then M for Helmholtz
  Tc64Op out;          // OB in the column order of Y: (Br, Bs) per node, then 4 per face-node entry
};
Tc64Apply g_t64[64][kMaxN + 1];  // [device][degree]

int vol_cols(int Np) { return (2 * Np + 31) / 32 * 32; }

cudaError_t build_t64(const RefElem& R, Tc64Apply& o) {
  const int N = R.N, Np = R.Np, Nfp = R.Nfp, NFN = 3 * Nfp;
  std::vector<double> A1(size_t(3 * Np) * Np);
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m) {
      A1[size_t(2 * n) * Np + m] = R.Dr[size_t(n) * Np + m];
      A1[size_t(2 * n + 1) * Np + m] = R.Ds[size_t(n) * Np + m];
      A1[size_t(2 * Np + n) * Np + m] = R.M[size_t(n) * Np + m];
    }
  const int VK = vol_cols(Np), KK = VK + 4 * NFN;
  std::vector<double> B(size_t(Np) * KK, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int n = 0; n < Np; ++n) {
      B[size_t(i) * KK + 2 * n] = R.Br[size_t(i) * Np + n];
      B[size_t(i) * KK + 2 * n + 1] = R.Bs[size_t(i) * Np + n];
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
        const int c = VK + 4 * (f * Nfp + l);
        B[size_t(i) * KK + c] = dr;
        B[size_t(i) * KK + c + 1] = ds;
        B[size_t(i) * KK + c + 2] = ef;
      }
  }
  cudaError_t e = tc64_op_create(std::vector<double>(A1.begin(), A1.begin() + size_t(2 * Np) * Np), 2 * Np, Np,
                                 &o.grad);
  if (e == cudaSuccess) e = tc64_op_create(A1, 3 * Np, Np, &o.gradh);
  if (e == cudaSuccess) e = tc64_op_create(B, Np, KK, &o.out);
  return e;
}
}  // namespace

bool tc64_supported(int degree) {
  const int Np = (degree + 1) * (degree + 2) / 2, NFN = 3 * (degree + 1);
  return vol_cols(Np) + 4 * NFN <= 224;
}

cudaError_t launch_apply_tc64(dg_mesh* m, int degree, int B, double lambda, const double* u, double* Au,
                              cudaStream_t st) {
  if (B < 1) return cudaSuccess;
  if (!tc64_supported(degree)) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const Tc64Apply* ops = nullptr;
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    Tc64Apply& o = g_t64[dev & 63][degree];
    if (!o.grad.blocks) {
      const RefElem R = m->ref[degree].N ? m->ref[degree] : build_reference(degree);
      Tc64Apply built;
      e = build_t64(R, built);
      if (e != cudaSuccess) return e;
      o = built;
    }
    ops = &o;
  }
  const int N = degree, Np = (N + 1) * (N + 2) / 2, NFN = 3 * (N + 1);
  const bool helm = lambda != 0.0;
  const int64_t nE = int64_t(B) * m->K;
  // scratch: C1 [nE][2 Np], M u [nE][Np] (Helmholtz), the face data [nE][NFN] (u, n.grad u),
  // FP64, and two exponent bounds per row
  const size_t words = size_t(nE) * (2 * Np + (helm ? Np : 0) + 2 * NFN) + size_t(nE) + 4;
  if (m->t64_cap < words) {
    cudaFree(m->t64_scratch);
    m->t64_scratch = nullptr;
    m->t64_cap = 0;
    e = cudaMalloc(&m->t64_scratch, words * sizeof(double));
    if (e == cudaSuccess) e = poison(m->t64_scratch, words * sizeof(double), POISON_APPLY);
    if (e != cudaSuccess) return e;
    m->t64_cap = words;
    ++m->scratch_gen;
  }
  double* C1 = m->t64_scratch;
  double* Mu = helm ? C1 + size_t(nE) * 2 * Np : nullptr;
  double2* FN = reinterpret_cast<double2*>(C1 + size_t(nE) * (2 * Np + (helm ? Np : 0)));
  int* exc = reinterpret_cast<int*>(FN + size_t(nE) * NFN);
  int* exfn = exc + nE;
  const ApplyArgs ap{N, m->K, m->geox, m->conn, C1, Mu, FN, exc, exfn, lambda, vol_cols(Np)};
  e = gemm_launch<1>(helm ? ops->gradh : ops->grad, nE, u, Np, nullptr, 0, ap, st);
  if (e != cudaSuccess) return e;
  return gemm_launch<2>(ops->out, nE, nullptr, 0, Au, Np, ap, st);
}

cudaError_t tc64_error(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc64_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc64_err, &zero, sizeof(int));
  return e;
}

}  // namespace dgx
