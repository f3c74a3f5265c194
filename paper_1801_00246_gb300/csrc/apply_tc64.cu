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
//  * tc64_fill: the pointwise stage (metric terms, jumps and averages at face
//    nodes, penalty) in float-float arithmetic on the FP32 pipe, every input
//    scaled by the largest exponent among the element and its neighbours;
//    writes Y in FP64.
//  * C1 and Au are tc64_gemm launches with [Dr; Ds] and OB.
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
constexpr int kSmem = 2 * kABytes + 2 * kBBytes + 4 * kT * 4 + 8 * 8;

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
// out[r][c] = sum_k A[c][k] X[r][k] for r < rows, c < M, k < Kd (A sliced in
// blocks of kNC rows x kKC columns: block (nc, kc) at (nc KCH + kc) kBBytes).
// ex_in (optional): per row, the scale exponent of X's row; ex_out (optional):
// per row, an exponent bound of the outputs.
__global__ void __launch_bounds__(512, 1) tc64_gemm(int64_t rows, int M, int Kd, int NCH, int KCH,
                                                    const double* __restrict__ X, int64_t ldx,
                                                    const uint8_t* __restrict__ Bops, const int* __restrict__ ea,
                                                    double* __restrict__ out, int64_t ldo, int* __restrict__ ex_in,
                                                    int* __restrict__ ex_out) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA = sm;                        // [2][8 slices][128 rows][32] canonical
  uint8_t* sB = sm + 2 * kABytes;          // [2][8 slices][48 rows][32] canonical
  int* pmax = reinterpret_cast<int*>(sB + 2 * kBBytes);  // [4][kT]
  uint64_t* bars = reinterpret_cast<uint64_t*>(pmax + 4 * kT);  // mma0, mma1, b0, b1
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 4);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int e = (warp & 3) * 32 + lane;
  const int q = warp >> 2;
  const uint32_t lanebase = uint32_t((warp & 3) * 32) << 16;
  const int64_t ntiles = (rows + kT - 1) / kT;
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(bars + i, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = *slot;
  constexpr uint32_t idesc = tc::idesc_f16(128, kNC, true);
  uint32_t cnt = 0;  // data chunks issued by this CTA
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * kT + e;
    const bool live = row < rows;
    const double* xr = X + (live ? row : 0) * ldx;
    // scale exponent of the row: the largest |X[row][k]| < 2^E
    int em = -1100;
    if (live)
      for (int kc = 0; kc < KCH; ++kc)
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int k = kc * kKC + 8 * q + t;
          if (k < Kd) em = max(em, exp_bound64(__ldg(xr + k)));
        }
    pmax[q * kT + e] = em;
    __syncthreads();
    int E = max(max(pmax[e], pmax[kT + e]), max(pmax[2 * kT + e], pmax[3 * kT + e]));
    if (E == -1100) E = 0;
    if (ex_in && q == 0 && live) ex_in[row] = E;
    int out_em = -1100;
    for (int nc = 0; nc < NCH; ++nc) {
      for (int kc = 0; kc < KCH; ++kc, ++cnt) {
        const uint32_t ab = cnt & 1u;
        // the buffers of chunk cnt - 2 are free once its products completed
        if (cnt >= 2 && !tc::mbar_wait(bars + ab, ((cnt - 2) >> 1) & 1u)) *abort_flag = 1;
        if (tid == 0) {
          tc::mbar_expect_tx(bars + 2 + ab, kBBytes);
          tc::bulk_g2s(sB + ab * kBBytes, Bops + size_t(nc * KCH + kc) * kBBytes, kBBytes, bars + 2 + ab);
        }
        // slices of X[row][kc*32 + 8q .. + 8): one 16-byte row of a core matrix per slice
        {
          uint64_t I[8];
          uint32_t sg[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int k = kc * kKC + 8 * q + t;
            const double v = (live && k < Kd) ? __ldg(xr + k) : 0.0;
            I[t] = fixed56(v, E, sg[t]);
          }
          uint8_t* dst = sA + ab * kABytes + (e >> 3) * 512 + q * 128 + (e & 7) * 16;
#pragma unroll
          for (int j = 0; j < kSl; ++j) {
            uint4 w;
            w.x = slice_bits(I[0], j, sg[0]) | (slice_bits(I[1], j, sg[1]) << 16);
            w.y = slice_bits(I[2], j, sg[2]) | (slice_bits(I[3], j, sg[3]) << 16);
            w.z = slice_bits(I[4], j, sg[4]) | (slice_bits(I[5], j, sg[5]) << 16);
            w.w = slice_bits(I[6], j, sg[6]) | (slice_bits(I[7], j, sg[7]) << 16);
            *reinterpret_cast<uint4*>(dst + j * kASlice) = w;
          }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (warp == 0) {  // the whole warp waits for the operator block, lane 0 issues
          tc::fence_after();
          if (!tc::mbar_wait(bars + 2 + ab, (cnt >> 1) & 1u)) *abort_flag = 1;
        }
        if (tid == 0) {
          const uint32_t sa = tc::smem_addr(sA + ab * kABytes), sb = tc::smem_addr(sB + ab * kBBytes);
          uint32_t started = kc > 0 ? 0xffu : 0u;
#pragma unroll
          for (int ks = 0; ks < kKC / 16; ++ks)
#pragma unroll
            for (int i = 0; i < kSl; ++i)
#pragma unroll
              for (int j = 0; j < kSl - i; ++j) {
                const int s = i + j;
                const uint64_t ad = tc::smem_desc(sa + j * kASlice + ks * 256, 128, (kKC / 8) * 128);
                const uint64_t bd = tc::smem_desc(sb + i * kBSlice + ks * 256, 128, (kKC / 8) * 128);
                tc::mma_ss(tb + s * kNC, ad, bd, idesc, (started >> s) & 1u);
                started |= 1u << s;
              }
          tc::mma_commit(bars + ab);
        }
      }
      // drain: output columns [12q, 12q + 12) of this pass
      const uint32_t last = cnt - 1;
      if (!tc::mbar_wait(bars + (last & 1u), (last >> 1) & 1u)) *abort_flag = 1;
      tc::fence_after();
#pragma unroll 1
      for (int p = 0; p < 3; ++p) {
        const int c0 = 12 * q + 4 * p;
        uint32_t acc[kSl][4];
#pragma unroll
        for (int s = 0; s < kSl; ++s) {
          uint32_t v[4];
          tc::tmem_ld4(tb + lanebase + s * kNC + c0, v);
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[s][c] = v[c];
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col = nc * kNC + c0 + c;
          if (live && col < M) {
            // value = 2^{ea + E - 14} sum_s acc_s 2^{-7 s}: Horner from the last slice sum
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
            const double o = ff_to_double(h, l, __ldg(ea + col) + E - 14);
            out[row * ldo + col] = o;
            out_em = max(out_em, exp_bound64(o));
          }
        }
      }
      tc::fence_before();
      __syncthreads();  // the accumulators are read; the next pass may overwrite them
    }
    if (ex_out) {
      pmax[q * kT + e] = out_em;
      __syncthreads();
      if (q == 0 && live)
        ex_out[row] = max(max(pmax[e], pmax[kT + e]), max(pmax[2 * kT + e], pmax[3 * kT + e]));
      __syncthreads();
    }
    if (*abort_flag) break;
  }
  if (*abort_flag && tid == 0) atomicExch(&g_tc64_err, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ------------------------------------------------------------------ pointwise stage
__device__ __forceinline__ int fnode(int N, int f, int j) {
  auto rs = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

// One warp per element: Y[be] = [wr, ws | 1/2 nr sJ [u], 1/2 ns sJ [u],
// -sJ ({n.grad u} + tau [u]) (| lambda J u)] from C1 = [ur; us] (ldc per
// element), u, the derived geometry gx (16 FP64 words per element) and the
// neighbours' rows, in float-float scaled by 2^{-R}, R the largest exponent
// of the element's and its neighbours' u and C1 rows (exu, exc).
__global__ void __launch_bounds__(256) tc64_fill(int N, int64_t K, int64_t nE, const double* __restrict__ gx,
                                                 const int32_t* __restrict__ conn, const double* __restrict__ u,
                                                 const double* __restrict__ C1, int ldc, const int* __restrict__ exu,
                                                 const int* __restrict__ exc, double lambda, double* __restrict__ Y,
                                                 int ldy) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  const ff cpen{float((N + 1) * (N + 2)) * 0.5f, 0.f};
  const ff half{0.5f, 0.f};
  const ff lam = d2ff(lambda, 0);
  for (int64_t be = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); be < nE; be += warps) {
    const int64_t el = be % K, boff = be - el;
    // scale: the largest exponent among this element and its neighbours
    int r = -1100;
    if (lane < 3) {
      const int code = __ldg(conn + 3 * el + lane);
      if (code >= 0) {
        const int64_t nb = boff + (code >> 2);
        r = max(__ldg(exu + nb), __ldg(exc + nb));
      }
    } else if (lane == 3) {
      r = max(__ldg(exu + be), __ldg(exc + be));
    }
    int R = __reduce_max_sync(0xffffffffu, r);
    if (R == -1100) R = 0;
    const double* g = gx + 16 * el;
    const double* c = C1 + be * ldc;
    const double* ue = u + be * Np;
    double* y = Y + be * ldy;
    const ff grr = d2ff(__ldg(g + 1), 0), grs = d2ff(__ldg(g + 2), 0), gss = d2ff(__ldg(g + 3), 0);
    for (int n = lane; n < Np; n += 32) {
      const ff ur = d2ff(__ldg(c + n), R), us = d2ff(__ldg(c + Np + n), R);
      const ff wr = ff_add(ff_mul(grr, ur), ff_mul(grs, us));
      const ff ws = ff_add(ff_mul(grs, ur), ff_mul(gss, us));
      y[n] = ff_to_double(wr.h, wr.l, R);
      y[Np + n] = ff_to_double(ws.h, ws.l, R);
      if (ldy > 2 * Np + 3 * NFN) {  // Helmholtz column lambda J u
        const ff lj = ff_mul(lam, d2ff(__ldg(g), 0));
        const ff v = ff_mul(lj, d2ff(__ldg(ue + n), R));
        y[2 * Np + 3 * NFN + n] = ff_to_double(v.h, v.l, R);
      }
    }
    if (lane < NFN) {
      const int f = lane / Nfp, j = lane - f * Nfp;
      const int kf = fnode(N, f, j);
      const ff nr = d2ff(__ldg(g + 4 + 4 * f), 0), ns = d2ff(__ldg(g + 5 + 4 * f), 0);
      const ff sJ = d2ff(__ldg(g + 6 + 4 * f), 0);
      const ff tau = ff_mul(cpen, d2ff(__ldg(g + 7 + 4 * f), 0));
      const ff um = d2ff(__ldg(ue + kf), R);
      const ff dnm = ff_add(ff_mul(nr, d2ff(__ldg(c + kf), R)), ff_mul(ns, d2ff(__ldg(c + Np + kf), R)));
      const int code = __ldg(conn + 3 * el + f);
      ff jm{0.f, 0.f}, av{0.f, 0.f};
      if (code >= 0) {
        const int64_t nb = boff + (code >> 2);
        const int fn = code & 3;
        const int kn = fnode(N, fn, Nfp - 1 - j);
        const double* gn = gx + 16 * (code >> 2) + 4 + 4 * fn;
        const double* cn = C1 + nb * ldc;
        const ff up = d2ff(__ldg(u + nb * Np + kn), R);
        const ff dnp = ff_add(ff_mul(d2ff(__ldg(gn), 0), d2ff(__ldg(cn + kn), R)),
                              ff_mul(d2ff(__ldg(gn + 1), 0), d2ff(__ldg(cn + Np + kn), R)));
        jm = ff_sub(up, um);
        av = ff_pow2(ff_sub(dnm, dnp), 0.5f);
      } else if (code == -2) {  // Dirichlet
        jm = ff_pow2(um, -2.0f);
        av = dnm;
      }
      const ff hs = ff_pow2(ff_mul(sJ, jm), 0.5f);
      const ff a = ff_mul(nr, hs), b = ff_mul(ns, hs);
      const ff fl = ff_neg(ff_mul(sJ, ff_add(av, ff_mul(tau, jm))));
      y[2 * Np + f * Nfp + j] = ff_to_double(a.h, a.l, R);
      y[2 * Np + NFN + f * Nfp + j] = ff_to_double(b.h, b.l, R);
      y[2 * Np + 2 * NFN + f * Nfp + j] = ff_to_double(fl.h, fl.l, R);
    }
  }
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

cudaError_t tc64_gemm_launch(const Tc64Op& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                             int* ex_in, int* ex_out, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int grid[64];
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    if (!grid[dev & 63]) {
      e = cudaFuncSetAttribute(tc64_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
      int sms = 0;
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      grid[dev & 63] = sms;  // one CTA per SM (all of tensor memory, most of shared memory)
    }
  }
  const int64_t tiles = (rows + kT - 1) / kT;
  const unsigned g = unsigned(std::min<int64_t>(tiles, grid[dev & 63]));
  tc64_gemm<<<g, 512, kSmem, st>>>(rows, op.M, op.K, op.NCH, op.KCH, X, ldx, op.blocks, op.ea, out, ldo, ex_in,
                                   ex_out);
  note_launch();
  return cudaGetLastError();
}

namespace {
struct Tc64Apply {
  Tc64Op grad;      // [Dr; Ds]
  Tc64Op out, outh;  // OB, [OB | M]
};
Tc64Apply g_t64[64][kMaxN + 1];  // [device][degree]

cudaError_t build_t64(const RefElem& R, Tc64Apply& o) {
  const int N = R.N, Np = R.Np, Nfp = R.Nfp, NFN = 3 * Nfp;
  std::vector<double> A1(size_t(2 * Np) * Np);
  for (int i = 0; i < Np * Np; ++i) {
    A1[i] = R.Dr[i];
    A1[Np * Np + i] = R.Ds[i];
  }
  const int KY = 2 * Np + 3 * NFN, KH = KY + Np;
  std::vector<double> B(size_t(Np) * KY, 0.0), BH(size_t(Np) * KH, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int m = 0; m < Np; ++m) {
      B[size_t(i) * KY + m] = R.Br[size_t(i) * Np + m];
      B[size_t(i) * KY + Np + m] = R.Bs[size_t(i) * Np + m];
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
        B[size_t(i) * KY + 2 * Np + f * Nfp + l] = dr;
        B[size_t(i) * KY + 2 * Np + NFN + f * Nfp + l] = ds;
        B[size_t(i) * KY + 2 * Np + 2 * NFN + f * Nfp + l] = ef;
      }
    for (int k = 0; k < KY; ++k) BH[size_t(i) * KH + k] = B[size_t(i) * KY + k];
    for (int m = 0; m < Np; ++m) BH[size_t(i) * KH + KY + m] = R.M[size_t(i) * Np + m];
  }
  cudaError_t e = tc64_op_create(A1, 2 * Np, Np, &o.grad);
  if (e == cudaSuccess) e = tc64_op_create(B, Np, KY, &o.out);
  if (e == cudaSuccess) e = tc64_op_create(BH, Np, KH, &o.outh);
  return e;
}
}  // namespace

bool tc64_supported(int degree) {
  const int Np = (degree + 1) * (degree + 2) / 2, NFN = 3 * (degree + 1);
  return 2 * Np + 3 * NFN + Np <= 224;
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
  const int ldc = 2 * Np, ldy = 2 * Np + 3 * NFN + (helm ? Np : 0);
  const int64_t nE = int64_t(B) * m->K;
  // scratch: C1 [nE][2Np], Y [nE][ldy] (FP64), exponents exu, exc [nE]
  const size_t words = size_t(nE) * (ldc + ldy) + size_t(nE) + 8;
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
  double* Y = C1 + size_t(nE) * ldc;
  int* exu = reinterpret_cast<int*>(Y + size_t(nE) * ldy);
  int* exc = exu + nE;
  e = tc64_gemm_launch(ops->grad, nE, u, Np, C1, ldc, exu, exc, st);
  if (e != cudaSuccess) return e;
  {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((nE + 7) / 8, int64_t(sms) * 8);
    tc64_fill<<<unsigned(blocks), 256, 0, st>>>(N, m->K, nE, m->geox, m->conn, u, C1, ldc, exu, exc, lambda, Y, ldy);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return tc64_gemm_launch(helm ? ops->outh : ops->out, nE, Y, ldy, Au, Np, nullptr, nullptr, st);
}

cudaError_t tc64_error(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc64_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc64_err, &zero, sizeof(int));
  return e;
}

}  // namespace dgx
