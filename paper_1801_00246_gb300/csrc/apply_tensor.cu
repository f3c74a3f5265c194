// SIPDG apply with its dense products on the BF16 tensor cores, in FP64 or FP32.
//
// The two dense products of the operator (Eq. ellipticOp3 written as in
// apply_gemm.cuh),
//   C1 = [Dr; Ds] U   and   Au = OB Y,
// are evaluated exactly enough for the working precision with integer-sliced
// BF16 products (the error-free splitting of Ozaki et al., "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012):
//   * every operator row r is scaled by a power of two 2^{ea_r} and written as
//     sum_i a_i 2^{-7i}, i = 1..KS, with signed integers |a_i| <= 127 (host);
//   * every element's data column is scaled by 2^{ex_e} and sliced the same way
//     on the fly from the value's bit pattern (integer shifts only);
//   * a_i x_j products summed over K <= 256 are integers below 2^22 (127^2 * 256),
//     exact in the FP32 accumulators of mma.sync m16n8k16; products with the
//     same i + j share an accumulator, which stays exact (below 2^24) for groups
//     of up to 4 products at K = 256 (up to 6 at K = 171); the larger groups carry weights
//     below 2^-28 of the leading one, so their rounding is below 2^-50 of the
//     result; only i + j <= KS + 1 is formed;
//   * the KS accumulators are combined by Horner's rule (float-float for FP64)
//     and scaled back by building the exponent bits.
// That is the FP64 scheme: KS = 8 slices (56 bits, 36 products; relative error
// near 2^-44 of |A||x|). FP32 needs no exactness, only FP32-level accuracy, so
// it splits operands by round-to-nearest into three BF16 pieces (hi, mid, lo:
// x - hi - mid - lo is below 2^-24 |x|), forms the 6 products with
// i + j <= 2 into a single FP32 accumulator and needs no exponents, scaling or
// integer extraction at all.
//
// The face mass is folded into the output operator
//   OB = [Br Bs | Dr_f^T Mf  Ds_f^T Mf | E_f Mf | M],
// so the pointwise stage between the two products only forms
//   Y = [wr; ws; 1/2 nr sJ [u]; 1/2 ns sJ [u]; -sJ ({n.grad u} + tau [u]); lambda J u].
// That stage runs inside the output product's slicing phase (Y is built in
// shared memory, never in HBM); the neighbour's trace and normal derivative at
// a shared face node are read from its nodal values and its rows of C1.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dg_internal.h"
#include "tc05.cuh"

namespace dgx {
namespace {

constexpr int kSliceBits = 7;
constexpr int OE = 32;       // elements per CTA tile
constexpr int ONT = OE / 8;  // n-tiles (8 elements each)

template <typename T>
struct Slices;
template <>
struct Slices<double> {
  static constexpr int KS = 8;  // 56 bits
};
template <>
struct Slices<float> {
  static constexpr int KS = 3;  // round-to-nearest BF16 pieces hi, mid, lo
};

// ---------------------------------------------------------------- host side
// KS slices of v relative to 2^{scale_exp} (|v| < 2^{scale_exp}):
// floor(|v| 2^{7 KS - scale_exp}) cut into KS chunks of 7 bits, sign applied.
void slice_host(double v, int scale_exp, int KS, int* out) {
  const int bits = kSliceBits * KS;
  for (int j = 0; j < KS; ++j) out[j] = 0;
  if (v == 0.0 || !std::isfinite(v)) return;
  int e = 0;
  const double fr = std::frexp(std::fabs(v), &e);  // |v| = fr 2^e, fr in [0.5, 1)
  const int sh = e + bits - scale_exp;
  if (sh <= 0) return;
  const unsigned long long I = (unsigned long long)std::ldexp(fr, sh);  // exact for sh <= 53, truncated beyond
  const int sgn = v < 0 ? -1 : 1;
  for (int j = 0; j < KS; ++j) out[j] = sgn * int((I >> (bits - kSliceBits * (j + 1))) & 127ull);
}

int row_scale_exp(const double* row, int K) {
  double mx = 0.0;
  for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(row[k]));
  if (mx == 0.0) return 0;
  int e = 0;
  std::frexp(mx, &e);  // mx < 2^e
  return e;
}

// round-to-nearest-even BF16 bits of a float
inline uint16_t bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return uint16_t(u >> 16);
  u += 0x7fffu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}
inline double bf16_value(uint16_t b) {
  const uint32_t u = uint32_t(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return double(f);
}

// v = hi + mid + lo + (a remainder below 2^-24 |v|), each piece BF16
void split_host(double v, int KS, int* out) {
  double r = v;
  for (int j = 0; j < KS; ++j) {
    const uint16_t b = bf16_rne(float(r));
    out[j] = int(b);
    r -= bf16_value(b);
  }
}

inline uint16_t bf16_of_int(int x) {  // exact for |x| <= 256
  const float f = float(x);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return uint16_t(u >> 16);
}

// A (M x K, row-major FP64) -> fragment-ordered slices [KS][Mt][Kt][32 lanes] of
// 4 uint32 (2 bf16 each) for mma.m16n8k16 row-major A, plus row exponents.
// split = true: round-to-nearest BF16 pieces (already BF16 bit patterns), no exponents.
void slice_operator(const std::vector<double>& A, int M, int K, int KS, bool split, int& Mt, int& Kt,
                    std::vector<uint32_t>& frag, std::vector<int>& ea) {
  Mt = (M + 15) / 16;
  Kt = (K + 15) / 16;
  ea.assign(Mt * 16, 0);
  std::vector<int> sl(size_t(Mt) * 16 * Kt * 16 * KS, 0);  // [row][k][slice]
  for (int r = 0; r < M; ++r) {
    if (!split) ea[r] = row_scale_exp(&A[size_t(r) * K], K);
    for (int k = 0; k < K; ++k) {
      int* o = &sl[(size_t(r) * Kt * 16 + k) * KS];
      if (split) split_host(A[size_t(r) * K + k], KS, o);
      else slice_host(A[size_t(r) * K + k], ea[r], KS, o);
    }
  }
  auto S = [&](int r, int k, int i) { return sl[(size_t(r) * Kt * 16 + k) * KS + i]; };
  frag.assign(size_t(KS) * Mt * Kt * 32 * 4, 0);
  for (int i = 0; i < KS; ++i)
    for (int mt = 0; mt < Mt; ++mt)
      for (int kt = 0; kt < Kt; ++kt)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane >> 2, t = lane & 3;
          const int r0 = mt * 16 + g, r1 = r0 + 8, c0 = kt * 16 + 2 * t, c1 = c0 + 8;
          auto bits = [&](int r, int c) { return split ? uint16_t(S(r, c, i)) : bf16_of_int(S(r, c, i)); };
          auto pack = [&](int r, int c) { return uint32_t(bits(r, c)) | (uint32_t(bits(r, c + 1)) << 16); };
          uint32_t* q = &frag[((((size_t(i) * Mt + mt) * Kt + kt) * 32) + lane) * 4];
          q[0] = pack(r0, c0);
          q[1] = pack(r1, c0);
          q[2] = pack(r0, c1);
          q[3] = pack(r1, c1);
        }
}

// ---------------------------------------------------------------- device side
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// ldmatrix: 8x8 b16 matrices from shared memory, one 16-byte row address per
// lane (lanes 0-7 matrix 0, 8-15 matrix 1, ...); lane (g, t) receives row g,
// columns 2t, 2t+1 of each matrix: the B-fragment layout of mma m16n8k16 when
// rows are elements and columns the k index.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const void* p) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// (double) f * 2^sc built from the float's bits (exact; f normal or zero,
// result within the double range)
__device__ __forceinline__ double f2d_scaled(float f, int sc) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ef = (u >> 23) & 0xffu;
  if (ef == 0u) return 0.0;
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const unsigned long long e = (unsigned long long)(int(ef) - 127 + 1023 + sc) << 52;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(s | e | m));
}

// unbiased exponent e such that |v| < 2^e (a very negative value for zero)
__device__ __forceinline__ int exp_bound(double v) {
  const int E = int((__double_as_longlong(v) >> 52) & 0x7ff);
  return E == 0 ? -1100 : E - 1022;
}

// 8 signed 7-bit slices of v relative to 2^{sc} (|v| < 2^{sc}), as bf16 bits.
// I = floor(|v| 2^{56 - sc}) is formed as two 28-bit halves; each slice is a
// bit-field of one half, turned into a float exactly by OR-ing it into the
// mantissa of 2^23 and subtracting 2^23 (no integer-to-float conversion), whose
// top 16 bits are its bf16 pattern. A zero slice gives +-0, which adds nothing.
template <int KS>
__device__ __forceinline__ void slice_dev(double v, int sc, uint16_t (&s)[KS]) {
  static_assert(KS == 8, "FP64 slicing: 8 slices of 7 bits");
  const unsigned int hi = unsigned(__double2hiint(v)), lo = unsigned(__double2loint(v));
  const int E = int((hi >> 20) & 0x7ffu);
  const unsigned long long m = ((unsigned long long)((hi & 0xfffffu) | (E ? 0x100000u : 0u)) << 32) | lo;
  // |v| = m 2^{E-1075};  I = m 2^{sh}
  const int sh = (E ? E : 1) - 1075 + 56 - sc;
  unsigned long long I = 0;
  if (sh >= 0) I = sh < 11 ? (m << sh) : 0ull;  // I < 2^56 whenever |v| < 2^sc
  else if (sh > -63) I = m >> (-sh);
  const unsigned int H = unsigned(I >> 28), L = unsigned(I) & 0xfffffffu;
  const unsigned int sgn = (hi >> 31) << 15;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const unsigned int x = ((j < 4 ? H : L) >> (21 - 7 * (j & 3))) & 127u;
    const float f = __uint_as_float(0x4B000000u | x) - 8388608.0f;  // exactly x
    s[j] = uint16_t((__float_as_uint(f) >> 16) | sgn);
  }
}

// round-to-nearest BF16 pieces of an FP32 value (hi, mid, lo)
__device__ __forceinline__ void split_dev(float v, uint16_t (&s)[3]) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
  s[0] = __bfloat16_as_ushort(h);
  s[1] = __bfloat16_as_ushort(m);
  s[2] = __bfloat16_as_ushort(l);
}

// value -> stored pieces: exponent-scaled integer slices (FP64) or BF16 split (FP32)
template <int KS>
__device__ __forceinline__ void pieces(double v, int sc, uint16_t (&s)[KS]) { slice_dev<KS>(v, sc, s); }
template <int KS>
__device__ __forceinline__ void pieces(float v, int, uint16_t (&s)[KS]) { split_dev(v, s); }

// The product phase of a tile: out[e0 + n][r] = sum_k A[r][k] X[n][k] from the
// data slices Xs (per element n: scale exponent exs[n]) and the operator's
// fragment-ordered slices Af (row exponents ea). Warp w takes fragments
// w, w + OWARPS, ... (a fragment: 16 operator rows x 8 elements).
// With `add` set, out[e0 + n][r] += addsc[n] * add[(e0 + n) * ldadd + r].
template <int MAXF, int OWARPS, typename T>
__device__ __forceinline__ void oz_mma_tile(const uint16_t* __restrict__ Xs, const int* __restrict__ exs, int KP,
                                            int M, int Mt, int Kt, int ne, int64_t e0,
                                            const uint4* __restrict__ Af, const int* __restrict__ ea,
                                            T* __restrict__ out, int64_t ldo, const T* __restrict__ add = nullptr,
                                            int64_t ldadd = 0, const T* __restrict__ addsc = nullptr) {
  constexpr int KS = Slices<T>::KS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int nfrag = Mt * ONT;
#pragma unroll 1
  for (int q = 0; q < MAXF; ++q) {
    const int f = warp + OWARPS * q;
    if (f >= nfrag) break;
    const int mt = f / ONT, nt = f - mt * ONT;
    // FP64: one accumulator per slice-exponent sum i + j; FP32: all products in one
    constexpr int NACC = sizeof(T) == 8 ? KS : 1;
    float acc[NACC][4];
#pragma unroll
    for (int s = 0; s < NACC; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = 0.f;
    // ldmatrix row addresses: matrix m = lane >> 3 takes slice pair member m >> 1,
    // k half m & 1; row = element nt * 8 + (lane & 7)
    const int lrow = lane & 7, lmat = lane >> 3;
    const uint16_t* xrow = Xs + (size_t(nt) * 8 + lrow) * KP + 8 * (lmat & 1);
    for (int kt = 0; kt < Kt; ++kt) {
      uint32_t b0[KS], b1[KS];
#pragma unroll
      for (int j = 0; j + 1 < KS; j += 2) {
        uint32_t r[4];
        ldsm_x4(r, xrow + size_t(j + (lmat >> 1)) * OE * KP + kt * 16);
        b0[j] = r[0];
        b1[j] = r[1];
        b0[j + 1] = r[2];
        b1[j + 1] = r[3];
      }
      if (KS & 1) {  // the last slice: matrices 0 and 1 only
        uint32_t r[2];
        ldsm_x2(r, xrow + size_t(KS - 1) * OE * KP + kt * 16);
        b0[KS - 1] = r[0];
        b1[KS - 1] = r[1];
      }
#pragma unroll
      for (int i = 0; i < KS; ++i) {
        const uint4 a = __ldg(Af + ((size_t(i) * Mt + mt) * Kt + kt) * 32 + lane);
#pragma unroll
        for (int j = KS - 1 - i; j >= 0; --j) mma_bf16(acc[NACC == 1 ? 0 : i + j], a, b0[j], b1[j]);
      }
    }
    // recombine: value = 2^{ea_r + ex_e - 14} sum_s acc[s] 2^{-7 s}
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int r = mt * 16 + g + ((c & 2) ? 8 : 0);
      const int n = nt * 8 + 2 * t + (c & 1);
      if constexpr (sizeof(T) == 8) {
        float h = acc[NACC - 1][c], l = 0.f;
#pragma unroll
        for (int s = NACC - 2; s >= 0; --s) {
          const float hs = h * 0.0078125f, ls = l * 0.0078125f;  // exact scaling by 2^-7
          const float sum = acc[s][c] + hs;
          const float bb = sum - acc[s][c];
          const float err = (acc[s][c] - (sum - bb)) + (hs - bb);
          h = sum;
          l = ls + err;
        }
        if (r < M && n < ne) {
          T o = f2d_scaled(h, ea[r] + exs[n] - 14) + f2d_scaled(l, ea[r] + exs[n] - 14);
          if (add) o += addsc[n] * add[(e0 + n) * ldadd + r];
          out[(e0 + n) * ldo + r] = o;
        }
      } else {
        if (r < M && n < ne) {
          T o = acc[0][c];
          if (add) o += addsc[n] * add[(e0 + n) * ldadd + r];
          out[(e0 + n) * ldo + r] = o;
        }
      }
    }
  }
}

// out[e][r] = sum_k A[r][k] X[e][k] for e < nE, r < M.
// X rows have Kd entries at stride ldx; out rows stride ldo.
template <int MAXF, int OWARPS, typename T>
__global__ void __launch_bounds__(OWARPS * 32) oz_gemm(int64_t nE, int M, int Kd, int Mt, int Kt,
                                                    const uint4* __restrict__ Af, const int* __restrict__ ea,
                                                    const T* __restrict__ X, int64_t ldx, T* __restrict__ out,
                                                    int64_t ldo) {
  constexpr int KS = Slices<T>::KS;
  extern __shared__ __align__(16) uint16_t osm[];
  const int KP = Kt * 16 + 8;                 // row stride (bf16) of a slice; +8 breaks bank alignment
  uint16_t* Xs = osm;                         // [KS][OE][KP]
  int* exs = reinterpret_cast<int*>(osm + size_t(KS) * OE * KP);  // [OE]
  const int64_t ntiles = (nE + OE - 1) / OE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * OE;
    const int ne = int((nE - e0) < OE ? (nE - e0) : OE);
    __syncthreads();
    // one warp per element row: scale exponent as a warp maximum (FP64), then
    // the row's pieces; padding columns and rows past the tile's end are zero
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = warp; e < OE; e += OWARPS) {
      const T* xr = X + (e0 + e) * ldx;
      const bool live = e < ne;
      if (Kd <= 64) {
        // the row is read once into two registers per lane
        const T x0 = (live && lane < Kd) ? __ldg(xr + lane) : T(0);
        const T x1 = (live && lane + 32 < Kd) ? __ldg(xr + lane + 32) : T(0);
        int emax = -1100;
        if (sizeof(T) == 8 && live) {
          emax = max(exp_bound(x0), exp_bound(x1));
          emax = __reduce_max_sync(0xffffffffu, emax);
          if (lane == 0) exs[e] = emax;
        }
        for (int k = lane; k < Kt * 16; k += 32) {
          uint16_t s[KS];
          pieces<KS>(k < 32 ? x0 : x1, emax, s);  // zero (and padding) slices to zero
#pragma unroll
          for (int j = 0; j < KS; ++j) Xs[(size_t(j) * OE + e) * KP + k] = s[j];
        }
      } else {
        // long rows: a pass for the exponent, a pass for the slices
        int emax = -1100;
        if (sizeof(T) == 8 && live) {
          for (int k = lane; k < Kd; k += 32) emax = max(emax, exp_bound(__ldg(xr + k)));
          emax = __reduce_max_sync(0xffffffffu, emax);
          if (lane == 0) exs[e] = emax;
        }
        for (int k = lane; k < Kt * 16; k += 32) {
          uint16_t s[KS];
          pieces<KS>((live && k < Kd) ? __ldg(xr + k) : T(0), emax, s);
#pragma unroll
          for (int j = 0; j < KS; ++j) Xs[(size_t(j) * OE + e) * KP + k] = s[j];
        }
      }
    }
    __syncthreads();
    oz_mma_tile<MAXF, OWARPS, T>(Xs, exs, KP, M, Mt, Kt, ne, e0, Af, ea, out, ldo);
  }
}

__device__ __forceinline__ int fnode_rt(int N, int f, int j) {
  auto rs = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

// The output product with the pointwise stage fused into its slicing phase:
// warp w builds the Y row of element n (columns: wr, ws (Np each) |
// 1/2 nr sJ [u], 1/2 ns sJ [u] (NFN each) | -sJ ({n.grad u} + tau [u]) (NFN))
// in registers, from C1, u, the geometry
// gx (16 words per element: J, Grr, Grs, Gss | per face nr, ns, sJ, ihmax) and
// the neighbours' C1 and u rows; takes the row's scale exponent as a warp
// maximum and writes the slices straight to shared memory. For the Helmholtz
// form C1 carries a third block M u (rows 2Np..3Np of the first product) and
// the epilogue adds lambda J (M u), which keeps the output product as narrow as
// the Poisson one.
// Per-lane constants of the fused fill (the same for every element): volume
// nodes lane and lane + 32, face node q = lane (face f, position jf, local node
// kf), and the neighbour's matching node for each of its three possible faces.
struct LaneNodes {
  bool vol0, vol1, fq;
  int f, jf, kf, kn0, kn1, kn2;
};
__device__ __forceinline__ LaneNodes lane_nodes(int N, int lane) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  LaneNodes L;
  L.vol0 = lane < Np;
  L.vol1 = lane + 32 < Np;
  L.fq = lane < NFN;
  L.f = L.fq ? lane / Nfp : 0;
  L.jf = L.fq ? lane - L.f * Nfp : 0;
  L.kf = fnode_rt(N, L.f, L.jf);
  L.kn0 = fnode_rt(N, 0, Nfp - 1 - L.jf);
  L.kn1 = fnode_rt(N, 1, Nfp - 1 - L.jf);
  L.kn2 = fnode_rt(N, 2, Nfp - 1 - L.jf);
  return L;
}

// The fused fill of one tile by the warps fw, fw + nfw, ... (one element row
// per warp at a time): the Y row of element n (columns: wr, ws (Np each) |
// 1/2 nr sJ [u], 1/2 ns sJ [u] (NFN each) | -sJ ({n.grad u} + tau [u]) (NFN))
// from C1, u, the geometry gx (16 words per element: J, Grr, Grs, Gss | per
// face nr, ns, sJ, ihmax) and the neighbours' C1 and u rows; the row's scale
// exponent as a warp maximum (FP64); the slices into Xs; lambda J into addsc.
template <typename T>
__device__ __forceinline__ void oz_fill(int fw, int nfw, int lane, const LaneNodes& Ln, int N, int64_t K, int Kd,
                                        int Kt, int KP, int64_t e0, int ne, const T* __restrict__ gx,
                                        const int32_t* __restrict__ conn, const T* __restrict__ u,
                                        const T* __restrict__ C1, int ldc, T lambda, uint16_t* Xs, int* exs,
                                        T* addsc) {
  constexpr int KS = Slices<T>::KS;
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  const T cpen = T((N + 1) * (N + 2)) / T(2);
  const bool vol0 = Ln.vol0, vol1 = Ln.vol1, fq = Ln.fq;
  const int f = Ln.f, kf = Ln.kf, kn0 = Ln.kn0, kn1 = Ln.kn1, kn2 = Ln.kn2;
  (void)Nfp;
  for (int n = fw; n < OE; n += nfw) {
    // slots: 0-1 (wr, ws) at node lane, 2-3 at node lane + 32, 4-6 at face node lane
    T v[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = T(0);
    const bool live = n < ne;
    if (live) {
      const int64_t be = e0 + n;
      const int64_t e = be < K ? be : be % K;  // first right-hand side: no division
      const int64_t boff = be - e;
      const T* g = gx + 16 * e;
      const T* c = C1 + be * ldc;
      if (lane == 0) addsc[n] = lambda * g[0];
      const T g1 = g[1], g2 = g[2], g3 = g[3];
      if (vol0) {
        const T ur = c[lane], us = c[Np + lane];
        v[0] = g1 * ur + g2 * us;
        v[1] = g2 * ur + g3 * us;
      }
      if (vol1) {
        const T ur = c[lane + 32], us = c[Np + lane + 32];
        v[2] = g1 * ur + g2 * us;
        v[3] = g2 * ur + g3 * us;
      }
      if (fq) {
        const T nr = g[4 + 4 * f], ns = g[5 + 4 * f], sJ = g[6 + 4 * f], tau = cpen * g[7 + 4 * f];
        const T um = u[be * Np + kf];
        const T dnm = nr * c[kf] + ns * c[Np + kf];
        const int code = conn[3 * e + f];
        T jm = T(0), av = T(0);
        if (code >= 0) {
          const int64_t nb = code >> 2;
          const int fn = code & 3;
          const int kn = fn == 0 ? kn0 : (fn == 1 ? kn1 : kn2);
          const T* gn = gx + 16 * nb + 4 + 4 * fn;
          const T* cn = C1 + (boff + nb) * ldc;
          const T up = u[(boff + nb) * Np + kn];
          const T dnp = gn[0] * cn[kn] + gn[1] * cn[Np + kn];
          jm = up - um;
          av = T(0.5) * (dnm - dnp);
        } else if (code == -2) {
          jm = T(-2) * um;
          av = dnm;
        }
        const T hs = T(0.5) * sJ * jm;
        v[4] = nr * hs;
        v[5] = ns * hs;
        v[6] = -sJ * (av + tau * jm);
      }
    }
    const bool w0 = live && vol0, w1 = live && vol1, wf = live && fq;
    int emax = -1100;
    if constexpr (sizeof(T) == 8) {
      if (w0) emax = max(emax, max(exp_bound(v[0]), exp_bound(v[1])));
      if (w1) emax = max(emax, max(exp_bound(v[2]), exp_bound(v[3])));
      if (wf) emax = max(emax, max(exp_bound(v[4]), max(exp_bound(v[5]), exp_bound(v[6]))));
      emax = __reduce_max_sync(0xffffffffu, emax);
      if (lane == 0) exs[n] = emax;
    }
    uint16_t* row = Xs + size_t(n) * KP;  // slice jj of this row at row + jj * OE * KP
    auto put = [&](T val, int colx) {
      uint16_t sl[KS];
      pieces<KS>(val, emax, sl);
#pragma unroll
      for (int jj = 0; jj < KS; ++jj) row[size_t(jj) * OE * KP + colx] = sl[jj];
    };
    if (w0) {
      put(v[0], lane);
      put(v[1], Np + lane);
    }
    if (w1) {
      put(v[2], lane + 32);
      put(v[3], Np + lane + 32);
    }
    if (wf) {
      put(v[4], 2 * Np + lane);
      put(v[5], 2 * Np + NFN + lane);
      put(v[6], 2 * Np + 2 * NFN + lane);
    }
    // zero padding: the columns past Kd, or the whole row past the tile's end
    for (int k = (live ? Kd : 0) + lane; k < Kt * 16; k += 32)
#pragma unroll
      for (int jj = 0; jj < KS; ++jj) row[size_t(jj) * OE * KP + k] = 0;
  }
}

template <int MAXF, int OWARPS, typename T>
__global__ void __launch_bounds__(OWARPS * 32) oz_out(int N, int64_t K, int64_t nE, int Kd, int Mt, int Kt,
                                                   const T* __restrict__ gx, const int32_t* __restrict__ conn,
                                                   const T* __restrict__ u, const T* __restrict__ C1, int ldc,
                                                   T lambda, const uint4* __restrict__ Af,
                                                   const int* __restrict__ ea, T* __restrict__ out) {
  constexpr int KS = Slices<T>::KS;
  extern __shared__ __align__(16) uint16_t osm[];
  const int KP = Kt * 16 + 8;
  uint16_t* Xs = osm;
  int* exs = reinterpret_cast<int*>(osm + size_t(KS) * OE * KP);
  T* addsc = reinterpret_cast<T*>(exs + OE);  // [OE]: lambda J per element (Helmholtz)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Np = (N + 1) * (N + 2) / 2;
  const LaneNodes Ln = lane_nodes(N, lane);
  const int64_t ntiles = (nE + OE - 1) / OE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * OE;
    const int ne = int((nE - e0) < OE ? (nE - e0) : OE);
    __syncthreads();
    oz_fill<T>(warp, OWARPS, lane, Ln, N, K, Kd, Kt, KP, e0, ne, gx, conn, u, C1, ldc, lambda, Xs, exs, addsc);
    __syncthreads();
    if (lambda != T(0))  // + lambda J (M u), M u being C1's third block
      oz_mma_tile<MAXF, OWARPS, T>(Xs, exs, KP, Np, Mt, Kt, ne, e0, Af, ea, out, Np, C1 + 2 * Np, ldc, addsc);
    else
      oz_mma_tile<MAXF, OWARPS, T>(Xs, exs, KP, Np, Mt, Kt, ne, e0, Af, ea, out, Np);
  }
}

// ------------------------------------------------ pipelined output product
// The same output product with its fill and product phases on separate warps:
// 8 producer warps fill tile i + 1 into one of two shared-memory stages while
// 8 consumer warps run the products and epilogue of tile i from the other.
// The hand-off uses two mbarriers per stage (full: all 256 producer threads
// arrive after writing; empty: all 256 consumer threads arrive after reading),
// waited on by phase parity. Every wait gives up after a fixed number of
// polls, sets g_tensor_err and leaves the loop, so a broken hand-off ends the
// kernel with an error flag instead of hanging it.
__device__ int g_tensor_err;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Warp-collective: true once the phase of barrier b with the given parity has
// completed (seen by every lane), false after one second (the time-bounded
// wait of tc05.cuh). The vote keeps the warp converged, so the aligned
// ldmatrix / mma / shuffle instructions that follow see all 32 lanes, and a
// timeout leaves the loop with the whole warp.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) { return tc::mbar_wait(b, parity); }

template <int MAXF, typename T>
__global__ void __launch_bounds__(512, 1) oz_out_pipe(int N, int64_t K, int64_t nE, int Kd, int Mt, int Kt,
                                                   const T* __restrict__ gx, const int32_t* __restrict__ conn,
                                                   const T* __restrict__ u, const T* __restrict__ C1, int ldc,
                                                   T lambda, const uint4* __restrict__ Af,
                                                   const int* __restrict__ ea, T* __restrict__ out) {
  constexpr int KS = Slices<T>::KS;
  constexpr int NW = 8;  // warps per role
  extern __shared__ __align__(16) uint16_t osm[];
  const int KP = Kt * 16 + 8;
  const size_t stage = size_t(KS) * OE * KP;  // bf16 words of one stage's slices
  int* exs_all = reinterpret_cast<int*>(osm + 2 * stage);  // [2][OE]
  T* addsc_all = reinterpret_cast<T*>(exs_all + 2 * OE);   // [2][OE]
  uint64_t* bar = reinterpret_cast<uint64_t*>(addsc_all + 2 * OE);  // full[2], empty[2]
  if (threadIdx.x == 0) {
    mbar_init(bar + 0, NW * 32);
    mbar_init(bar + 1, NW * 32);
    mbar_init(bar + 2, NW * 32);
    mbar_init(bar + 3, NW * 32);
  }
  __syncthreads();  // the only CTA-wide barrier: before the roles split
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool producer = warp >= NW;
  const int Np = (N + 1) * (N + 2) / 2;
  const LaneNodes Ln = lane_nodes(N, lane);
  const int64_t ntiles = (nE + OE - 1) / OE;
  unsigned use = 0;  // tile counter of this CTA: stage = use & 1, round = use >> 1
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++use) {
    const int s = int(use & 1u);
    const unsigned parity = (use >> 1) & 1u;
    uint16_t* Xs = osm + s * stage;
    int* exs = exs_all + s * OE;
    T* addsc = addsc_all + s * OE;
    const int64_t e0 = tile * OE;
    const int ne = int((nE - e0) < OE ? (nE - e0) : OE);
    if (producer) {
      // the stage is free once the consumers released its previous round
      // (the first round waits on the already-complete parity, i.e. not at all)
      if (!mbar_wait(bar + 2 + s, parity ^ 1u)) {
        atomicExch(&g_tensor_err, 1);
        break;
      }
      oz_fill<T>(warp - NW, NW, lane, Ln, N, K, Kd, Kt, KP, e0, ne, gx, conn, u, C1, ldc, lambda, Xs, exs, addsc);
      mbar_arrive(bar + s);
    } else {
      if (!mbar_wait(bar + s, parity)) {
        atomicExch(&g_tensor_err, 1);
        break;
      }
      if (lambda != T(0))
        oz_mma_tile<MAXF, NW, T>(Xs, exs, KP, Np, Mt, Kt, ne, e0, Af, ea, out, Np, C1 + 2 * Np, ldc, addsc);
      else
        oz_mma_tile<MAXF, NW, T>(Xs, exs, KP, Np, Mt, Kt, ne, e0, Af, ea, out, Np);
      mbar_arrive(bar + 2 + s);
    }
  }
}

// arguments of the fused output product (null: plain product from X)
template <typename T>
struct FusedArgs {
  int N;
  int64_t K;
  const T* gx;
  const int32_t* conn;
  const T* u;
  const T* C1;
  int ldc;
  T lambda;
};

struct OzOps {
  int Mt1 = 0, Kt1 = 0, Mt1h = 0, Mt2 = 0, Kt2 = 0;
  uint4 *A1 = nullptr, *A1h = nullptr, *A2 = nullptr;  // [Dr; Ds], [Dr; Ds; M], OB
  int *ea1 = nullptr, *ea1h = nullptr, *ea2 = nullptr;
};

cudaError_t build_oz_ops(const RefElem& R, int KS, bool split, OzOps& o) {
  const int N = R.N, Np = R.Np, Nfp = R.Nfp, NFN = 3 * Nfp;
  // [Dr; Ds; M]: 3Np x Np (the Poisson form uses the first 2Np rows)
  std::vector<double> A1(size_t(3 * Np) * Np);
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < Np; ++m) {
      A1[size_t(i) * Np + m] = R.Dr[size_t(i) * Np + m];
      A1[size_t(Np + i) * Np + m] = R.Ds[size_t(i) * Np + m];
      A1[size_t(2 * Np + i) * Np + m] = R.M[size_t(i) * Np + m];
    }
  // OB: Np x (2Np + 3NFN)
  const int Kc = 2 * Np + 3 * NFN;
  std::vector<double> B(size_t(Np) * Kc, 0.0);
  for (int i = 0; i < Np; ++i) {
    for (int m = 0; m < Np; ++m) {
      B[size_t(i) * Kc + m] = R.Br[size_t(i) * Np + m];
      B[size_t(i) * Kc + Np + m] = R.Bs[size_t(i) * Np + m];
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
        B[size_t(i) * Kc + 2 * Np + f * Nfp + l] = dr;
        B[size_t(i) * Kc + 2 * Np + NFN + f * Nfp + l] = ds;
        B[size_t(i) * Kc + 2 * Np + 2 * NFN + f * Nfp + l] = ef;
      }
  }
  std::vector<uint32_t> f1, f1h, f2;
  std::vector<int> e1, e1h, e2;
  int Kt1h = 0;
  slice_operator(std::vector<double>(A1.begin(), A1.begin() + size_t(2 * Np) * Np), 2 * Np, Np, KS, split, o.Mt1,
                 o.Kt1, f1, e1);
  slice_operator(A1, 3 * Np, Np, KS, split, o.Mt1h, Kt1h, f1h, e1h);
  slice_operator(B, Np, Kc, KS, split, o.Mt2, o.Kt2, f2, e2);
  auto up = [](auto& dst, const auto& v) -> cudaError_t {
    cudaError_t e = cudaMalloc(&dst, v.size() * sizeof(v[0]));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
  };
  cudaError_t e;
  if ((e = up(o.A1, f1)) != cudaSuccess) return e;
  if ((e = up(o.A1h, f1h)) != cudaSuccess) return e;
  if ((e = up(o.A2, f2)) != cudaSuccess) return e;
  if ((e = up(o.ea1, e1)) != cudaSuccess) return e;
  if ((e = up(o.ea1h, e1h)) != cudaSuccess) return e;
  return up(o.ea2, e2);
}

template <int MAXF, int OWARPS, typename T>
cudaError_t launch_gemm(int64_t nE, int M, int Kd, int Mt, int Kt, const uint4* Af, const int* ea, const T* X,
                        int64_t ldx, T* out, int64_t ldo, const FusedArgs<T>* fa, cudaStream_t st) {
  constexpr int OTHREADS = OWARPS * 32;
  const size_t smem = size_t(Slices<T>::KS) * OE * (Kt * 16 + 8) * sizeof(uint16_t) + OE * sizeof(int) +
                      OE * sizeof(T);
  static size_t configured[64][2] = {};  // per device and variant: the largest dynamic shared memory set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* kern = fa ? reinterpret_cast<const void*>(oz_out<MAXF, OWARPS, T>)
                        : reinterpret_cast<const void*>(oz_gemm<MAXF, OWARPS, T>);
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    if (configured[dev & 63][fa ? 1 : 0] < smem) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
      configured[dev & 63][fa ? 1 : 0] = smem;
    }
  }
  int sms = 0, per = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, OTHREADS, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (nE + OE - 1) / OE;
  int64_t grid = int64_t(sms) * (per > 0 ? per : 1);
  if (grid > tiles) grid = tiles;
  if (fa)
    oz_out<MAXF, OWARPS, T><<<unsigned(grid), OTHREADS, smem, st>>>(fa->N, fa->K, nE, Kd, Mt, Kt, fa->gx, fa->conn,
                                                                   fa->u, fa->C1, fa->ldc, fa->lambda, Af, ea, out);
  else
    oz_gemm<MAXF, OWARPS, T><<<unsigned(grid), OTHREADS, smem, st>>>(nE, M, Kd, Mt, Kt, Af, ea, X, ldx, out, ldo);
  note_launch();
  return cudaGetLastError();
}

// 8 warps per CTA (the fill phase, one warp per element, wants them even where
// the product phase leaves some idle: measured faster than 6 at 12 fragments),
// except for products of at most 4 fragments (small degrees), where 4 warps
// per CTA measured faster. Every fragment must be covered (MAXF x warps >= fragments).
template <typename T>
cudaError_t gemm(int Mt, int64_t nE, int M, int Kd, int Kt, const uint4* Af, const int* ea, const T* X, int64_t ldx,
                 T* out, int64_t ldo, const FusedArgs<T>* fa, cudaStream_t st) {
  const int nfrag = Mt * ONT;
  if (nfrag <= 4) return launch_gemm<1, 4, T>(nE, M, Kd, Mt, Kt, Af, ea, X, ldx, out, ldo, fa, st);
#define OZ_L(F) return launch_gemm<F, 8, T>(nE, M, Kd, Mt, Kt, Af, ea, X, ldx, out, ldo, fa, st)
  switch ((nfrag + 7) / 8) {
    case 1: OZ_L(1);
    case 2: OZ_L(2);
    case 3: OZ_L(3);
    case 4: OZ_L(4);
    case 5: OZ_L(5);
    case 6: OZ_L(6);
    default: break;
  }
#undef OZ_L
  return cudaErrorInvalidValue;  // more fragments than any instantiation covers
}

template <int MAXF, typename T>
cudaError_t launch_pipe(int64_t nE, int Kd, int Mt, int Kt, const uint4* Af, const int* ea, T* out,
                        const FusedArgs<T>& fa, cudaStream_t st) {
  const size_t smem = 2 * (size_t(Slices<T>::KS) * OE * (Kt * 16 + 8) * sizeof(uint16_t) + OE * sizeof(int) +
                           OE * sizeof(T)) + 4 * sizeof(uint64_t);
  static size_t configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    if (configured[dev & 63] < smem) {
      e = cudaFuncSetAttribute(oz_out_pipe<MAXF, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (e != cudaSuccess) return e;
      configured[dev & 63] = smem;
    }
  }
  int sms = 0, per = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, oz_out_pipe<MAXF, T>, 512, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;  // the two stages do not fit
  const int64_t tiles = (nE + OE - 1) / OE;
  int64_t grid = int64_t(sms) * per;
  if (grid > tiles) grid = tiles;
  oz_out_pipe<MAXF, T><<<unsigned(grid), 512, smem, st>>>(fa.N, fa.K, nE, Kd, Mt, Kt, fa.gx, fa.conn, fa.u, fa.C1,
                                                          fa.ldc, fa.lambda, Af, ea, out);
  note_launch();
  return cudaGetLastError();
}

// the pipelined output product: 8 consumer warps cover every fragment
template <typename T>
cudaError_t gemm_pipe(int Mt, int64_t nE, int Kd, int Kt, const uint4* Af, const int* ea, T* out,
                      const FusedArgs<T>& fa, cudaStream_t st) {
  switch ((Mt * ONT + 7) / 8) {
    case 1: return launch_pipe<1, T>(nE, Kd, Mt, Kt, Af, ea, out, fa, st);
    case 2: return launch_pipe<2, T>(nE, Kd, Mt, Kt, Af, ea, out, fa, st);
    case 3: return launch_pipe<3, T>(nE, Kd, Mt, Kt, Af, ea, out, fa, st);
    default: return cudaErrorInvalidValue;
  }
}

OzOps g_oz[2][64][kMaxN + 1];  // [0: FP64, 1: FP32][device][degree]

// The per-device operator slices of one degree and precision, built on first
// use (under the table lock; the slices of a built entry never change).
template <typename T>
cudaError_t tensor_ops(dg_mesh* m, int degree, const OzOps** out) {
  constexpr bool f64 = sizeof(T) == 8;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(table_mutex());
  OzOps& o = g_oz[f64 ? 0 : 1][dev & 63][degree];
  if (!o.A1) {
    const RefElem R = m->ref[degree].N ? m->ref[degree] : build_reference(degree);
    OzOps built;
    e = build_oz_ops(R, Slices<T>::KS, !f64, built);
    if (e != cudaSuccess) return e;
    o = built;
  }
  *out = &o;
  return cudaSuccess;
}

template <typename T>
cudaError_t apply_tensor(dg_mesh* m, int degree, int B, double lambda, const T* u, T* Au, bool pipe,
                         cudaStream_t st, double* c1_scratch) {
  constexpr bool f64 = sizeof(T) == 8;
  if (!tensor_supported(degree)) return cudaErrorInvalidValue;
  const OzOps* op = nullptr;
  cudaError_t e = tensor_ops<T>(m, degree, &op);
  if (e != cudaSuccess) return e;
  const OzOps& o = *op;
  const int N = degree, Np = (N + 1) * (N + 2) / 2, NFN = 3 * (N + 1);
  const bool helm = lambda != 0.0;
  const int KY = 2 * Np + 3 * NFN;
  const int ldc = helm ? 3 * Np : 2 * Np;  // C1 rows: ur, us (+ M u)
  const int64_t nE = int64_t(B) * m->K;
  const size_t words = size_t(nE) * ldc * sizeof(T) / sizeof(double) + 1;
  if (!c1_scratch && m->oz_cap < words) {
    cudaFree(m->oz_scratch);
    m->oz_scratch = nullptr;
    m->oz_cap = 0;
    e = cudaMalloc(&m->oz_scratch, words * sizeof(double));
    if (e == cudaSuccess) e = poison(m->oz_scratch, words * sizeof(double), POISON_APPLY);
    if (e != cudaSuccess) return e;
    m->oz_cap = words;
    ++m->scratch_gen;
  }
  T* C1 = reinterpret_cast<T*>(c1_scratch ? c1_scratch : m->oz_scratch);
  const T* gx = f64 ? reinterpret_cast<const T*>(m->geox) : reinterpret_cast<const T*>(m->geox32);
  if (helm) e = gemm<T>(o.Mt1h, nE, 3 * Np, Np, o.Kt1, o.A1h, o.ea1h, u, Np, C1, ldc, nullptr, st);
  else e = gemm<T>(o.Mt1, nE, 2 * Np, Np, o.Kt1, o.A1, o.ea1, u, Np, C1, ldc, nullptr, st);
  if (e != cudaSuccess) return e;
  const FusedArgs<T> fa{N, m->K, gx, m->conn, u, C1, ldc, T(lambda)};
  if (pipe) return gemm_pipe<T>(o.Mt2, nE, KY, o.Kt2, o.A2, o.ea2, Au, fa, st);
  return gemm<T>(o.Mt2, nE, Np, KY, o.Kt2, o.A2, o.ea2, nullptr, 0, Au, Np, &fa, st);
}

}  // namespace

cudaError_t launch_apply_tensor(dg_mesh* m, int degree, bool f64, int B, double lambda, const void* u, void* Au,
                                bool pipe, cudaStream_t st, double* c1_scratch) {
  if (f64)
    return apply_tensor<double>(m, degree, B, lambda, static_cast<const double*>(u), static_cast<double*>(Au), pipe,
                                st, c1_scratch);
  return apply_tensor<float>(m, degree, B, lambda, static_cast<const float*>(u), static_cast<float*>(Au), pipe, st,
                             c1_scratch);
}

// The fill phase maps a node to lane and lane + 32 and a face-node entry to a
// lane: Np <= 64 and 3 (N + 1) <= 32, so degrees up to 9.
bool tensor_supported(int degree) { return degree >= 1 && degree <= 9; }

bool tensor_ops_ready(int degree, bool f64) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lk(table_mutex());
  return g_oz[f64 ? 0 : 1][dev & 63][degree].A1 != nullptr;
}

cudaError_t ensure_tensor_ops(dg_mesh* m, int degree, bool f64) {
  if (!tensor_supported(degree)) return cudaSuccess;
  const OzOps* op = nullptr;
  return f64 ? tensor_ops<double>(m, degree, &op) : tensor_ops<float>(m, degree, &op);
}

// A general FP64 operator for batched row products out[r] = A X[r] (the
// advection's cubature interpolation and projection): sliced once on the host.
cudaError_t sliced_op_create(const std::vector<double>& A, int M, int K, SlicedOp* op) {
  std::vector<uint32_t> frag;
  std::vector<int> ea;
  op->M = M;
  op->K = K;
  // too long a sum for the FP32 group sums to stay exact (both kernels: 4 products
  // of |slice| <= 127 over 256 terms stay below 2^24)
  if (K > 256) return cudaErrorInvalidValue;
  // the tcgen05 GEMM takes any row count; the mma.sync copy only within its
  // instantiated shapes (it serves when the tcgen05 one is not built)
  cudaError_t e = tc64_op_create(A, M, K, &op->t64);
  if (e != cudaSuccess) return e;
  slice_operator(A, M, K, Slices<double>::KS, false, op->Mt, op->Kt, frag, ea);
  if (op->Mt * ONT > 48) return cudaSuccess;
  e = cudaMalloc(&op->A, frag.size() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(op->A, frag.data(), frag.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&op->ea, ea.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(op->ea, ea.data(), ea.size() * sizeof(int), cudaMemcpyHostToDevice);
  return e;
}

void sliced_op_free(SlicedOp* op) {
  cudaFree(op->A);
  cudaFree(op->ea);
  op->A = nullptr;
  op->ea = nullptr;
  tc64_op_free(&op->t64);
}

cudaError_t sliced_gemm(const SlicedOp& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                        cudaStream_t st) {
  if (op.t64.blocks) return tc64_gemm_launch(op.t64, rows, X, ldx, out, ldo, st);
  if (!op.A) return cudaErrorInvalidValue;
  return gemm<double>(op.Mt, rows, op.M, op.K, op.Kt, reinterpret_cast<const uint4*>(op.A), op.ea, X, ldx, out, ldo,
                      nullptr, st);
}

// Reads and clears the pipelined kernels' timeout flag (synchronises the device).
cudaError_t tensor_pipe_error(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tensor_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tensor_err, &zero, sizeof(int));
  return e;
}

}  // namespace dgx
