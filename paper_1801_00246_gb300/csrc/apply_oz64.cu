// FP64-accurate SIPDG apply with its dense products on the BF16 tensor cores.
//
// GB300 executes FP64 at 1/62 of its FP32 rate, so the FP64 tile kernel
// (apply.cu) is bound by the FP64 pipe. Here the two dense products of the
// operator (Eq. ellipticOp3 written as in apply_gemm.cuh),
//   C1 = [Dr; Ds] U   and   Au = OB Y,
// are evaluated exactly enough for FP64 with integer-sliced BF16 products
// (the error-free splitting of Ozaki et al., "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012):
//   * every operator row r is scaled by a power of two 2^{ea_r} and written as
//     sum_i a_i 2^{-7i}, i = 1..8, a_i signed integers |a_i| <= 127 (host);
//   * every element's data column is scaled by 2^{ex_e} and sliced the same way
//     on the fly from the FP64 bit pattern (integer shifts, no FP64 work);
//   * a_i x_j products summed over K <= 176 are integers below 2^22, exact in the
//     FP32 accumulators of mma.sync m16n8k16; products with the same i + j share
//     an accumulator (exact up to the 2^-49 level), i + j <= 9 (36 products),
//     which leaves a relative error near 2^-44 of |A||x|;
//   * the 8 accumulators are combined by Horner's rule in float-float
//     arithmetic and converted to FP64 once.
// The face mass is folded into the output operator
//   OB = [Br Bs | Dr_f^T Mf  Ds_f^T Mf | E_f Mf | M],
// so the pointwise stage between the two products only forms
//   Y = [wr; ws; 1/2 nr sJ [u]; 1/2 ns sJ [u]; -sJ ({n.grad u} + tau [u]); lambda J u].
// The pointwise stage runs inside the output product's slicing phase (Y is
// built in shared memory, never in HBM); the neighbour's trace and normal
// derivative at a shared face node are read from its nodal values and its
// rows of C1.
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_internal.h"

namespace dgx {
namespace {

constexpr int kSlices = 8;        // 7-bit slices per operand: 56 bits
constexpr int kSliceBits = 7;
constexpr int kGroups = 8;        // i + j = 2..9 -> 8 accumulators
constexpr int OE = 32;            // elements per CTA tile
constexpr int ONT = OE / 8;       // n-tiles (8 elements each)


// ---------------------------------------------------------------- host side
// Slices of one FP64 value relative to 2^{scale_exp} (|v| < 2^{scale_exp}):
// floor(|v| 2^{56 - scale_exp}) cut into 8 chunks of 7 bits, sign applied.
void slice_host(double v, int scale_exp, int out[kSlices]) {
  for (int j = 0; j < kSlices; ++j) out[j] = 0;
  if (v == 0.0 || !std::isfinite(v)) return;
  int e = 0;
  const double fr = std::frexp(std::fabs(v), &e);  // |v| = fr 2^e, fr in [0.5, 1)
  // |v| 2^{56 - scale_exp} = fr 2^{e + 56 - scale_exp}
  const int sh = e + 56 - scale_exp;
  if (sh <= 0) return;
  const unsigned long long I = (unsigned long long)std::ldexp(fr, sh);  // exact for sh <= 53, truncated beyond
  const int sgn = v < 0 ? -1 : 1;
  for (int j = 0; j < kSlices; ++j) out[j] = sgn * int((I >> (56 - kSliceBits * (j + 1))) & 127ull);
}

int row_scale_exp(const double* row, int K) {
  double mx = 0.0;
  for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(row[k]));
  if (mx == 0.0) return 0;
  int e = 0;
  std::frexp(mx, &e);  // mx < 2^e
  return e;
}

inline uint16_t bf16_of_int(int x) {  // exact for |x| <= 256
  const float f = float(x);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return uint16_t(u >> 16);
}

// A (M x K, row-major FP64) -> fragment-ordered slices [8][Mt][Kt][32 lanes] of
// 4 uint32 (2 bf16 each) for mma.m16n8k16 row-major A, plus row exponents.
void slice_operator(const std::vector<double>& A, int M, int K, int& Mt, int& Kt, std::vector<uint32_t>& frag,
                    std::vector<int>& ea) {
  Mt = (M + 15) / 16;
  Kt = (K + 15) / 16;
  ea.assign(Mt * 16, 0);
  std::vector<int> sl(size_t(Mt) * 16 * Kt * 16 * kSlices, 0);  // [row][k][slice]
  for (int r = 0; r < M; ++r) {
    ea[r] = row_scale_exp(&A[size_t(r) * K], K);
    for (int k = 0; k < K; ++k) slice_host(A[size_t(r) * K + k], ea[r], &sl[(size_t(r) * Kt * 16 + k) * kSlices]);
  }
  auto S = [&](int r, int k, int i) { return sl[(size_t(r) * Kt * 16 + k) * kSlices + i]; };
  frag.assign(size_t(kSlices) * Mt * Kt * 32 * 4, 0);
  for (int i = 0; i < kSlices; ++i)
    for (int mt = 0; mt < Mt; ++mt)
      for (int kt = 0; kt < Kt; ++kt)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane >> 2, t = lane & 3;
          const int r0 = mt * 16 + g, r1 = r0 + 8, c0 = kt * 16 + 2 * t, c1 = c0 + 8;
          auto pack = [&](int r, int c) {
            return uint32_t(bf16_of_int(S(r, c, i))) | (uint32_t(bf16_of_int(S(r, c + 1, i))) << 16);
          };
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

// unbiased exponent e such that |v| < 2^e (0 for v = 0)
__device__ __forceinline__ int exp_bound(double v) {
  const long long b = __double_as_longlong(v);
  const int E = int((b >> 52) & 0x7ff);
  return E == 0 ? -1100 : E - 1022;
}

// 8 signed 7-bit slices of v relative to 2^{sc} (|v| < 2^{sc}), as packed bf16 bits
__device__ __forceinline__ void slice_dev(double v, int sc, uint16_t (&s)[kSlices]) {
  const long long b = __double_as_longlong(v);
  const int E = int((b >> 52) & 0x7ff);
  const unsigned long long m = (unsigned long long)(b & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  // |v| = m 2^{E-1075};  I = floor(|v| 2^{56 - sc}) = m 2^{E - 1075 + 56 - sc}
  const int sh = (E ? E : 1) - 1019 - sc;
  unsigned long long I = 0;
  if (sh >= 0) I = sh < 11 ? (m << sh) : 0ull;  // sh <= 3 whenever |v| < 2^sc
  else if (sh > -63) I = m >> (-sh);
  const uint16_t sgn = (b < 0) ? 0x8000 : 0;
#pragma unroll
  for (int j = 0; j < kSlices; ++j) {
    const int x = int((I >> (56 - kSliceBits * (j + 1))) & 127ull);
    const uint16_t bits = uint16_t(__float_as_uint(float(x)) >> 16);
    s[j] = x ? (bits | sgn) : 0;
  }
}

// The product phase of a tile: out[e0 + n][r] = sum_k A[r][k] X[n][k] from the
// data slices Xs (per element n: scale exponent exs[n]) and the operator's
// fragment-ordered slices Af (row exponents ea). Warp w takes fragments
// w, w + OWARPS, ... (a fragment: 16 operator rows x 8 elements).
template <int MAXF, int OWARPS>
__device__ __forceinline__ void oz_mma_tile(const uint16_t* __restrict__ Xs, const int* __restrict__ exs, int KP,
                                            int M, int Mt, int Kt, int ne, int64_t e0,
                                            const uint4* __restrict__ Af, const int* __restrict__ ea,
                                            double* __restrict__ out, int64_t ldo) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int nfrag = Mt * ONT;
#pragma unroll 1
  for (int q = 0; q < MAXF; ++q) {
    const int f = warp + OWARPS * q;
    if (f >= nfrag) break;
    const int mt = f / ONT, nt = f - mt * ONT;
    float acc[kGroups][4];
#pragma unroll
    for (int s = 0; s < kGroups; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = 0.f;
    for (int kt = 0; kt < Kt; ++kt) {
      uint32_t b0[kSlices], b1[kSlices];
#pragma unroll
      for (int j = 0; j < kSlices; ++j) {
        const uint16_t* col = Xs + (size_t(j) * OE + nt * 8 + g) * KP + kt * 16 + 2 * t;
        b0[j] = *reinterpret_cast<const uint32_t*>(col);
        b1[j] = *reinterpret_cast<const uint32_t*>(col + 8);
      }
#pragma unroll
      for (int i = 0; i < kSlices; ++i) {
        const uint4 a = __ldg(Af + ((size_t(i) * Mt + mt) * Kt + kt) * 32 + lane);
#pragma unroll
        for (int j = 0; j < kSlices - i; ++j) mma_bf16(acc[i + j], a, b0[j], b1[j]);
      }
    }
    // recombine: value = 2^{ea_r + ex_e - 14} sum_s acc[s] 2^{-7 s}
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float h = acc[kGroups - 1][c], l = 0.f;
#pragma unroll
      for (int s = kGroups - 2; s >= 0; --s) {
        const float hs = h * 0.0078125f, ls = l * 0.0078125f;  // exact scaling by 2^-7
        const float sum = acc[s][c] + hs;
        const float bb = sum - acc[s][c];
        const float err = (acc[s][c] - (sum - bb)) + (hs - bb);
        h = sum;
        l = ls + err;
      }
      const int r = mt * 16 + g + ((c & 2) ? 8 : 0);
      const int n = nt * 8 + 2 * t + (c & 1);
      if (r < M && n < ne) {
        const int sc = ea[r] + exs[n] - 14;
        out[(e0 + n) * ldo + r] = f2d_scaled(h, sc) + f2d_scaled(l, sc);
      }
    }
  }
}

// out[e][r] = sum_k A[r][k] X[e][k] for e < nE, r < M (FP64 in and out).
// X rows have Kd entries at stride ldx; out rows stride ldo.
template <int MAXF, int OWARPS>
__global__ void __launch_bounds__(OWARPS * 32) oz_gemm(int64_t nE, int M, int Kd, int Mt, int Kt,
                                                    const uint4* __restrict__ Af, const int* __restrict__ ea,
                                                    const double* __restrict__ X, int64_t ldx,
                                                    double* __restrict__ out, int64_t ldo) {
  extern __shared__ __align__(16) uint16_t osm[];
  const int KP = Kt * 16 + 8;                 // row stride (bf16) of a slice; +8 breaks bank alignment
  uint16_t* Xs = osm;                         // [kSlices][OE][KP]
  int* exs = reinterpret_cast<int*>(osm + size_t(kSlices) * OE * KP);  // [OE]
  constexpr int OTHREADS = OWARPS * 32;
  const int64_t ntiles = (nE + OE - 1) / OE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * OE;
    const int ne = int((nE - e0) < OE ? (nE - e0) : OE);
    __syncthreads();
    // per-element scale exponents
    for (int e = threadIdx.x; e < OE; e += OTHREADS) exs[e] = -1100;
    __syncthreads();
    for (int idx = threadIdx.x; idx < ne * Kd; idx += OTHREADS) {
      const int e = idx / Kd, k = idx - e * Kd;
      atomicMax(&exs[e], exp_bound(__ldg(X + (e0 + e) * ldx + k)));
    }
    __syncthreads();
    // slices, zero-padded in k and e
    for (int idx = threadIdx.x; idx < OE * Kt * 16; idx += OTHREADS) {
      const int e = idx / (Kt * 16), k = idx - e * (Kt * 16);
      uint16_t s[kSlices];
      if (e < ne && k < Kd) {
        slice_dev(__ldg(X + (e0 + e) * ldx + k), exs[e], s);
      } else {
#pragma unroll
        for (int j = 0; j < kSlices; ++j) s[j] = 0;
      }
#pragma unroll
      for (int j = 0; j < kSlices; ++j) Xs[(size_t(j) * OE + e) * KP + k] = s[j];
    }
    __syncthreads();
    oz_mma_tile<MAXF, OWARPS>(Xs, exs, KP, M, Mt, Kt, ne, e0, Af, ea, out, ldo);
  }
}

__device__ __forceinline__ int fnode_rt(int N, int f, int j) {
  auto rs = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

// Y row of an element (the output product's input), columns:
//   wr, ws (Np each) | 1/2 nr sJ [u], 1/2 ns sJ [u] (NFN each) |
//   -sJ ({n.grad u} + tau [u]) (NFN) | lambda J u (Np, Helmholtz only)
// The output product with the pointwise stage fused into its slicing phase:
// warp w builds the Y row of element n (the columns listed above, from C1, u,
// the geometry and the neighbours' C1 and u rows) in registers, takes the
// row's scale exponent as a warp maximum and writes the 8 slices straight to
// shared memory, so Y never touches HBM.
template <int MAXF, int OWARPS>
__global__ void __launch_bounds__(OWARPS * 32) oz_out(int N, int64_t K, int64_t nE, int Kd, int Mt, int Kt,
                                                   const double* __restrict__ gx, const int32_t* __restrict__ conn,
                                                   const double* __restrict__ u, const double* __restrict__ C1,
                                                   double lambda, const uint4* __restrict__ Af,
                                                   const int* __restrict__ ea, double* __restrict__ out) {
  extern __shared__ __align__(16) uint16_t osm[];
  const int KP = Kt * 16 + 8;
  uint16_t* Xs = osm;
  int* exs = reinterpret_cast<int*>(osm + size_t(kSlices) * OE * KP);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  const double cpen = double((N + 1) * (N + 2)) / 2.0;
  const int64_t ntiles = (nE + OE - 1) / OE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * OE;
    const int ne = int((nE - e0) < OE ? (nE - e0) : OE);
    __syncthreads();
    for (int n = warp; n < OE; n += OWARPS) {
      // slots: 0-2 volume node lane (wr, ws, lambda J u), 3-5 node lane + 32, 6-8 face node lane
      double v[9];
      int col[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        v[k] = 0.0;
        col[k] = -1;
      }
      if (n < ne) {
        const int64_t be = e0 + n;
        const int64_t e = be % K;
        const int64_t boff = be - e;
        const double* g = gx + 16 * e;
        const double* c = C1 + be * (2 * Np);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = lane + 32 * h;
          if (i < Np) {
            const double ur = c[i], us = c[Np + i];
            v[3 * h] = g[1] * ur + g[2] * us;
            col[3 * h] = i;
            v[3 * h + 1] = g[2] * ur + g[3] * us;
            col[3 * h + 1] = Np + i;
            if (lambda != 0.0) {
              v[3 * h + 2] = lambda * g[0] * u[be * Np + i];
              col[3 * h + 2] = 2 * Np + 3 * NFN + i;
            }
          }
        }
        if (lane < NFN) {
          const int q = lane, f = q / Nfp, j = q - f * Nfp;
          const double nr = g[4 + 4 * f], ns = g[5 + 4 * f], sJ = g[6 + 4 * f], tau = cpen * g[7 + 4 * f];
          const int k = fnode_rt(N, f, j);
          const double um = u[be * Np + k];
          const double dnm = nr * c[k] + ns * c[Np + k];
          const int code = conn[3 * e + f];
          double jm = 0.0, av = 0.0;
          if (code >= 0) {
            const int64_t nb = code >> 2;
            const int fn = code & 3;
            const int kn = fnode_rt(N, fn, Nfp - 1 - j);
            const double* gn = gx + 16 * nb + 4 + 4 * fn;
            const double* cn = C1 + (boff + nb) * (2 * Np);
            const double up = u[(boff + nb) * Np + kn];
            const double dnp = gn[0] * cn[kn] + gn[1] * cn[Np + kn];
            jm = up - um;
            av = 0.5 * (dnm - dnp);
          } else if (code == -2) {
            jm = -2.0 * um;
            av = dnm;
          }
          const double hs = 0.5 * sJ * jm;
          v[6] = nr * hs;
          col[6] = 2 * Np + q;
          v[7] = ns * hs;
          col[7] = 2 * Np + NFN + q;
          v[8] = -sJ * (av + tau * jm);
          col[8] = 2 * Np + 2 * NFN + q;
        }
      }
      int emax = -1100;
#pragma unroll
      for (int k = 0; k < 9; ++k)
        if (col[k] >= 0) emax = max(emax, exp_bound(v[k]));
      emax = __reduce_max_sync(0xffffffffu, emax);
      if (lane == 0) exs[n] = emax;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        if (col[k] < 0) continue;
        uint16_t sl[kSlices];
        slice_dev(v[k], emax, sl);
#pragma unroll
        for (int jj = 0; jj < kSlices; ++jj) Xs[(size_t(jj) * OE + n) * KP + col[k]] = sl[jj];
      }
      // zero padding: the columns past Kd, or the whole row past the tile's end
      for (int k = (n < ne ? Kd : 0) + lane; k < Kt * 16; k += 32)
#pragma unroll
        for (int jj = 0; jj < kSlices; ++jj) Xs[(size_t(jj) * OE + n) * KP + k] = 0;
    }
    __syncthreads();
    oz_mma_tile<MAXF, OWARPS>(Xs, exs, KP, Np, Mt, Kt, ne, e0, Af, ea, out, Np);
  }
}

// arguments of the fused output product (null: plain product from X)
struct FusedArgs {
  int N;
  int64_t K;
  const double* gx;
  const int32_t* conn;
  const double* u;
  const double* C1;
  double lambda;
};

struct OzOps {
  int Mt1 = 0, Kt1 = 0, Mt2 = 0, Kt2p = 0, Kt2h = 0;
  uint4 *A1 = nullptr, *A2p = nullptr, *A2h = nullptr;
  int *ea1 = nullptr, *ea2p = nullptr, *ea2h = nullptr;
};

cudaError_t build_oz_ops(const RefElem& R, OzOps& o) {
  const int N = R.N, Np = R.Np, Nfp = R.Nfp, NFN = 3 * Nfp;
  // [Dr; Ds]: 2Np x Np
  std::vector<double> A1(size_t(2 * Np) * Np);
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < Np; ++m) {
      A1[size_t(i) * Np + m] = R.Dr[size_t(i) * Np + m];
      A1[size_t(Np + i) * Np + m] = R.Ds[size_t(i) * Np + m];
    }
  // OB: Np x (2Np + 3NFN [+ Np])
  const int KPo = 2 * Np + 3 * NFN, KHo = KPo + Np;
  auto build_ob = [&](int Kc) {
    std::vector<double> B(size_t(Np) * Kc, 0.0);
    for (int i = 0; i < Np; ++i) {
      for (int m = 0; m < Np; ++m) {
        B[size_t(i) * Kc + m] = R.Br[size_t(i) * Np + m];
        B[size_t(i) * Kc + Np + m] = R.Bs[size_t(i) * Np + m];
        if (Kc == KHo) B[size_t(i) * Kc + KPo + m] = R.M[size_t(i) * Np + m];
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
    return B;
  };
  std::vector<uint32_t> f1, f2p, f2h;
  std::vector<int> e1, e2p, e2h;
  int Mt2h = 0;
  slice_operator(A1, 2 * Np, Np, o.Mt1, o.Kt1, f1, e1);
  slice_operator(build_ob(KPo), Np, KPo, o.Mt2, o.Kt2p, f2p, e2p);
  slice_operator(build_ob(KHo), Np, KHo, Mt2h, o.Kt2h, f2h, e2h);
  auto up = [](auto& dst, const auto& v) -> cudaError_t {
    cudaError_t e = cudaMalloc(&dst, v.size() * sizeof(v[0]));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
  };
  cudaError_t e;
  if ((e = up(o.A1, f1)) != cudaSuccess) return e;
  if ((e = up(o.A2p, f2p)) != cudaSuccess) return e;
  if ((e = up(o.A2h, f2h)) != cudaSuccess) return e;
  if ((e = up(o.ea1, e1)) != cudaSuccess) return e;
  if ((e = up(o.ea2p, e2p)) != cudaSuccess) return e;
  return up(o.ea2h, e2h);
}

template <int MAXF, int OWARPS>
cudaError_t launch_gemm(int64_t nE, int M, int Kd, int Mt, int Kt, const uint4* Af, const int* ea, const double* X,
                        int64_t ldx, double* out, int64_t ldo, const FusedArgs* fa, cudaStream_t st) {
  constexpr int OTHREADS = OWARPS * 32;
  const size_t smem = size_t(kSlices) * OE * (Kt * 16 + 8) * sizeof(uint16_t) + OE * sizeof(int);
  static size_t configured[64][2] = {};  // per device and variant: the largest dynamic shared memory set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* kern = fa ? reinterpret_cast<const void*>(oz_out<MAXF, OWARPS>)
                        : reinterpret_cast<const void*>(oz_gemm<MAXF, OWARPS>);
  if (configured[dev & 63][fa ? 1 : 0] < smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    configured[dev & 63][fa ? 1 : 0] = smem;
  }
  int sms = 0, per = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, OTHREADS, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (nE + OE - 1) / OE;
  int64_t grid = int64_t(sms) * (per > 0 ? per : 1);
  if (grid > tiles) grid = tiles;
  if (fa)
    oz_out<MAXF, OWARPS><<<unsigned(grid), OTHREADS, smem, st>>>(fa->N, fa->K, nE, Kd, Mt, Kt, fa->gx, fa->conn, fa->u,
                                                                fa->C1, fa->lambda, Af, ea, out);
  else
    oz_gemm<MAXF, OWARPS><<<unsigned(grid), OTHREADS, smem, st>>>(nE, M, Kd, Mt, Kt, Af, ea, X, ldx, out, ldo);
  note_launch();
  return cudaGetLastError();
}

// warps per CTA chosen so every warp gets the same number of fragments
cudaError_t gemm(int Mt, int64_t nE, int M, int Kd, int Kt, const uint4* Af, const int* ea, const double* X,
                 int64_t ldx, double* out, int64_t ldo, const FusedArgs* fa, cudaStream_t st) {
  const int nfrag = Mt * ONT;
#define OZ_L(F, W) return launch_gemm<F, W>(nE, M, Kd, Mt, Kt, Af, ea, X, ldx, out, ldo, fa, st)
  if (nfrag % 8 == 0) {
    const int f = nfrag / 8;
    if (f == 1) OZ_L(1, 8);
    if (f == 2) OZ_L(2, 8);
    if (f == 3) OZ_L(3, 8);
  }
  if (nfrag % 6 == 0 && nfrag / 6 <= 3) {
    const int f = nfrag / 6;
    if (f == 1) OZ_L(1, 6);
    if (f == 2) OZ_L(2, 6);
    OZ_L(3, 6);
  }
  if (nfrag <= 4) OZ_L(1, 4);
  const int maxf = (nfrag + 7) / 8;
  if (maxf <= 2) OZ_L(2, 8);
  if (maxf <= 3) OZ_L(3, 8);
  OZ_L(4, 8);
#undef OZ_L
}


}  // namespace

// Per-degree operator slices (device, built once per process and device).
static OzOps g_oz[64][kMaxN + 1];

cudaError_t launch_apply_oz64(dg_mesh* m, int degree, int B, double lambda, const double* u, double* Au,
                              cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  OzOps& o = g_oz[dev & 63][degree];
  if (!o.A1) {
    if (m->ref[degree].N == 0) m->ref[degree] = build_reference(degree);
    e = build_oz_ops(m->ref[degree], o);
    if (e != cudaSuccess) return e;
  }
  const int N = degree, Np = (N + 1) * (N + 2) / 2, NFN = 3 * (N + 1);
  const bool helm = lambda != 0.0;
  const int KY = 2 * Np + 3 * NFN + (helm ? Np : 0);
  const int64_t nE = int64_t(B) * m->K;
  const size_t need = size_t(nE) * (2 * Np);  // doubles: C1 (Y is built in shared memory)
  if (m->oz_cap < need) {
    cudaFree(m->oz_scratch);
    m->oz_scratch = nullptr;
    m->oz_cap = 0;
    e = cudaMalloc(&m->oz_scratch, need * sizeof(double));
    if (e != cudaSuccess) return e;
    m->oz_cap = need;
    ++m->scratch_gen;
  }
  double* C1 = m->oz_scratch;
  e = gemm(o.Mt1, nE, 2 * Np, Np, o.Kt1, o.A1, o.ea1, u, Np, C1, 2 * Np, nullptr, st);
  if (e != cudaSuccess) return e;
  const FusedArgs fa{N, m->K, m->geox, m->conn, u, C1, lambda};
  if (helm) return gemm(o.Mt2, nE, Np, KY, o.Kt2h, o.A2h, o.ea2h, nullptr, 0, Au, Np, &fa, st);
  return gemm(o.Mt2, nE, Np, KY, o.Kt2p, o.A2p, o.ea2p, nullptr, 0, Au, Np, &fa, st);
}

}  // namespace dgx
