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
//    exponent i + j: integer sums below 2^24 for K <= 256 and up to 4 products,
//    exact); the accumulators are recombined by Horner's rule in float-float
//    and rebuilt as doubles from the exponent bits. Data slices are written by
//    the threads into a double-buffered shared-memory chunk (32 columns) while
//    the previous chunk's products run; operator blocks (48 rows x 32 columns,
//    8 slices) arrive by bulk copy.
//  * the gradient product C1 = [Dr; Ds] u (rows interleaved, so one thread
//    holds ur and us of a node) with an epilogue that forms the volume columns
//    of Y (wr, ws), the Helmholtz columns and every element's face data
//    (u, n.grad u at its face nodes) in float-float on the FP32 pipe;
//  * tc64_face_fill: the face columns of Y (jumps and averages against the
//    neighbour's face data, penalty of Eq. PenaltyParameter), float-float,
//    one thread per face-node entry;
//  * the output product Au = OB Y, a plain tc64_gemm launch.
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
// Longest sum: a slice product is below 127^2 in magnitude, and an accumulator
// group with up to 4 products over 256 terms stays below 4 * 256 * 127^2 <
// 2^24, an integer FP32 represents exactly; groups with more products carry
// weights below 2^-28 of the leading one (the fifth group stays exact up to
// 208 terms: 5 * 208 * 127^2 < 2^24).
constexpr int kMaxDepth = 256;
// The output product at depths above this runs per column block (volume,
// face, Helmholtz), each block with its own row exponent, accumulated into Au.
constexpr int kSplitDepth = 208;
constexpr int kABytes = kSl * kT * kKC * 2;  // one data chunk, 8 slices: 64 KB
constexpr int kBBytes = kSl * kNC * kKC * 2; // one operator block, 8 slices: 24 KB
constexpr int kASlice = kT * kKC * 2, kBSlice = kNC * kKC * 2;
constexpr int kNodeTab = 72;  // entries of the gradient product's node-to-face table (Np <= 66)
// the tail: 10 mbarriers, slot, 2 flags, the node-to-face table, the tile's face normals
// (MODE 1: n.grad r and n.grad s of the three faces as float-float, [3 faces][4][kT])
constexpr int kSmem = 2 * kABytes + 2 * kBBytes + 4 * kT * 4 + 12 * 8 + kNodeTab * 4 + 12 * kT * 4;

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

// Arguments of the gradient product's epilogue (MODE 1): the rows of A are
// [Dr; Ds] interleaved (column 2n = ur at node n, 2n + 1 = us), and instead of
// C1 the epilogue writes the volume columns of Y (wr, ws), the Helmholtz
// columns lambda J u, and every element's face data FN = (u, n.grad u) at its
// face nodes (outward normal of the element itself).
// Y and the face data are column-major with leading dimension ldc (a multiple
// of 32 rows), so a warp's 32 rows write 256 contiguous bytes per column.
struct GradOut {
  int N;
  int64_t K;
  const double* gx;  // derived geometry, 16 words per element
  double* Y;         // [columns][ldc]
  int64_t ldc;
  int helm;
  double lambda;
  double *FNu, *FNd;  // [3 (N+1)][ldc]: u and n.grad u at the element's face nodes
  int* exy;     // [rows]: largest exponent of the row's Y values (for the output product)
  int* exf;     // [rows] or null: set to "none" here when the face columns keep their own exponent
  int64_t row0;  // global index of the launch's first row (Y, FNu, FNd, exy, exf start there)
};

// out[r][c] = sum_k A[c][k] X[r][k] for r < rows, c < M, k < Kd (A sliced in
// blocks of kNC rows x kKC columns: block (nc, kc) at (nc KCH + kc) kBBytes).
//
// Warp-specialised pipeline over a stream of data chunks (tile, output pass
// nc, column chunk kc), chunk g using shared-memory buffer g & 1:
//  * warps 0-15 (four threads per row of the 128-row tile) find each row's
//    scale exponent, slice chunk g into buffer g & 1 once the products of
//    chunk g - 2 have released it (mbarrier `empty`), signal `full`, and after
//    a pass's last chunk wait for its accumulators (`acc_full`), drain them
//    (Horner's rule, epilogue) and release them (`acc_empty`);
//  * warp 16 loads operator block g by bulk copy, waits for `full`, issues the
//    36 slice products per 16 columns from one lane and commits to `empty`
//    (and to `acc_full` after a pass's last chunk); before a pass's first
//    chunk it waits until the previous pass has been drained.
// No CTA-wide barrier in the steady state; every wait is bounded in time.
constexpr int kSlicers = 512;  // threads of warps 0-15
template <int MODE>
__global__ void __launch_bounds__(kSlicers + 32, 1) tc64_gemm(int64_t rows, int M, int Kd, int NCH, int KCH,
                                                              const double* __restrict__ X, int64_t ldx, int vec2,
                                                              int xcol,
                                                              const int* __restrict__ ex_given,
                                                              const uint8_t* __restrict__ Bops,
                                                              const int* __restrict__ ea, double* __restrict__ out,
                                                              int64_t ldo, int accum, GradOut go) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA = sm;                        // [2][8 slices][128 rows][32] canonical
  uint8_t* sB = sm + 2 * kABytes;          // [2][8 slices][48 rows][32] canonical
  int* pmax = reinterpret_cast<int*>(sB + 2 * kBBytes);  // [4][kT]
  // full[2], empty[2], bfull[2], acc_full, acc_empty, bempty[2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(pmax + 4 * kT);
  uint64_t *full = bars, *empty = bars + 2, *bfull = bars + 4, *acc_full = bars + 6, *acc_empty = bars + 7,
           *bempty = bars + 8;
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 10);
  int* abort_flag = reinterpret_cast<int*>(slot + 1);
  int* tile_abort = abort_flag + 1;  // the slicers' common copy of abort_flag at a tile's start
  // MODE 1: per node n the face nodes it is, packed (fa + 1) | ja << 4 | (fb + 1) << 8 | jb << 12
  // (face f, position j; a corner is on two faces; 0 in the face field: none)
  int* nodetab = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(bars) + 12 * 8);
  float* snrm = reinterpret_cast<float*>(nodetab + kNodeTab);  // [f][nr.h, nr.l, ns.h, ns.l][kT]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (rows + kT - 1) / kT;
  // with at most two data chunks per row, both stay in the two buffers for all
  // output passes of a tile: sliced once per tile instead of once per pass
  const bool resident = KCH <= 2 && NCH > 1;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(full + i, kSlicers / 32);  // one arrival per slicing warp
      tc::mbar_init(empty + i, 1);             // the products' commit
      tc::mbar_init(bfull + i, 1);             // the bulk copy
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, kSlicers / 32);
    for (int i = 0; i < 2; ++i) tc::mbar_init(bempty + i, 1);  // an operator stage's products completed
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(slot, 512);
  if (MODE == 1 && tid < (go.N + 1) * (go.N + 2) / 2 && tid < kNodeTab) {
    const int N = go.N, n = tid;
    int rrow = 0;  // n's row of constant s
    while (n >= (rrow + 1) * (N + 1) - (rrow + 1) * rrow / 2) ++rrow;
    const int rs0 = rrow * (N + 1) - rrow * (rrow - 1) / 2, len = N + 1 - rrow;
    int fa = -1, ja = 0, fb = -1, jb = 0;
    if (rrow == 0) fa = 0, ja = n;  // face 0, j = n
    if (n == rs0 + len - 1) {       // face 1, j = row
      if (fa < 0) fa = 1, ja = rrow;
      else fb = 1, jb = rrow;
    }
    if (n == rs0 && fb < 0) {  // face 2, j = N - row
      if (fa < 0) fa = 2, ja = N - rrow;
      else fb = 2, jb = N - rrow;
    }
    nodetab[n] = (fa + 1) | (ja << 4) | ((fb + 1) << 8) | (jb << 12);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = *slot;
  constexpr uint32_t idesc = tc::idesc_f16(128, kNC, true);

  if (warp == kSlicers / 32) {
    // ================= products
    uint32_t g = 0, pass = 0, it = 0;
    const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(sA), 128, (kKC / 8) * 128);
    const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sB), 128, (kKC / 8) * 128);
    for (int64_t tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++it) {
      for (int nc = 0; nc < NCH; ++nc, ++pass) {
        // the accumulators are free once the previous pass has been drained
        if (pass > 0 && !tc::mbar_wait(acc_empty, (pass - 1) & 1u)) *abort_flag = 1;
        tc::fence_after();
        for (int kc = 0; kc < KCH; ++kc, ++g) {
          const uint32_t bs = g & 1u;                 // operator stage
          const uint32_t bd = resident ? kc : bs;     // data buffer
          // the operator stage is free once chunk g - 2's products completed
          if (g >= 2 && !tc::mbar_wait(bempty + bs, ((g - 2) >> 1) & 1u)) *abort_flag = 1;
          if (lane == 0) {
            tc::mbar_expect_tx(bfull + bs, kBBytes);
            tc::bulk_g2s(sB + bs * kBBytes, Bops + size_t(nc * KCH + kc) * kBBytes, kBBytes, bfull + bs);
          }
          __syncwarp();
          // the data chunk: sliced once per chunk, or (resident) once per tile for all passes
          if (!resident && !tc::mbar_wait(full + bd, (g >> 1) & 1u)) *abort_flag = 1;
          if (resident && nc == 0 && !tc::mbar_wait(full + bd, it & 1u)) *abort_flag = 1;
          if (!tc::mbar_wait(bfull + bs, (g >> 1) & 1u)) *abort_flag = 1;
          tc::fence_after();
          if (lane == 0) {
            const uint64_t ab = adesc0 + ((bd * kABytes) >> 4), bb = bdesc0 + ((bs * kBBytes) >> 4);
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
            tc::mma_commit(bempty + bs);
            if (!resident || nc == NCH - 1) tc::mma_commit(empty + bd);  // the data buffer is free
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
    uint32_t g = 0, pass = 0, it = 0;
    auto load8 = [&](const double* xr, bool live, int k0, double (&v)[8]) {
      if (xcol) {  // column-major X: element (row, k) at xr[k ldx], xr = X + row
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (live && k0 + t < Kd) ? __ldg(xr + int64_t(k0 + t) * ldx) : 0.0;
      } else if (live && vec2 && k0 + 8 <= Kd) {
        const double2* p2 = reinterpret_cast<const double2*>(xr + k0);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const double2 w = __ldg(p2 + t);
          v[2 * t] = w.x;
          v[2 * t + 1] = w.y;
        }
      } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (live && k0 + t < Kd) ? __ldg(xr + k0 + t) : 0.0;
      }
    };
    // output product (row exponents given): the last chunk of a tile requests the
    // next tile's first chunk and exponent (vn, En), so that their latency overlaps
    // the drain
    bool have_next = false;
    int En = 0;
    double vn[8];  // the next chunk's values (loaded one chunk ahead)
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      // every slicer takes the same decision to stop (they meet at named barriers below)
      asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
      if (tid == 0) *reinterpret_cast<volatile int*>(tile_abort) = *reinterpret_cast<volatile int*>(abort_flag);
      if (MODE == 1 && q < 3) {  // face q's normal metric of this row, once per tile (read by the drains)
        const int64_t rw = tile * kT + e;
        const double* gq = go.gx + 16 * (((rw < rows ? rw : 0) + go.row0) % go.K) + 4 + 4 * q;
        const ff nr = d2ff(__ldg(gq), 0), ns = d2ff(__ldg(gq + 1), 0);
        snrm[(q * 4 + 0) * kT + e] = nr.h;
        snrm[(q * 4 + 1) * kT + e] = nr.l;
        snrm[(q * 4 + 2) * kT + e] = ns.h;
        snrm[(q * 4 + 3) * kT + e] = ns.l;
      }
      asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
      if (*reinterpret_cast<volatile int*>(tile_abort)) break;
      const int64_t row = tile * kT + e;
      const bool live = row < rows;
      const double* xr = xcol ? X + (live ? row : 0) : X + (live ? row : 0) * ldx;
      // scale exponent of the row: a bound |X[row][k]| < 2^E, given by the producer
      // of X or found here
      int E;
      if (ex_given) {
        E = have_next ? En : (live ? __ldg(ex_given + row) : 0);
        if (E == -1100) E = 0;
      } else {
        int em = -1100;
        if (live) {
          double v[2][8];
          for (int kc = 0; kc < KCH; kc += 2) {
            load8(xr, live, kc * kKC + 8 * q, v[0]);
            load8(xr, live && kc + 1 < KCH, (kc + 1) * kKC + 8 * q, v[1]);
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
      if (!have_next) load8(xr, live, 8 * q, vn);
      have_next = false;
      int ymax = -1100;  // MODE 1: largest exponent of the Y columns this thread writes
      float gh[6];  // MODE 1: Grr, Grs, Gss as float-float
      const double* gg = nullptr;  // MODE 1: the row's element geometry
      if (MODE == 1) {
        gg = go.gx + 16 * (((live ? row : 0) + go.row0) % go.K);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const ff gf = d2ff(__ldg(gg + 1 + t), 0);
          gh[2 * t] = gf.h;
          gh[2 * t + 1] = gf.l;
        }
      }
      for (int nc = 0; nc < NCH; ++nc, ++pass) {
        for (int kc = 0; kc < KCH; ++kc, ++g) {
          if (resident && nc > 0) continue;  // the tile's chunks are still in the buffers
          const uint32_t b = resident ? uint32_t(kc) : (g & 1u);
          double v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) v[t] = vn[t];
          {  // request the next chunk of this row (the next pass starts again at chunk 0)
            const int kn = kc + 1 < KCH ? kc + 1 : 0;
            if (kc + 1 < KCH || (nc + 1 < NCH && !resident)) {
              load8(xr, live, kn * kKC + 8 * q, vn);
            } else if (MODE == 0 && ex_given && nc + 1 == NCH && tile + gridDim.x < ntiles) {
              const int64_t nrow = row + int64_t(gridDim.x) * kT;
              const bool nlive = nrow < rows;
              load8(xcol ? X + (nlive ? nrow : 0) : X + (nlive ? nrow : 0) * ldx, nlive, 8 * q, vn);
              En = nlive ? __ldg(ex_given + nrow) : 0;
              have_next = true;
            }
          }
          // each value's 56-bit fixed-point magnitude as two 28-bit halves, and its sign
          // as the pair (s, c) with fma(2^23 + x, s, c) = +-x exactly for 0 <= x < 2^23
          uint32_t hi[8], lo[8];
          float sm[8], sc[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            uint32_t sgn;
            const uint64_t I = fixed56(v[t], E, sgn);
            hi[t] = uint32_t(I >> 28);
            lo[t] = uint32_t(I) & 0xFFFFFFFu;
            sm[t] = sgn ? -1.0f : 1.0f;
            sc[t] = sgn ? 8388608.0f : -8388608.0f;
          }
          // buffer b is free once the products that read it completed: chunk g - 2's, or
          // (resident) the previous tile's last pass
          if (!resident && g >= 2 && !tc::mbar_wait(empty + b, ((g - 2) >> 1) & 1u)) *abort_flag = 1;
          if (resident && it >= 1 && !tc::mbar_wait(empty + b, (it - 1) & 1u)) *abort_flag = 1;
          uint8_t* dst = sA + b * kABytes + (e >> 3) * 512 + q * 128 + (e & 7) * 16;
#pragma unroll
          for (int j = 0; j < kSl; ++j) {
            // slice j: 7 bits of the magnitude below bit 56 - 7j, as a signed float,
            // whose upper 16 bits are its BF16 pattern (at most 8 significant bits)
            uint32_t fb[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const uint32_t x = ((j < 4 ? hi[t] : lo[t]) >> (21 - 7 * (j & 3))) & 127u;
              fb[t] = __float_as_uint(__fmaf_rn(__uint_as_float(0x4B000000u | x), sm[t], sc[t]));
            }
            uint4 w;  // value 2i in the low half of word i, value 2i + 1 in the high half
            w.x = __byte_perm(fb[0], fb[1], 0x7632);
            w.y = __byte_perm(fb[2], fb[3], 0x7632);
            w.z = __byte_perm(fb[4], fb[5], 0x7632);
            w.w = __byte_perm(fb[6], fb[7], 0x7632);
            *reinterpret_cast<uint4*>(dst + j * kASlice) = w;
          }
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
          const int c0 = 12 * q + 4 * p;
          uint32_t acc[kSl][4];
#pragma unroll
          for (int s = 0; s < kSl; ++s) {
            uint32_t vv[4];
            tc::tmem_ld4(tb + lanebase + s * kNC + c0, vv);
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
          if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int col = nc * kNC + c0 + c;
              if (live && col < M) {
                // value = 2^{ea + E - 14} sum_s acc_s 2^{-7 s}
                const ff hl = horner8(acc, c);
                const double v = ff_to_double(hl.h, hl.l, __ldg(ea + col) + E - 14);
                if (accum) out[row * ldo + col] += v;  // (the Helmholtz or face block of a split product)
                else out[row * ldo + col] = v;
              }
            }
          } else {
            // nodes n = col / 2: (ur, us) in columns (2n, 2n + 1)
            const int N = go.N, Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
              const int n = (nc * kNC + c0 + c) >> 1;
              if (live && n < Np) {
                const int er = __ldg(ea + 2 * n), es = __ldg(ea + 2 * n + 1);
                const int ec = max(er, es);
                ff ur = horner8(acc, c), us = horner8(acc, c + 1);
                ur = ff_pow2(ur, __uint_as_float(uint32_t(127 + er - ec) << 23));
                us = ff_pow2(us, __uint_as_float(uint32_t(127 + es - ec) << 23));
                const int S = ec + E - 14;  // ur, us, wr, ws, n.grad u all carry 2^S
                const ff grr{gh[0], gh[1]}, grs{gh[2], gh[3]}, gss{gh[4], gh[5]};
                const ff wr = ff_add(ff_mul(grr, ur), ff_mul(grs, us));
                const ff ws = ff_add(ff_mul(grs, ur), ff_mul(gss, us));
                double* yr = go.Y + row;  // column c of this row at yr[c ldc]
                const int64_t ldc = go.ldc;
                const double dwr = ff_to_double(wr.h, wr.l, S), dws = ff_to_double(ws.h, ws.l, S);
                yr[n * ldc] = dwr;
                yr[(Np + n) * ldc] = dws;
                ymax = max(ymax, max(exp_bound64(dwr), exp_bound64(dws)));
                const double un = __ldg(X + row * ldx + n);
                if (go.helm) {
                  const int eu = exp_bound64(un);
                  const ff lj = ff_mul(d2ff(go.lambda, 0), d2ff(__ldg(gg), 0));
                  const ff vv = ff_mul(lj, d2ff(un, eu));
                  const double dv = ff_to_double(vv.h, vv.l, eu);
                  yr[(2 * Np + 3 * NFN + n) * ldc] = dv;
                  ymax = max(ymax, exp_bound64(dv));
                }
                // face data at the face nodes this node is (a corner belongs to two faces)
                const int nt = nodetab[n];
                const int fa = (nt & 15) - 1, ja = (nt >> 4) & 15, fb = ((nt >> 8) & 15) - 1, jb = (nt >> 12) & 15;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                  const int f = t == 0 ? fa : fb, j = t == 0 ? ja : jb;
                  if (f >= 0) {
                    const ff nr{snrm[(f * 4 + 0) * kT + e], snrm[(f * 4 + 1) * kT + e]};
                    const ff ns{snrm[(f * 4 + 2) * kT + e], snrm[(f * 4 + 3) * kT + e]};
                    const ff dn = ff_add(ff_mul(nr, ur), ff_mul(ns, us));
                    const int64_t fi = int64_t(f * Nfp + j) * ldc + row;
                    go.FNu[fi] = un;
                    go.FNd[fi] = ff_to_double(dn.h, dn.l, S);
                  }
                }
              }
            }
          }
        }
      }
      if (MODE == 1) {  // the row's largest Y exponent so far (the face columns add theirs)
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        pmax[q * kT + e] = ymax;
        asm volatile("bar.sync 1, %0;\n" ::"r"(kSlicers) : "memory");
        if (q == 0 && live)
          go.exy[row] = max(max(pmax[e], pmax[kT + e]), max(pmax[2 * kT + e], pmax[3 * kT + e]));
        if (q == 0 && live && go.exf) go.exf[row] = -1100;  // raised by the face fill
      }
    }
  }
  if (*abort_flag && tid == 0) atomicExch(&g_tc64_err, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ------------------------------------------------------------------ face columns of Y
// One thread per element (consecutive threads take consecutive rows, so every
// access to the column-major face data and Y is coalesced except the
// neighbour's): for each face f and face node j, entry i = f (N+1) + j, from
// the element's face data and its neighbour's across face f (FNu, FNd, written
// by the gradient product), Y[2Np + i] = 1/2 nr sJ [u], Y[2Np + NFN + i] =
// 1/2 ns sJ [u], Y[2Np + 2 NFN + i] = -sJ ({n.grad u} + tau [u]), in
// float-float scaled by the entry's largest input; the row's largest exponent
// (exy: raised from the value the gradient product wrote for the volume
// columns) for the output product's slicing.
__global__ void __launch_bounds__(256) tc64_face_fill(int N, int64_t K, int64_t r0, int64_t nE,
                                                      const double* __restrict__ gx,
                                                      const int32_t* __restrict__ conn,
                                                      const double* __restrict__ FNu,
                                                      const double* __restrict__ FNd, double* __restrict__ Y,
                                                      int64_t ldc, int* __restrict__ exy) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  const ff cpen{float((N + 1) * (N + 2)) * 0.5f, 0.f};
  for (int64_t be = r0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; be < nE;
       be += int64_t(gridDim.x) * blockDim.x) {  // rows r0 .. nE - 1
    const int64_t el = be < K ? be : be % K, boff = be - el;  // first right-hand side: no division
    int ym = -1100;
    for (int f = 0; f < 3; ++f) {
      const double* g = gx + 16 * el + 4 + 4 * f;
      const ff nr = d2ff(__ldg(g), 0), ns = d2ff(__ldg(g + 1), 0), sJ = d2ff(__ldg(g + 2), 0);
      const ff tau = ff_mul(cpen, d2ff(__ldg(g + 3), 0));
      const int code = __ldg(conn + 3 * el + f);
      const int64_t nb = code >= 0 ? boff + (code >> 2) : 0;
      const int fn = code >= 0 ? (code & 3) : 0;
      for (int j = 0; j < Nfp; ++j) {
        const int i = f * Nfp + j;
        const double ou = __ldg(FNu + int64_t(i) * ldc + be), od = __ldg(FNd + int64_t(i) * ldc + be);
        double pu = 0.0, pd = 0.0;
        if (code >= 0) {
          const int64_t pi = int64_t(fn * Nfp + (Nfp - 1 - j)) * ldc + nb;
          pu = __ldg(FNu + pi);
          pd = __ldg(FNd + pi);
        }
        const int R = max(max(exp_bound64(ou), exp_bound64(od)), max(exp_bound64(pu), exp_bound64(pd)));
        const int Rs = R == -1100 ? 0 : R;
        const ff um = d2ff(ou, Rs), dnm = d2ff(od, Rs);
        ff jm{0.f, 0.f}, av{0.f, 0.f};
        if (code >= 0) {
          jm = ff_sub(d2ff(pu, Rs), um);
          av = ff_pow2(ff_sub(dnm, d2ff(pd, Rs)), 0.5f);
        } else if (code == -2) {  // Dirichlet
          jm = ff_pow2(um, -2.0f);
          av = dnm;
        }
        const ff hs = ff_pow2(ff_mul(sJ, jm), 0.5f);
        const ff a = ff_mul(nr, hs), b = ff_mul(ns, hs);
        const ff fl = ff_neg(ff_mul(sJ, ff_add(av, ff_mul(tau, jm))));
        double* y = Y + int64_t(2 * Np + i) * ldc + be;
        const double da = ff_to_double(a.h, a.l, Rs), db = ff_to_double(b.h, b.l, Rs), dc = ff_to_double(fl.h, fl.l, Rs);
        y[0] = da;
        y[int64_t(NFN) * ldc] = db;
        y[int64_t(2 * NFN) * ldc] = dc;
        ym = max(ym, max(exp_bound64(da), max(exp_bound64(db), exp_bound64(dc))));
      }
    }
    if (ym > -1100) exy[be] = max(exy[be], ym);  // with the volume columns' bound, set before
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
  if (K > kMaxDepth) return cudaErrorInvalidValue;  // longer sums would leave the FP32 group sums inexact
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
                        const int* ex_given, const GradOut& go, cudaStream_t st, int accum = 0, int xcol = 0) {
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
      int sms = 0;
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      grid[dev & 63] = sms;  // one CTA per SM (all of tensor memory, most of shared memory)
    }
  }
  const int vec2 = (ldx % 2 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) ? 1 : 0;
  const int64_t tiles = (rows + kT - 1) / kT;
  const unsigned g = unsigned(std::min<int64_t>(tiles, grid[dev & 63]));
  tc64_gemm<MODE><<<g, kSlicers + 32, kSmem, st>>>(rows, op.M, op.K, op.NCH, op.KCH, X, ldx, vec2, xcol, ex_given,
                                                   op.blocks, op.ea, out, ldo, accum, go);
  note_launch();
  return cudaGetLastError();
}
}  // namespace

cudaError_t tc64_gemm_launch(const Tc64Op& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                             cudaStream_t st, int accum, const int* ex) {
  return gemm_launch<0>(op, rows, X, ldx, out, ldo, ex, GradOut{}, st, accum);
}

namespace {
struct Tc64Apply {
  Tc64Op grad;       // [Dr; Ds] with rows interleaved (Dr row n, Ds row n, ...)
  Tc64Op out, outh;  // OB, [OB | M] (when its depth stays within kMaxDepth)
  Tc64Op mh;         // M alone, otherwise: the Helmholtz term as a second, accumulating product
  Tc64Op outv, outf; // [Br Bs] and the face blocks of OB, when OB is deeper than kSplitDepth
};
Tc64Apply g_t64[64][kMaxN + 1];  // [device][degree]

cudaError_t build_t64(const RefElem& R, Tc64Apply& o) {
  const int N = R.N, Np = R.Np, Nfp = R.Nfp, NFN = 3 * Nfp;
  std::vector<double> A1(size_t(2 * Np) * Np);
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m) {
      A1[size_t(2 * n) * Np + m] = R.Dr[size_t(n) * Np + m];
      A1[size_t(2 * n + 1) * Np + m] = R.Ds[size_t(n) * Np + m];
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
  if (KY > kSplitDepth) {  // column blocks [Br Bs], [face blocks], M, each from its own Y columns
    std::vector<double> Bv(size_t(Np) * 2 * Np), Bf(size_t(Np) * 3 * NFN), Mm(R.M.begin(), R.M.begin() + size_t(Np) * Np);
    for (int i = 0; i < Np; ++i) {
      for (int k = 0; k < 2 * Np; ++k) Bv[size_t(i) * 2 * Np + k] = B[size_t(i) * KY + k];
      for (int k = 0; k < 3 * NFN; ++k) Bf[size_t(i) * 3 * NFN + k] = B[size_t(i) * KY + 2 * Np + k];
    }
    if (e == cudaSuccess) e = tc64_op_create(Bv, Np, 2 * Np, &o.outv);
    if (e == cudaSuccess) e = tc64_op_create(Bf, Np, 3 * NFN, &o.outf);
    if (e == cudaSuccess) e = tc64_op_create(Mm, Np, Np, &o.mh);
    return e;
  }
  if (e == cudaSuccess) e = tc64_op_create(B, Np, KY, &o.out);
  if (e == cudaSuccess) {
    if (KH <= kMaxDepth) {
      e = tc64_op_create(BH, Np, KH, &o.outh);
    } else {
      std::vector<double> Mm(R.M.begin(), R.M.begin() + size_t(Np) * Np);
      e = tc64_op_create(Mm, Np, Np, &o.mh);
    }
  }
  return e;
}
}  // namespace

bool tc64_supported(int degree) {
  const int Np = (degree + 1) * (degree + 2) / 2, NFN = 3 * (degree + 1);
  return 2 * Np + 3 * NFN <= kMaxDepth && Np <= kMaxDepth;
}

namespace {
// The degree's sliced operators on the current device, built on first use
// when `build` is set (null if not built, or if building failed: *err says why).
const Tc64Apply* t64_ops(dg_mesh* m, int degree, bool build, cudaError_t* err) {
  *err = cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *err = e;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(table_mutex());
  Tc64Apply& o = g_t64[dev & 63][degree];
  if (!o.grad.blocks) {
    if (!build) return nullptr;
    const RefElem R = m->ref[degree].N ? m->ref[degree] : build_reference(degree);
    Tc64Apply built;
    e = build_t64(R, built);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    o = built;
  }
  return &o;
}
int t64_cols(int degree, bool helm) {  // Y's columns
  const int Np = (degree + 1) * (degree + 2) / 2, NFN = 3 * (degree + 1);
  return 2 * Np + 3 * NFN + (helm ? Np : 0);
}
int64_t t64_ldc(int64_t nE) { return (nE + 31) & ~int64_t(31); }
}  // namespace

size_t tc64_scratch_words(int degree, int64_t nE, bool helm) {
  const int NFN = 3 * (degree + 1);
  return size_t(t64_ldc(nE)) * (t64_cols(degree, helm) + 2 * NFN) + 2 * (size_t(nE + 1) / 2) + 2;
}

cudaError_t ensure_tc64_ops(dg_mesh* m, int degree) {
  if (!tc64_supported(degree)) return cudaSuccess;
  cudaError_t e;
  t64_ops(m, degree, true, &e);
  return e;
}

bool tc64_ops_ready(int degree) {
  if (!tc64_supported(degree)) return false;
  cudaError_t e;
  return t64_ops(nullptr, degree, false, &e) != nullptr;
}

namespace {
// The largest forward distance from an element to one of its neighbours (rows),
// from the host copy of the connectivity; kept with the mesh.
int64_t t64_reach(dg_mesh* m) {
  if (m->nb_reach < 0) {
    int64_t r = 0;
    for (int64_t e = 0; e < m->K; ++e)
      for (int f = 0; f < 3; ++f) {
        const int32_t code = m->conn_h[size_t(3 * e + f)];
        if (code >= 0) r = std::max<int64_t>(r, int64_t(code >> 2) - e);
      }
    m->nb_reach = r;
  }
  return m->nb_reach;
}
}  // namespace

cudaError_t launch_apply_tc64(dg_mesh* m, int degree, int B, double lambda, const double* u, double* Au,
                              cudaStream_t st, double* scratch, const ApplyChunks* chunks) {
  if (B < 1) return cudaSuccess;
  if (!tc64_supported(degree)) return cudaErrorInvalidValue;
  cudaError_t e;
  const Tc64Apply* ops = t64_ops(m, degree, scratch == nullptr, &e);
  if (!ops) return e != cudaSuccess ? e : cudaErrorNotReady;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int N = degree, Np = (N + 1) * (N + 2) / 2, NFN = 3 * (N + 1);
  const bool helm = lambda != 0.0;
  const int64_t nE = int64_t(B) * m->K;
  const int64_t ldc = t64_ldc(nE);
  // scratch: Y [columns][ldc], the face data FNu, FNd [NFN][ldc] (u, n.grad u), FP64,
  // and the rows' largest Y exponents; every word read is written first by this call
  const size_t words = tc64_scratch_words(N, nE, helm);
  if (!scratch && m->t64_cap < words) {
    cudaFree(m->t64_scratch);
    m->t64_scratch = nullptr;
    m->t64_cap = 0;
    e = cudaMalloc(&m->t64_scratch, words * sizeof(double));
    if (e == cudaSuccess) e = poison(m->t64_scratch, words * sizeof(double), POISON_APPLY);
    if (e != cudaSuccess) return e;
    m->t64_cap = words;
    ++m->scratch_gen;
  }
  double* Y = scratch ? scratch : m->t64_scratch;
  double* FNu = Y + size_t(ldc) * t64_cols(N, helm);
  double* FNd = FNu + size_t(ldc) * NFN;
  int* exy = reinterpret_cast<int*>(FNd + size_t(ldc) * NFN);
  const bool split = ops->outv.blocks != nullptr;
  int* exf = split ? exy + 2 * (size_t(nE + 1) / 2) : nullptr;  // the face columns' own exponents
  const bool chunked = chunks && chunks->n > 0 && chunks->bounds && chunks->bounds[chunks->n] == nE;
  const int nch = chunked ? chunks->n : 1;
  const int64_t whole[2] = {0, nE};
  const int64_t* bnd = chunked ? chunks->bounds : whole;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // a chunk's neighbour phase needs the gradient products of every chunk that
  // holds one of its rows' neighbours: rows up to (last row + reach)
  const int64_t reach = nch > 1 ? t64_reach(m) : nE;
  auto ready_after = [&](int c) {  // the last chunk whose gradient product chunk c's face fill needs
    const int64_t last = std::min<int64_t>(nE - 1, bnd[c + 1] - 1 + reach);
    int j = c;
    while (j + 1 < nch && bnd[j + 1] <= last) ++j;
    return j;
  };
  auto finish = [&](int c) -> cudaError_t {  // face fill and output product of chunk c
    const int64_t r0 = bnd[c], n = bnd[c + 1] - r0;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, int64_t(sms) * 16);  // a thread per element
    tc64_face_fill<<<unsigned(blocks), 256, 0, st>>>(N, m->K, r0, r0 + n, m->geox, m->conn, FNu, FNd, Y, ldc,
                                                     split ? exf : exy);
    note_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    double* out = Au + r0 * Np;
    const double* Yc = Y + r0;
    const int* ey = exy + r0;
    if (split) {  // Au = [Br Bs] Y_v + (face blocks) Y_f (+ M Y_h), the face block with its own exponents
      err = gemm_launch<0>(ops->outv, n, Yc, ldc, out, Np, ey, GradOut{}, st, 0, 1);
      if (err == cudaSuccess)
        err = gemm_launch<0>(ops->outf, n, Yc + 2 * Np * ldc, ldc, out, Np, exf + r0, GradOut{}, st, 1, 1);
      if (err == cudaSuccess && helm)
        err = gemm_launch<0>(ops->mh, n, Yc + (2 * Np + 3 * NFN) * ldc, ldc, out, Np, ey, GradOut{}, st, 1, 1);
    } else if (helm && !ops->outh.blocks) {  // [OB | M] is too deep for exact group sums: OB Y, then += M (lambda J u)
      const int KY = 2 * Np + 3 * NFN;
      err = gemm_launch<0>(ops->out, n, Yc, ldc, out, Np, ey, GradOut{}, st, 0, 1);
      if (err == cudaSuccess) err = gemm_launch<0>(ops->mh, n, Yc + KY * ldc, ldc, out, Np, ey, GradOut{}, st, 1, 1);
    } else {
      err = gemm_launch<0>(helm ? ops->outh : ops->out, n, Yc, ldc, out, Np, ey, GradOut{}, st, 0, 1);
    }
    if (err != cudaSuccess) return err;
    if (chunked && chunks->after) err = chunks->after(chunks->ctx, c, r0, r0 + n);
    return err;
  };
  int done = 0;  // chunks whose face fill and output product are issued
  for (int c = 0; c < nch; ++c) {  // gradient product, element-local
    const int64_t r0 = bnd[c], r1 = bnd[c + 1];
    if (chunked && chunks->before && (e = chunks->before(chunks->ctx, c, r0, r1)) != cudaSuccess) return e;
    GradOut go{N, m->K, m->geox, Y + r0, ldc, helm ? 1 : 0, lambda, FNu + r0, FNd + r0, exy + r0,
               exf ? exf + r0 : nullptr, r0};
    e = gemm_launch<1>(ops->grad, r1 - r0, u + r0 * Np, Np, nullptr, 0, nullptr, go, st);
    if (e != cudaSuccess) return e;
    while (done < nch && ready_after(done) <= c)
      if ((e = finish(done++)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t tc64_error(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc64_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc64_err, &zero, sizeof(int));
  return e;
}

}  // namespace dgx
