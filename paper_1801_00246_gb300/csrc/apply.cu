// Fused matrix-free SIPDG Poisson / screened-Poisson apply on affine triangles.
//
// Computes the weak coefficient vector (A u)_i = a(u, l_i) of the bilinear
// form of Eq. ellipticOp1 (Section 5.2) for every element in one pass:
//
//   (A u)_i = [Br wr + Bs ws]_i                          volume  (grad l_i, grad u)
//           + lambda J [M u]_i                           screening
//           + sum_f sum_j (nr_f Dr[k_fj][i] + ns_f Ds[k_fj][i]) F2_fj
//                                                        1/2 (n.grad l_i, [u])_f
//           + sum_{f,j: k_fj = i} F1_fj                  -(l_i, n.{grad u} + tau [u])_f
//
// with ur = Dr u, us = Ds u, (wr, ws) = J G G^T (ur, us), Br = Dr^T M,
// Bs = Ds^T M, and at the face nodes (face mass Mf, surface Jacobian sJ):
//   F1 = sJ Mf (-{n.grad u} - tau [u]),  F2 = 1/2 sJ Mf [u].
// This is the grouping of Eq. ellipticOp3 with the lift written through the
// face mass (M L^f = E_f Mf), so no lift matrix and no transposed operator
// beyond Dr^T M / Ds^T M is needed.
//
// Unlike the paper's two-kernel scheme (Algorithms 1 and 2: gradient to global
// memory, then the operator), the neighbour's normal derivative at the shared
// face nodes is recomputed from the neighbour's nodal values, which are read
// through L2; HBM sees u once and A u once. Geometry is 4 words per element
// (r_x, s_x, r_y, s_y); J, normals, surface Jacobians and the penalty follow
// from them for affine triangles.
#include "dg_internal.h"

#include <cstdio>
#include <type_traits>

namespace dgx {
namespace {

template <int N>
struct Dim {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int NFN = 3 * (N + 1);
  static constexpr int LD = (Np % 2 == 0) ? Np + 1 : Np;  // odd smem stride: no bank conflicts
  // elements per tile: about 320 nodes of work per tile
  static constexpr int E = (320 / Np) < 2 ? 2 : (320 / Np);
};

constexpr int kThreads = 256;

__host__ __device__ constexpr int row_start(int N, int row) { return row * (N + 1) - row * (row - 1) / 2; }

__device__ __forceinline__ int fnode(int N, int f, int j) {
  return f == 0 ? j : (f == 1 ? row_start(N, j) + (N - j) : row_start(N, N - j));
}

template <typename T>
struct FaceGeo {
  T sJ, nr, ns, tau, ap, bp;
};

// Shared-memory carve-up, in units of T.
template <int N, typename T, bool HELM>
struct Smem {
  using D = Dim<N>;
  static constexpr int Np = D::Np, LD = D::LD, Nfp = D::Nfp, NFN = D::NFN, E = D::E;
  static constexpr int oDr = 0, oDs = oDr + Np * LD, oBr = oDs + Np * LD, oBs = oBr + Np * LD;
  static constexpr int oM = oBs + Np * LD;
  static constexpr int oMf = oM + (HELM ? Np * LD : 0);
  static constexpr int oU = oMf + Nfp * Nfp;
  static constexpr int oUN = oU + E * LD;            // neighbours' nodal values [E][3][LD]
  static constexpr int oUR = oUN + E * 3 * LD;
  static constexpr int oUS = oUR + E * LD;
  static constexpr int oWR = oUS + E * LD;
  static constexpr int oWS = oWR + E * LD;
  static constexpr int oUP = oWS + E * LD;            // [E][NFN] neighbour trace
  static constexpr int oDNP = oUP + E * NFN;          // neighbour normal derivative
  static constexpr int oJMP = oDNP + E * NFN;
  static constexpr int oAVG = oJMP + E * NFN;
  static constexpr int oF1 = oAVG + E * NFN;
  static constexpr int oF2R = oF1 + E * NFN;
  static constexpr int oF2S = oF2R + E * NFN;
  static constexpr int oFG = oF2S + E * NFN;           // FaceGeo [E][3]
  static constexpr int oVG = oFG + E * 3 * 6;           // Grr, Grs, Gss, J per element
  static constexpr int nT = oVG + E * 4;
  static constexpr size_t bytes = size_t(nT) * sizeof(T) + size_t(E) * 3 * sizeof(int);
};

template <int N, typename T, bool HELM>
__global__ void __launch_bounds__(kThreads)
    sipdg_apply_kernel(int64_t K, int B, const T* __restrict__ geo, const int32_t* __restrict__ conn,
                       const T* __restrict__ ops, T lambda, const T* __restrict__ u, T* __restrict__ Au) {
  using S = Smem<N, T, HELM>;
  constexpr int Np = S::Np, LD = S::LD, Nfp = S::Nfp, NFN = S::NFN, E = S::E;
  constexpr T cpen = T((N + 1) * (N + 2)) / T(2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* sDr = sm + S::oDr;
  T* sDs = sm + S::oDs;
  T* sBr = sm + S::oBr;
  T* sBs = sm + S::oBs;
  T* sM = sm + S::oM;
  T* sMf = sm + S::oMf;
  T* su = sm + S::oU;
  T* sun = sm + S::oUN;
  T* sur = sm + S::oUR;
  T* sus = sm + S::oUS;
  T* swr = sm + S::oWR;
  T* sws = sm + S::oWS;
  T* sup = sm + S::oUP;
  T* sdnp = sm + S::oDNP;
  T* sjmp = sm + S::oJMP;
  T* savg = sm + S::oAVG;
  T* sF1 = sm + S::oF1;
  T* sF2r = sm + S::oF2R;
  T* sF2s = sm + S::oF2S;
  FaceGeo<T>* sfg = reinterpret_cast<FaceGeo<T>*>(sm + S::oFG);
  T* svg = sm + S::oVG;
  int* scode = reinterpret_cast<int*>(sm + S::nT);

  const int tid = threadIdx.x;
  // reference operators -> padded shared memory (row-major, stride LD)
  for (int idx = tid; idx < Np * Np; idx += kThreads) {
    const int i = idx / Np, j = idx - i * Np;
    sDr[i * LD + j] = ops[idx];
    sDs[i * LD + j] = ops[Np * Np + idx];
    sBr[i * LD + j] = ops[2 * Np * Np + idx];
    sBs[i * LD + j] = ops[3 * Np * Np + idx];
    if (HELM) sM[i * LD + j] = ops[4 * Np * Np + idx];
  }
  for (int idx = tid; idx < Nfp * Nfp; idx += kThreads) sMf[idx] = ops[5 * Np * Np + idx];
  __syncthreads();

  const int64_t ntiles = (K + E - 1) / E;
  const int64_t nwork = ntiles * B;
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int b = int(w / ntiles);
    const int64_t e0 = (w - int64_t(b) * ntiles) * E;
    const int ne = int((K - e0) < E ? (K - e0) : E);
    const T* ub = u + size_t(b) * size_t(K) * Np;
    T* Aub = Au + size_t(b) * size_t(K) * Np;

    // ---- stage 1: own nodal values, face geometry, neighbours' nodal values
    for (int idx = tid; idx < ne * Np; idx += kThreads) {
      const int e = idx / Np, i = idx - e * Np;
      su[e * LD + i] = ub[size_t(e0) * Np + idx];
    }
    for (int idx = tid; idx < ne * 3; idx += kThreads) {
      const int e = idx / 3, f = idx - 3 * e;
      const int64_t ge = e0 + e;
      const T rx = geo[4 * ge + 0], sx = geo[4 * ge + 1], ry = geo[4 * ge + 2], sy = geo[4 * ge + 3];
      const T J = T(1) / (rx * sy - ry * sx);
      T gx, gy;
      if (f == 0) { gx = -sx; gy = -sy; }
      else if (f == 1) { gx = rx + sx; gy = ry + sy; }
      else { gx = -rx; gy = -ry; }
      const T gn = sqrt(gx * gx + gy * gy);   // = sJ / J = 1 / h
      const T nx = gx / gn, ny = gy / gn;
      FaceGeo<T> fg;
      fg.sJ = J * gn;
      fg.nr = nx * rx + ny * ry;
      fg.ns = nx * sx + ny * sy;
      const int c = conn[3 * ge + f];
      if (c >= 0) {
        const int64_t nb = c >> 2;
        const int fn = c & 3;
        const T prx = geo[4 * nb + 0], psx = geo[4 * nb + 1], pry = geo[4 * nb + 2], psy = geo[4 * nb + 3];
        T hx, hy;
        if (fn == 0) { hx = -psx; hy = -psy; }
        else if (fn == 1) { hx = prx + psx; hy = pry + psy; }
        else { hx = -prx; hy = -pry; }
        const T hn = sqrt(hx * hx + hy * hy);
        fg.tau = cpen * (gn > hn ? gn : hn);
        fg.ap = nx * prx + ny * pry;
        fg.bp = nx * psx + ny * psy;
      } else {
        fg.tau = cpen * gn;
        fg.ap = T(0);
        fg.bp = T(0);
      }
      sfg[idx] = fg;
      scode[idx] = c;
      if (f == 0) {
        svg[4 * e + 0] = J * (rx * rx + ry * ry);
        svg[4 * e + 1] = J * (rx * sx + ry * sy);
        svg[4 * e + 2] = J * (sx * sx + sy * sy);
        svg[4 * e + 3] = J;
      }
    }
    for (int idx = tid; idx < ne * 3 * Np; idx += kThreads) {
      const int ef = idx / Np, m = idx - ef * Np;
      const int e = ef / 3, f = ef - 3 * e;
      const int c = conn[3 * (e0 + e) + f];
      if (c >= 0) sun[ef * LD + m] = ub[size_t(c >> 2) * Np + m];
    }
    __syncthreads();

    // ---- stage 2: local gradient (r,s) and neighbour traces / normal derivatives
    for (int idx = tid; idx < ne * (Np + NFN); idx += kThreads) {
      if (idx < ne * Np) {
        const int e = idx / Np, i = idx - e * Np;
        const T* ue = su + e * LD;
        T ar = T(0), as = T(0);
#pragma unroll 5
        for (int j = 0; j < Np; ++j) {
          const T uj = ue[j];
          ar += sDr[i * LD + j] * uj;
          as += sDs[i * LD + j] * uj;
        }
        sur[e * LD + i] = ar;
        sus[e * LD + i] = as;
      } else {
        const int q = idx - ne * Np;
        const int ef = q / Nfp, j = q - ef * Nfp;
        const int c = scode[ef];
        if (c >= 0) {
          const int k = fnode(N, c & 3, Nfp - 1 - j);
          const T* un = sun + ef * LD;
          T ar = T(0), as = T(0);
#pragma unroll 5
          for (int m = 0; m < Np; ++m) {
            const T um = un[m];
            ar += sDr[k * LD + m] * um;
            as += sDs[k * LD + m] * um;
          }
          const FaceGeo<T> fg = sfg[ef];
          sdnp[q] = fg.ap * ar + fg.bp * as;
          sup[q] = un[k];
        }
      }
    }
    __syncthreads();

    // ---- stage 3: geometric weights of the gradient; jumps and averages at face nodes
    for (int idx = tid; idx < ne * (Np + NFN); idx += kThreads) {
      if (idx < ne * Np) {
        const int e = idx / Np, i = idx - e * Np;
        const T ur = sur[e * LD + i], us = sus[e * LD + i];
        swr[e * LD + i] = svg[4 * e + 0] * ur + svg[4 * e + 1] * us;
        sws[e * LD + i] = svg[4 * e + 1] * ur + svg[4 * e + 2] * us;
      } else {
        const int q = idx - ne * Np;
        const int ef = q / Nfp, j = q - ef * Nfp;
        const int e = ef / 3, f = ef - 3 * e;
        const int k = fnode(N, f, j);
        const FaceGeo<T> fg = sfg[ef];
        const T um = su[e * LD + k];
        const T dnm = fg.nr * sur[e * LD + k] + fg.ns * sus[e * LD + k];
        const int c = scode[ef];
        T jmp, avg;
        if (c >= 0) {
          jmp = sup[q] - um;
          avg = T(0.5) * (dnm + sdnp[q]);
        } else if (c == -2) {  // Dirichlet: u+ = -u-, grad u+ = grad u-
          jmp = T(-2) * um;
          avg = dnm;
        } else {               // Neumann: u+ = u-, grad u+ = -grad u-
          jmp = T(0);
          avg = T(0);
        }
        sjmp[q] = jmp;
        savg[q] = avg;
      }
    }
    __syncthreads();

    // ---- stage 4: face mass on the face-node data
    for (int q = tid; q < ne * NFN; q += kThreads) {
      const int ef = q / Nfp, j = q - ef * Nfp;
      const FaceGeo<T> fg = sfg[ef];
      const T* jf = sjmp + ef * Nfp;
      const T* af = savg + ef * Nfp;
      T m1 = T(0), m2 = T(0);
#pragma unroll
      for (int l = 0; l < Nfp; ++l) {
        const T mf = sMf[j * Nfp + l];
        m1 += mf * (af[l] + fg.tau * jf[l]);
        m2 += mf * jf[l];
      }
      sF1[q] = -fg.sJ * m1;
      const T f2 = T(0.5) * fg.sJ * m2;
      sF2r[q] = fg.nr * f2;
      sF2s[q] = fg.ns * f2;
    }
    __syncthreads();

    // ---- stage 5: volume term, lifted face terms, output
    for (int idx = tid; idx < ne * Np; idx += kThreads) {
      const int e = idx / Np, i = idx - e * Np;
      const T* wr = swr + e * LD;
      const T* ws = sws + e * LD;
      T acc = T(0);
#pragma unroll 5
      for (int j = 0; j < Np; ++j) acc += sBr[i * LD + j] * wr[j] + sBs[i * LD + j] * ws[j];
      if (HELM) {
        const T* ue = su + e * LD;
        T am = T(0);
#pragma unroll 5
        for (int j = 0; j < Np; ++j) am += sM[i * LD + j] * ue[j];
        acc += lambda * svg[4 * e + 3] * am;
      }
      const T* f2r = sF2r + e * NFN;
      const T* f2s = sF2s + e * NFN;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
#pragma unroll
        for (int j = 0; j < Nfp; ++j) {
          const int k = fnode(N, f, j);
          acc += sDr[k * LD + i] * f2r[f * Nfp + j] + sDs[k * LD + i] * f2s[f * Nfp + j];
        }
      }
      // face-node contributions (vertices lie on two faces; fixed order 0,1,2)
      int row = 0, rs = 0;
      while (i >= rs + (N + 1 - row)) {
        rs += N + 1 - row;
        ++row;
      }
      const int col = i - rs;
      const T* f1 = sF1 + e * NFN;
      if (row == 0) acc += f1[0 * Nfp + col];
      if (col == N - row) acc += f1[1 * Nfp + row];
      if (col == 0) acc += f1[2 * Nfp + (N - row)];
      Aub[size_t(e0) * Np + idx] = acc;
    }
    __syncthreads();
  }
}

struct LaunchCfg {
  int grid = 0;
  size_t smem = 0;
  bool ready = false;
};

template <int N, typename T, bool HELM>
cudaError_t launch_t(const dg_mesh* m, int B, double lambda, const void* u, void* Au, cudaStream_t st) {
  using S = Smem<N, T, HELM>;
  static LaunchCfg cfg[64];  // per device ordinal
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev >= 64) return cudaErrorInvalidDevice;
  LaunchCfg& c = cfg[dev];
  auto kern = sipdg_apply_kernel<N, T, HELM>;
  std::unique_lock<std::mutex> lk(table_mutex());
  if (!c.ready) {
    c.smem = S::bytes;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(c.smem));
    if (err != cudaSuccess) return err;
    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, c.smem);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    c.grid = (per_sm > 0 ? per_sm : 1) * sms;
    c.ready = true;
  }
  lk.unlock();
  const int64_t ntiles = (m->K + S::E - 1) / S::E;
  const int64_t work = ntiles * B;
  const int grid = int(work < c.grid ? work : c.grid);
  if (grid <= 0) return cudaSuccess;
  const T* geo = std::is_same<T, double>::value ? reinterpret_cast<const T*>(m->geo64)
                                                 : reinterpret_cast<const T*>(m->geo32);
  const T* ops = reinterpret_cast<const T*>(std::is_same<T, double>::value ? m->ops64[N].buf : m->ops32[N].buf);
  kern<<<grid, kThreads, c.smem, st>>>(m->K, B, geo, m->conn, ops, T(lambda), reinterpret_cast<const T*>(u),
                                       reinterpret_cast<T*>(Au)); note_launch();
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_n(const dg_mesh* m, dg_prec prec, int B, double lambda, const void* u, void* Au, cudaStream_t st) {
  const bool helm = lambda != 0.0;
  if (prec == DG_F64)
    return helm ? launch_t<N, double, true>(m, B, lambda, u, Au, st) : launch_t<N, double, false>(m, B, lambda, u, Au, st);
  return helm ? launch_t<N, float, true>(m, B, lambda, u, Au, st) : launch_t<N, float, false>(m, B, lambda, u, Au, st);
}

}  // namespace

#define DG_TE_DECL(n)                                                                                       \
  cudaError_t launch_apply_f32_n##n(const dg_mesh* m, int B, double lambda, const float* u, float* Au, float2* face, \
                                   cudaStream_t st);
DG_TE_DECL(1) DG_TE_DECL(2) DG_TE_DECL(3) DG_TE_DECL(4) DG_TE_DECL(5) DG_TE_DECL(6) DG_TE_DECL(7) DG_TE_DECL(8)
DG_TE_DECL(9)
#undef DG_TE_DECL

// Kernel choice: the tile kernel above (FP64 or FP32), register-blocked FP32
// GEMMs (apply_gemm.cuh, with the mesh face scratch), FP64 products on the BF16
// tensor cores with exact integer slicing (apply_tensor.cu; FP64 and FP32), or one element per
// thread (apply_ept.cu). DG_F64_DFMA forces the tile kernel in FP64.

// Built-in kernel per degree and precision (the measured winners on the
// 524,288-triangle workload; dg_autotune replaces them per mesh). Above degree
// 8 the tcgen05 FP32 kernel's operands no longer fit in tensor memory.
int default_kernel(int degree, bool f64) {
  if (f64) return degree >= 3 ? DG_KERNEL_TC64 : DG_KERNEL_EPT;
  if (degree <= 3) return DG_KERNEL_EPT;
  if (degree <= 8) return DG_KERNEL_TC05;
  return degree == 9 ? DG_KERNEL_TENSOR : DG_KERNEL_TILE;
}

bool kernel_valid(int kernel, int degree, bool f64) {
  switch (kernel) {
    case DG_KERNEL_TILE: return true;
    case DG_KERNEL_GEMM: return !f64 && degree <= 9;  // shared memory
    case DG_KERNEL_TENSOR: return tensor_supported(degree);
    case DG_KERNEL_TENSOR_PIPE: return tensor_supported(degree);
    case DG_KERNEL_EPT: return ept_supported(degree);
    case DG_KERNEL_TC05: return !f64 && degree <= 8;  // tensor memory
    case DG_KERNEL_TC64: return f64 && tc64_supported(degree);
    default: return false;
  }
}

int selected_kernel(const dg_mesh* m, int degree, dg_prec prec, bool helm) {
  if (prec == DG_F64_DFMA) return DG_KERNEL_TILE;
  const int k = m->kern[degree][prec == DG_F32 ? 1 : 0][helm ? 1 : 0];
  return k == DG_KERNEL_AUTO ? default_kernel(degree, prec == DG_F64) : k;
}

cudaError_t launch_apply(const dg_mesh* mc, int degree, dg_prec prec, int B, double lambda, const void* u, void* Au,
                         cudaStream_t st, double* c1_scratch) {
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  const bool helm = lambda != 0.0;
  int k;
  if (prec == DG_F64_DFMA) {  // the tile kernel on the FP64 pipe, whatever the table says
    k = DG_KERNEL_TILE;
    prec = DG_F64;
  } else {
    k = m->kern[degree][prec == DG_F32 ? 1 : 0][helm ? 1 : 0];
    if (k == DG_KERNEL_AUTO) k = default_kernel(degree, prec == DG_F64);
  }
  const bool f64 = prec == DG_F64;
  if (!kernel_valid(k, degree, f64)) return cudaErrorInvalidValue;
  if (k == DG_KERNEL_EPT) return launch_apply_ept(m, degree, f64, B, lambda, u, Au, st);
  if (k == DG_KERNEL_TC64) {
    return launch_apply_tc64(m, degree, B, lambda, static_cast<const double*>(u), static_cast<double*>(Au), st,
                             c1_scratch);
  }
  if (k == DG_KERNEL_TC05) {
    if (tc05_usable(u, Au))
      return launch_apply_tc05(m, degree, B, lambda, static_cast<const float*>(u), static_cast<float*>(Au), st);
    k = DG_KERNEL_TENSOR;  // unaligned fields: the mma.sync tensor kernel takes them
  }
  if (k == DG_KERNEL_TENSOR || k == DG_KERNEL_TENSOR_PIPE)
    return launch_apply_tensor(m, degree, f64, B, lambda, u, Au, k == DG_KERNEL_TENSOR_PIPE, st, c1_scratch);
  if (k == DG_KERNEL_GEMM) {
    const int dmax = degree > m->N ? degree : m->N;
    const size_t need = size_t(B) * size_t(m->K) * 3 * size_t(dmax + 1);
    if (m->face32_cap < need) {
      cudaFree(m->face32);
      m->face32 = nullptr;
      m->face32_cap = 0;
      cudaError_t e = cudaMalloc(&m->face32, need * sizeof(float2));
      if (e == cudaSuccess) e = poison(m->face32, need * sizeof(float2), POISON_APPLY);
      if (e != cudaSuccess) return e;
      m->face32_cap = need;
      ++m->scratch_gen;
    }
    const float* uf = reinterpret_cast<const float*>(u);
    float* of = reinterpret_cast<float*>(Au);
    switch (degree) {
      case 1: return launch_apply_f32_n1(m, B, lambda, uf, of, m->face32, st);
      case 2: return launch_apply_f32_n2(m, B, lambda, uf, of, m->face32, st);
      case 3: return launch_apply_f32_n3(m, B, lambda, uf, of, m->face32, st);
      case 4: return launch_apply_f32_n4(m, B, lambda, uf, of, m->face32, st);
      case 5: return launch_apply_f32_n5(m, B, lambda, uf, of, m->face32, st);
      case 6: return launch_apply_f32_n6(m, B, lambda, uf, of, m->face32, st);
      case 7: return launch_apply_f32_n7(m, B, lambda, uf, of, m->face32, st);
      case 8: return launch_apply_f32_n8(m, B, lambda, uf, of, m->face32, st);
      case 9: return launch_apply_f32_n9(m, B, lambda, uf, of, m->face32, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (degree) {  // DG_KERNEL_TILE, FP64 or FP32
    case 1: return launch_n<1>(mc, prec, B, lambda, u, Au, st);
    case 2: return launch_n<2>(mc, prec, B, lambda, u, Au, st);
    case 3: return launch_n<3>(mc, prec, B, lambda, u, Au, st);
    case 4: return launch_n<4>(mc, prec, B, lambda, u, Au, st);
    case 5: return launch_n<5>(mc, prec, B, lambda, u, Au, st);
    case 6: return launch_n<6>(mc, prec, B, lambda, u, Au, st);
    case 7: return launch_n<7>(mc, prec, B, lambda, u, Au, st);
    case 8: return launch_n<8>(mc, prec, B, lambda, u, Au, st);
    case 9: return launch_n<9>(mc, prec, B, lambda, u, Au, st);
    case 10: return launch_n<10>(mc, prec, B, lambda, u, Au, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgx
