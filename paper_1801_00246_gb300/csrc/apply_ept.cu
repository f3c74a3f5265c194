// SIPDG apply with one element per thread, for low degrees (N <= 3).
//
// At low N an element is a handful of nodes and the apply is bound by memory
// traffic (FP32) or the FP64 pipe, not by the dense products, so the tiled
// kernels' shared-memory staging and block barriers are pure overhead. Here a
// thread keeps its element's nodal values in registers and evaluates the
// operator of Eq. ellipticOp3 in the factored order used throughout:
//   (ur, us) = (Dr u, Ds u),  (wr, ws) = G (ur, us),
//   Au = Br wr + Bs ws + sum_f [ (nr Dr_f + ns Ds_f)^T F2_f + E_f F1_f ] (+ lambda J M u)
// with, at the face nodes of face f, the jump [u] = u+ - u-, the average
// normal derivative {n.grad u}, F2 = 1/2 sJ Mf [u] and
// F1 = -sJ Mf ({n.grad u} + tau [u]). Dirichlet faces take the ghost state
// u+ = -u-, grad u+ = grad u-; Neumann faces u+ = u-, grad u+ = -grad u-.
//
// The reference operators sit in constant memory: every thread of a warp reads
// the same entry at the same time (a broadcast), and with the loops unrolled
// the entries become constant-bank operands of the multiply-adds. The
// neighbour's normal derivative at a shared face node needs rows of Dr, Ds
// picked by the neighbour's face number (a per-thread index), so those come
// from a shared-memory copy. The neighbour's nodal values and geometry are
// re-read (mostly L2 hits) instead of being passed through a face buffer.
#include <type_traits>
#include <vector>

#include "dg_internal.h"

namespace dgx {
namespace {

constexpr int kEptMaxN = 3;
__host__ __device__ constexpr int np_of(int N) { return (N + 1) * (N + 2) / 2; }
// per degree: Dr, Ds, Br, Bs, M (Np^2 each), Mf ((N+1)^2)
__host__ __device__ constexpr int block_of(int N) { return 5 * np_of(N) * np_of(N) + (N + 1) * (N + 1); }
__host__ __device__ constexpr int off_of(int N) { return N <= 1 ? 0 : off_of(N - 1) + block_of(N - 1); }
constexpr int kConstWords = off_of(kEptMaxN + 1);

__constant__ double c_ops64[kConstWords];
__constant__ float c_ops32[kConstWords];

// entries read straight from the constant arrays (with a compile-time index,
// a constant-bank operand; through a generic pointer they would be loads)
template <typename T>
__device__ __forceinline__ T cop(int i);
template <>
__device__ __forceinline__ double cop<double>(int i) { return c_ops64[i]; }
template <>
__device__ __forceinline__ float cop<float>(int i) { return c_ops32[i]; }

template <int N>
__host__ __device__ constexpr int fnode(int f, int j) {
  return f == 0 ? j : (f == 1 ? (j * (N + 1) - j * (j - 1) / 2) + (N - j) : ((N - j) * (N + 1) - (N - j) * (N - j - 1) / 2));
}
template <int N>
__device__ __forceinline__ int fnode_rt(int f, int j) {
  auto rs = [](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

template <typename T>
__device__ __forceinline__ void face_grad(T rx, T sx, T ry, T sy, int f, T& gx, T& gy) {
  if (f == 0) { gx = -sx; gy = -sy; }
  else if (f == 1) { gx = rx + sx; gy = ry + sy; }
  else { gx = -rx; gy = -ry; }
}

// geo: FP32 raw (rx, sx, ry, sy) per element with ih (max inverse length per
// face); FP64: gx, 16 words per element (J, Grr, Grs, Gss | per face nr, ns,
// sJ, ihmax) as set up with the mesh.
// Occupancy floor per degree: at N = 1 the kernel is latency-bound and wants
// more resident warps than an unconstrained register allocation leaves.
template <int N, typename T>
constexpr int ept_min_blocks() {
  return sizeof(T) == 4 ? (N == 1 ? 6 : (N == 2 ? 3 : 1)) : (N == 1 ? 3 : 1);
}

// Grid: x over the elements of one right-hand side, y over the batch, so no
// thread divides by K. Offsets within one right-hand side fit in 32 bits
// (checked by the launcher).
template <int N, typename T, bool HELM>
__global__ void __launch_bounds__(128, ept_min_blocks<N, T>()) ept_apply(
    int K, const float* __restrict__ geo32, const float* __restrict__ ih32, const double* __restrict__ gx,
    const int32_t* __restrict__ conn, T lambda, const T* __restrict__ ub, T* __restrict__ Aub) {
  constexpr int Np = np_of(N), Nfp = N + 1;
  constexpr int oDr = off_of(N), oDs = oDr + Np * Np, oBr = oDs + Np * Np, oBs = oBr + Np * Np,
                oM = oBs + Np * Np, oMf = oM + Np * Np;
  constexpr T cpen = T((N + 1) * (N + 2)) / T(2);
  __shared__ T sD[2 * Np * Np];  // Dr, Ds for the neighbour's face rows (degree 1 needs none)
  if (N > 1) {
    for (int i = threadIdx.x; i < 2 * Np * Np; i += blockDim.x) sD[i] = cop<T>(oDr + i);
    __syncthreads();
  }
  const T* __restrict__ u = ub + size_t(blockIdx.y) * size_t(K) * Np;  // this right-hand side
  T* __restrict__ Au = Aub + size_t(blockIdx.y) * size_t(K) * Np;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
    const int be = e;  // element offsets below are within this right-hand side
    // every load this element needs is issued up front (own values, the three
    // connectivity words, then all neighbours' values and metric), so their
    // latencies overlap instead of adding up face by face
    T uv[Np];
#pragma unroll
    for (int m = 0; m < Np; ++m) uv[m] = u[be * Np + m];
    int code[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) code[f] = conn[3 * e + f];
    T unv[3][Np];
    T ng[3][4];  // FP32: the neighbour's (rx, sx, ry, sy); FP64: its (nr, ns) on the shared face
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const int nb = code[f] >= 0 ? (code[f] >> 2) : e;
      const int fn = code[f] >= 0 ? (code[f] & 3) : 0;
#pragma unroll
      for (int m = 0; m < Np; ++m) unv[f][m] = u[nb * Np + m];
      if constexpr (std::is_same<T, double>::value) {
        const double* gg = gx + 16 * nb + 4 + 4 * fn;
        ng[f][0] = gg[0];
        ng[f][1] = gg[1];
        ng[f][2] = ng[f][3] = 0.0;
      } else {
        const float4 g = reinterpret_cast<const float4*>(geo32)[nb];
        ng[f][0] = g.x;
        ng[f][1] = g.y;
        ng[f][2] = g.z;
        ng[f][3] = g.w;
      }
    }
    // geometry
    T J, Grr, Grs, Gss, nr[3], ns[3], sJ[3], tau[3], nx[3], ny[3];
    if constexpr (std::is_same<T, double>::value) {
      const double* g = gx + 16 * e;
      J = g[0], Grr = g[1], Grs = g[2], Gss = g[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        nr[f] = g[4 + 4 * f];
        ns[f] = g[5 + 4 * f];
        sJ[f] = g[6 + 4 * f];
        tau[f] = cpen * g[7 + 4 * f];
        nx[f] = ny[f] = 0.0;
      }
    } else {
      const float4 g = reinterpret_cast<const float4*>(geo32)[e];
      const float rx = g.x, sx = g.y, ry = g.z, sy = g.w;
      // FP32 metric from the four stored words (fast reciprocal and reciprocal
      // square root: a few ulp, far inside the FP32 tolerance)
      J = __frcp_rn(rx * sy - ry * sx);
      Grr = J * (rx * rx + ry * ry);
      Grs = J * (rx * sx + ry * sy);
      Gss = J * (sx * sx + sy * sy);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        float fx, fy;
        face_grad(rx, sx, ry, sy, f, fx, fy);
        const float g2 = fx * fx + fy * fy;
        const float ig = rsqrtf(g2);
        nx[f] = fx * ig;
        ny[f] = fy * ig;
        nr[f] = nx[f] * rx + ny[f] * ry;
        ns[f] = nx[f] * sx + ny[f] * sy;
        sJ[f] = J * (g2 * ig);
        tau[f] = cpen * ih32[3 * e + f];
      }
    }
    // reference gradient
    T ur[Np], us[Np];
#pragma unroll
    for (int i = 0; i < Np; ++i) {
      if (N == 1 && i > 0) {  // degree 1: a constant gradient
        ur[i] = ur[0];
        us[i] = us[0];
        continue;
      }
      T a = T(0), b = T(0);
#pragma unroll
      for (int m = 0; m < Np; ++m) {
        a += cop<T>(oDr + i * Np + m) * uv[m];
        b += cop<T>(oDs + i * Np + m) * uv[m];
      }
      ur[i] = a;
      us[i] = b;
    }
    // own outward normal derivatives at the face nodes (ur, us die after the volume term)
    T dn[3][Nfp];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int j = 0; j < Nfp; ++j) dn[f][j] = nr[f] * ur[fnode<N>(f, j)] + ns[f] * us[fnode<N>(f, j)];
    // volume term
    T out[Np];
#pragma unroll
    for (int i = 0; i < Np; ++i) out[i] = T(0);
#pragma unroll
    for (int m = 0; m < Np; ++m) {
      const T wr = Grr * ur[m] + Grs * us[m];
      const T ws = Grs * ur[m] + Gss * us[m];
#pragma unroll
      for (int i = 0; i < Np; ++i) out[i] += cop<T>(oBr + i * Np + m) * wr + cop<T>(oBs + i * Np + m) * ws;
    }
    if (HELM) {
      const T lj = lambda * J;
#pragma unroll
      for (int i = 0; i < Np; ++i) {
        T a = T(0);
#pragma unroll
        for (int m = 0; m < Np; ++m) a += cop<T>(oM + i * Np + m) * uv[m];
        out[i] += lj * a;
      }
    }
    // faces
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T jm[Nfp], av[Nfp];
#pragma unroll
      for (int j = 0; j < Nfp; ++j) {
        const bool dir = code[f] == -2;
        jm[j] = dir ? T(-2) * uv[fnode<N>(f, j)] : T(0);
        av[j] = dir ? dn[f][j] : T(0);
      }
      if (code[f] >= 0) {
        const int fn = code[f] & 3;
        T gnr, gns;  // neighbour's outward normal derivative = gnr (Dr u+) + gns (Ds u+)
        if constexpr (std::is_same<T, double>::value) {
          gnr = ng[f][0];
          gns = ng[f][1];
        } else {
          // its outward normal is -n: -n.grad u+ with grad u+ from its own metric
          gnr = -(nx[f] * ng[f][0] + ny[f] * ng[f][2]);
          gns = -(nx[f] * ng[f][1] + ny[f] * ng[f][3]);
        }
        if constexpr (N == 1) {
          // degree 1: the neighbour's gradient is constant (every row of Dr, Ds is
          // the same), so one row serves both face nodes
          T a = T(0), b = T(0);
#pragma unroll
          for (int m = 0; m < Np; ++m) {
            a += cop<T>(oDr + m) * unv[f][m];
            b += cop<T>(oDs + m) * unv[f][m];
          }
          const T dnp = gnr * a + gns * b;
#pragma unroll
          for (int j = 0; j < Nfp; ++j) {
            const int kn = fnode_rt<N>(fn, Nfp - 1 - j);
            const T up = kn == 0 ? unv[f][0] : (kn == 1 ? unv[f][1] : unv[f][2]);
            jm[j] = up - uv[fnode<N>(f, j)];
            av[j] = T(0.5) * (dn[f][j] - dnp);
          }
        } else {
#pragma unroll
          for (int j = 0; j < Nfp; ++j) {
            const int kn = fnode_rt<N>(fn, Nfp - 1 - j);
            T a = T(0), b = T(0), up = T(0);
#pragma unroll
            for (int m = 0; m < Np; ++m) {
              a += sD[kn * Np + m] * unv[f][m];
              b += sD[Np * Np + kn * Np + m] * unv[f][m];
              up = (m == kn) ? unv[f][m] : up;
            }
            jm[j] = up - uv[fnode<N>(f, j)];
            av[j] = T(0.5) * (dn[f][j] - (gnr * a + gns * b));
          }
        }
      }
      // face mass along the face, then lift
#pragma unroll
      for (int j = 0; j < Nfp; ++j) {
        T m1 = T(0), m2 = T(0);
#pragma unroll
        for (int l = 0; l < Nfp; ++l) {
          const T mf = cop<T>(oMf + j * Nfp + l);
          m1 += mf * (av[l] + tau[f] * jm[l]);
          m2 += mf * jm[l];
        }
        const T f2 = T(0.5) * sJ[f] * m2;
        const T a2 = nr[f] * f2, b2 = ns[f] * f2;
        const int k = fnode<N>(f, j);
#pragma unroll
        for (int i = 0; i < Np; ++i) out[i] += cop<T>(oDr + k * Np + i) * a2 + cop<T>(oDs + k * Np + i) * b2;
        out[k] -= sJ[f] * m1;
      }
    }
#pragma unroll
    for (int i = 0; i < Np; ++i) Au[be * Np + i] = out[i];
  }
}

bool g_uploaded[64] = {};

cudaError_t upload(dg_mesh* m) {
  std::vector<double> h(kConstWords, 0.0);
  for (int N = 1; N <= kEptMaxN; ++N) {
    if (m->ref[N].N == 0) m->ref[N] = build_reference(N);
    const RefElem& R = m->ref[N];
    const int Np = R.Np, Nfp = R.Nfp;
    double* o = h.data() + off_of(N);
    for (int i = 0; i < Np * Np; ++i) {
      o[i] = R.Dr[i];
      o[Np * Np + i] = R.Ds[i];
      o[2 * Np * Np + i] = R.Br[i];
      o[3 * Np * Np + i] = R.Bs[i];
      o[4 * Np * Np + i] = R.M[i];
    }
    for (int i = 0; i < Nfp * Nfp; ++i) o[5 * Np * Np + i] = R.Mf[i];
  }
  std::vector<float> hf(h.begin(), h.end());
  cudaError_t e = cudaMemcpyToSymbol(c_ops64, h.data(), sizeof(double) * kConstWords);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_ops32, hf.data(), sizeof(float) * kConstWords);
}

template <int N, typename T, bool HELM>
cudaError_t launch(dg_mesh* m, int B, double lambda, const void* u, void* Au, cudaStream_t st) {
  constexpr int Np = np_of(N);
  if (m->K * Np + 16 * m->K >= (int64_t(1) << 31) || B > 65535) return cudaErrorInvalidValue;  // 32-bit offsets
  const int64_t blocks = (m->K + 127) / 128;
  if (blocks < 1 || B < 1) return cudaSuccess;
  ept_apply<N, T, HELM><<<dim3(unsigned(blocks), unsigned(B)), 128, 0, st>>>(
      int(m->K), m->geo32, m->ih32, m->geox, m->conn, T(lambda), reinterpret_cast<const T*>(u),
      reinterpret_cast<T*>(Au));
  note_launch();
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_n(dg_mesh* m, bool f64, int B, double lambda, const void* u, void* Au, cudaStream_t st) {
  const bool helm = lambda != 0.0;
  if (f64) return helm ? launch<N, double, true>(m, B, lambda, u, Au, st) : launch<N, double, false>(m, B, lambda, u, Au, st);
  return helm ? launch<N, float, true>(m, B, lambda, u, Au, st) : launch<N, float, false>(m, B, lambda, u, Au, st);
}

}  // namespace

bool ept_supported(int degree) { return degree >= 1 && degree <= kEptMaxN; }

cudaError_t launch_apply_ept(dg_mesh* m, int degree, bool f64, int B, double lambda, const void* u, void* Au,
                             cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(table_mutex());
    if (!g_uploaded[dev & 63]) {
      e = upload(m);
      if (e != cudaSuccess) return e;
      g_uploaded[dev & 63] = true;
    }
  }
  switch (degree) {
    case 1: return launch_n<1>(m, f64, B, lambda, u, Au, st);
    case 2: return launch_n<2>(m, f64, B, lambda, u, Au, st);
    case 3: return launch_n<3>(m, f64, B, lambda, u, Au, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgx
