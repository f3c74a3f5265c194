// SIPDG Poisson / screened-Poisson operator on affine tetrahedra, and its
// Jacobi-preconditioned CG solve: the three-dimensional extension the paper
// names as its next step (Section 6), with the bilinear form of
// Eq. ellipticOp1 on tetrahedra in the factored grouping of Eq. ellipticOp3
// (volume gradient through Dr/Ds/Dt and the element metric, face jumps and
// averages with the interior penalty, lift through the face mass):
//
//   (A u)_i = J [Br wr + Bs ws + Bt wt]_i             (w_a = sum_b G_ab u_b, u_b = D_b u)
//           + lambda J [M u]_i
//           + sum_f sum_j (sum_b nr_b D_b[k_fj][i]) F2_fj  1/2 (n.grad l_i, [u])_f
//           + sum_{f,j: k_fj = i} F1_fj                     -(l_i, n.{grad u} + tau [u])_f
//
// with B_b = D_b^T M, G = (grad r_a . grad r_b), nr_b = n . grad r_b, and at the
// face nodes F1 = sJ Mf(-{n.grad u} - tau [u]), F2 = 1/2 sJ Mf [u]. Readings
// for three dimensions: tau = (N+1)(N+3)/3 max(1/h-, 1/h+), h = |E| / |face|
// (the triangle's (N+1)(N+2)/2 is the d = 2 case of (N+1)(N+d)/d); boundary
// faces as on triangles (Dirichlet ghost u+ = -u-, grad u+ = grad u-;
// Neumann: no face terms); equispaced nodes (i, j, k)/N with i + j + k <= N,
// ordered by k, then j, then i, whose face nodes form the equispaced triangle
// of each face. Reference tetrahedron v0 = (-1,-1,-1), v1 = (1,-1,-1),
// v2 = (-1,1,-1), v3 = (-1,-1,1); faces (v0,v1,v2), (v0,v1,v3), (v1,v2,v3),
// (v0,v2,v3), opposite v3, v2, v0, v1.
//
// Reference operators are built on the host from a monomial Vandermonde
// matrix and Gauss-Jacobi quadrature; a neighbour's face nodes are matched to
// the element's by their physical coordinates at setup. The apply is two
// kernels with the reference operators in shared memory: the first forms the
// reference gradient once per element and writes w_a = G_ab D_b u and the face
// traces (u, n.grad u); the second takes jumps and averages from the element's
// and its neighbours' traces, lifts them through the face mass and applies
// D_b^T to J M w_b plus the lifted jumps, so that no gradient is formed twice.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>
#include <vector>

#include "dg_internal.h"

namespace dgx {
namespace tet {

constexpr int kMaxTetN = 5;
constexpr int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

inline int np3(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
inline int nfp3(int N) { return (N + 1) * (N + 2) / 2; }

struct TetRef {
  int N = 0, Np = 0, Nfp = 0;
  std::vector<double> r, s, t;
  std::vector<double> D[3];   // Dr, Ds, Dt (Np x Np, row-major: D[k][m] = d l_m / d r_b at node k)
  std::vector<double> Bm[3];  // B_b = D_b^T M
  std::vector<double> M;      // mass
  std::vector<double> Mf[4];  // face mass on each reference face, per unit reference-face area ratio
  std::vector<int> fmask[4];  // volume node of face node j
  double face_area[4] = {};   // reference face areas
  // Jacobi pieces: S_ab[i][i] (a <= b: rr, rs, rt, ss, st, tt), M[i][i], and per face
  // node fc_b[f][j] = sum_l Mf[j][l] D_b[k_l][k_j]
  std::vector<double> dS[6], dM, fc[3][4];
};

std::vector<int> monomial_exps(int N) {
  std::vector<int> ex;
  for (int c = 0; c <= N; ++c)
    for (int b = 0; b + c <= N; ++b)
      for (int a = 0; a + b + c <= N; ++a) {
        ex.push_back(a);
        ex.push_back(b);
        ex.push_back(c);
      }
  return ex;
}

double ipow(double x, int k) {
  double v = 1.0;
  for (int i = 0; i < k; ++i) v *= x;
  return v;
}

// monomial values (deriv = -1) or derivative along axis deriv at (r, s, t)
void monomial_row(int N, double r, double s, double t, int deriv, double* out) {
  const std::vector<int> ex = monomial_exps(N);
  const int n = int(ex.size()) / 3;
  for (int q = 0; q < n; ++q) {
    const int a = ex[3 * q], b = ex[3 * q + 1], c = ex[3 * q + 2];
    double v;
    if (deriv < 0) v = ipow(r, a) * ipow(s, b) * ipow(t, c);
    else if (deriv == 0) v = a ? a * ipow(r, a - 1) * ipow(s, b) * ipow(t, c) : 0.0;
    else if (deriv == 1) v = b ? b * ipow(r, a) * ipow(s, b - 1) * ipow(t, c) : 0.0;
    else v = c ? c * ipow(r, a) * ipow(s, b) * ipow(t, c - 1) : 0.0;
    out[q] = v;
  }
}

TetRef build_tet(int N) {
  TetRef R;
  R.N = N;
  R.Np = np3(N);
  R.Nfp = nfp3(N);
  const int Np = R.Np, Nfp = R.Nfp;
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j + k <= N; ++j)
      for (int i = 0; i + j + k <= N; ++i) {
        R.r.push_back(-1.0 + 2.0 * i / N);
        R.s.push_back(-1.0 + 2.0 * j / N);
        R.t.push_back(-1.0 + 2.0 * k / N);
      }
  // nodal basis: l_m = sum_q Vinv[q][m] mono_q
  std::vector<double> V(size_t(Np) * Np);
  for (int k = 0; k < Np; ++k) monomial_row(N, R.r[k], R.s[k], R.t[k], -1, &V[size_t(k) * Np]);
  const std::vector<double> Vinv = invert(Np, V);
  auto nodal_row = [&](double r, double s, double t, int deriv, double* out) {
    std::vector<double> m(Np);
    monomial_row(N, r, s, t, deriv, m.data());
    for (int c = 0; c < Np; ++c) {
      double a = 0.0;
      for (int q = 0; q < Np; ++q) a += m[q] * Vinv[size_t(q) * Np + c];
      out[c] = a;
    }
  };
  for (int b = 0; b < 3; ++b) {
    R.D[b].assign(size_t(Np) * Np, 0.0);
    for (int k = 0; k < Np; ++k) nodal_row(R.r[k], R.s[k], R.t[k], b, &R.D[b][size_t(k) * Np]);
  }
  // mass by a collapsed Gauss-Jacobi rule exact to degree 2N + 1
  std::vector<double> xa, wa, xb, wb, xc, wc;
  const int nq = N + 1;
  gauss_jacobi(nq, 0.0, 0.0, xa, wa);
  gauss_jacobi(nq, 1.0, 0.0, xb, wb);
  gauss_jacobi(nq, 2.0, 0.0, xc, wc);
  R.M.assign(size_t(Np) * Np, 0.0);
  std::vector<double> L(Np);
  for (int i = 0; i < nq; ++i)
    for (int j = 0; j < nq; ++j)
      for (int k = 0; k < nq; ++k) {
        const double a = xa[i], b = xb[j], c = xc[k], w = wa[i] * wb[j] * wc[k] / 8.0;
        nodal_row(0.25 * (1 + a) * (1 - b) * (1 - c) - 1, 0.5 * (1 + b) * (1 - c) - 1, c, -1, L.data());
        for (int p = 0; p < Np; ++p)
          for (int q = 0; q < Np; ++q) R.M[size_t(p) * Np + q] += w * L[p] * L[q];
      }
  for (int b = 0; b < 3; ++b) {  // B_b = D_b^T M
    R.Bm[b].assign(size_t(Np) * Np, 0.0);
    for (int i = 0; i < Np; ++i)
      for (int m = 0; m < Np; ++m) {
        double a = 0.0;
        for (int k = 0; k < Np; ++k) a += R.D[b][size_t(k) * Np + i] * R.M[size_t(k) * Np + m];
        R.Bm[b][size_t(i) * Np + m] = a;
      }
  }
  // faces: the nodes on each face, in volume-node order, and the face mass by a
  // collapsed triangle rule mapped onto the reference face
  const double V3[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  std::vector<double> ya, wya, yb, wyb;
  gauss_jacobi(nq, 0.0, 0.0, ya, wya);
  gauss_jacobi(nq, 1.0, 0.0, yb, wyb);
  for (int f = 0; f < 4; ++f) {
    const double* A = V3[kFaceVerts[f][0]];
    const double* Bv = V3[kFaceVerts[f][1]];
    const double* C = V3[kFaceVerts[f][2]];
    double e1[3], e2[3], cr[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = Bv[d] - A[d];
      e2[d] = C[d] - A[d];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    R.face_area[f] = area;
    const double nrm[3] = {cr[0] / (2 * area), cr[1] / (2 * area), cr[2] / (2 * area)};
    for (int k = 0; k < Np; ++k) {  // a node lies on the face when it is in the face's plane
      const double d = (R.r[k] - A[0]) * nrm[0] + (R.s[k] - A[1]) * nrm[1] + (R.t[k] - A[2]) * nrm[2];
      if (std::fabs(d) < 1e-10) R.fmask[f].push_back(k);
    }
    if (int(R.fmask[f].size()) != Nfp) throw std::runtime_error("tetrahedron face node count");
    R.Mf[f].assign(size_t(Nfp) * Nfp, 0.0);
    std::vector<double> Lv(Np);
    for (int i = 0; i < nq; ++i)
      for (int j = 0; j < nq; ++j) {
        // bi-unit triangle point (p, q) and weight (its area is 2), mapped to the face
        const double p = 0.5 * (1.0 + ya[i]) * (1.0 - yb[j]) - 1.0, q = yb[j];
        const double w = wya[i] * wyb[j] * 0.5 * (area / 2.0);  // reference-face area element
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = A[d] + 0.5 * (p + 1.0) * e1[d] + 0.5 * (q + 1.0) * e2[d];
        nodal_row(x[0], x[1], x[2], -1, Lv.data());
        for (int a = 0; a < Nfp; ++a)
          for (int c = 0; c < Nfp; ++c) R.Mf[f][size_t(a) * Nfp + c] += w * Lv[R.fmask[f][a]] * Lv[R.fmask[f][c]];
      }
  }
  // Jacobi pieces
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q) {
    R.dS[q].assign(Np, 0.0);
    for (int i = 0; i < Np; ++i) {  // (D_a^T M D_b)[i][i]
      double a = 0.0;
      for (int k = 0; k < Np; ++k)
        for (int m = 0; m < Np; ++m)
          a += R.D[pa[q]][size_t(k) * Np + i] * R.M[size_t(k) * Np + m] * R.D[pb[q]][size_t(m) * Np + i];
      R.dS[q][i] = a;
    }
  }
  R.dM.resize(Np);
  for (int i = 0; i < Np; ++i) R.dM[i] = R.M[size_t(i) * Np + i];
  for (int b = 0; b < 3; ++b)
    for (int f = 0; f < 4; ++f) {
      R.fc[b][f].assign(Nfp, 0.0);
      for (int j = 0; j < Nfp; ++j) {
        double a = 0.0;
        for (int l = 0; l < Nfp; ++l)
          a += R.Mf[f][size_t(j) * Nfp + l] * R.D[b][size_t(R.fmask[f][l]) * Np + R.fmask[f][j]];
        R.fc[b][f][j] = a;
      }
    }
  return R;
}

// Device copies of one precision's reference data (offsets in one buffer):
// D[3] (Np^2 each), B[3], M, Mf[4] (Nfp^2 each), dS[6] (Np each), dM (Np), fc[3][4] (Nfp each).
struct OpsLayout {
  int D[3], B[3], M, Mf[4], dS[6], dM, fc[3][4], total;
};
OpsLayout ops_layout(int Np, int Nfp) {
  OpsLayout L{};
  int o = 0;
  for (int b = 0; b < 3; ++b) L.D[b] = o, o += Np * Np;
  for (int b = 0; b < 3; ++b) L.B[b] = o, o += Np * Np;
  L.M = o, o += Np * Np;
  for (int f = 0; f < 4; ++f) L.Mf[f] = o, o += Nfp * Nfp;
  for (int q = 0; q < 6; ++q) L.dS[q] = o, o += Np;
  L.dM = o, o += Np;
  for (int b = 0; b < 3; ++b)
    for (int f = 0; f < 4; ++f) L.fc[b][f] = o, o += Nfp;
  L.total = o;
  return L;
}

// Geometry per element, kGeo words: J, G (rr, rs, rt, ss, st, tt), then per face
// f at 7 + 8 f: n.grad r_b of the element (3), n.grad r_b of the neighbour (3, the
// element's outward n), sJ (physical over reference face area), tau.
constexpr int kGeo = 40;

}  // namespace tet
}  // namespace dgx

struct dg_tet_mesh {
  int N = 0, Np = 0, Nfp = 0;
  int64_t K = 0;
  dgx::tet::TetRef ref;
  dgx::tet::OpsLayout L{};
  double* ops64 = nullptr;
  float* ops32 = nullptr;
  int* fmask = nullptr;    // [4][Nfp]
  double* geo64 = nullptr;  // [K][kGeo]
  float* geo32 = nullptr;
  int* conn = nullptr;     // [K][4]: neighbour element, or -1 - boundary tag
  int* mapJ = nullptr;     // [K][4 Nfp]: the neighbour's face-node slot f2 Nfp + j2 at face node (f, j)
  int* nfs = nullptr;      // [Np][3]: the face-node slots f Nfp + j at volume node i (-1 padded)
  double* xyz = nullptr;   // [3][K][Np] node coordinates
  // Jacobi-PCG workspace (grown on demand)
  double* work = nullptr;
  size_t work_cap = 0;
  // apply scratch: w ([B K][3][Np]) and face traces ([B K][4 Nfp][2]), grown on demand
  mutable void* ascr = nullptr;
  mutable size_t ascr_bytes = 0;
  // FP64 products on the tensor cores: [Dr; Ds; Dt], M, [Dr^T Ds^T Dt^T] (built at setup),
  // and their scratch (grown on demand)
  dgx::Tc64Op t64_grad, t64_mass, t64_out, t64_face[4];
  // every reference face's mass is face_ratio[f] times face 0's (the faces list their
  // nodes in one pattern): one face-mass product over all faces, scaled afterwards
  bool face_shared = false;
  double face_ratio[4] = {1.0, 1.0, 1.0, 1.0};
  mutable double* t64scr = nullptr;
  mutable size_t t64scr_bytes = 0;
};

namespace dgx {
namespace tet {

// Compile-time sizes of the degree-N apply: a block of kTetThreads threads
// handles EB elements, kR per thread in the node stages (each operator entry
// read from shared memory serves kR elements).
constexpr int kTetThreads = 256;
constexpr int kR = 2;
template <int N>
struct TetDims {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NF = 4 * Nfp;                  // face nodes of an element
  static constexpr int GS = kTetThreads / Np;         // element slots in the node stages
  static constexpr int EB = GS * kR;                  // elements per block iteration
};

// Shared-memory words of each kernel (operators, then per-element buffers).
template <int N>
constexpr int tet_grad_words() {
  using D = TetDims<N>;
  return 3 * D::Np * D::Np + D::EB * 4 * D::Np;
}
template <int N>
constexpr int tet_lift_words() {
  using D = TetDims<N>;
  return 4 * D::Np * D::Np + 4 * D::Nfp * D::Nfp + D::EB * (7 * D::Np + 4 * D::NF);
}

// The mesh element of batch row g, from the element e0 = be0 mod K of the
// batch's first row: subtractions only (rows past K wrap to the next
// right-hand side), no 64-bit division in the per-item loops.
__device__ __forceinline__ int64_t tet_elem(int64_t e0, int g, int64_t K) {
  int64_t e = e0 + g;
  while (e >= K) e -= K;
  return e;
}

// First kernel of the apply: per element the reference gradient ub_b = D_b u at
// every node, then (a) w_a = sum_b G_ab ub_b ([nE][3][Np]) and (b) the face
// traces (u, n.grad u) at the element's face nodes with its own outward normal
// ([nE][4 Nfp][2]), which the element and its neighbours read in the second kernel.
template <typename T, int N>
__global__ void __launch_bounds__(kTetThreads) tet_grad(int64_t K, int64_t nE, OpsLayout L, const T* __restrict__ ops,
                                                        const int* __restrict__ fmask, const T* __restrict__ geo,
                                                        const T* __restrict__ u, T* __restrict__ w,
                                                        T* __restrict__ tr) {
  using D = TetDims<N>;
  constexpr int Np = D::Np, NF = D::NF, EB = D::EB, GS = D::GS;
  extern __shared__ __align__(16) unsigned char tet_smem[];
  T* sDT = reinterpret_cast<T*>(tet_smem);  // [3][m][i] = D_b[i][m]
  T* su = sDT + 3 * Np * Np;                // [EB][Np]
  T* sub = su + EB * Np;                    // [EB][3][Np]
  for (int q = threadIdx.x; q < 3 * Np * Np; q += kTetThreads) {
    const int b = q / (Np * Np), r = q - b * Np * Np, m = r / Np, i = r - m * Np;
    sDT[q] = ops[L.D[b] + i * Np + m];
  }
  const int slot = threadIdx.x / Np, i = threadIdx.x - slot * Np;
  const int64_t stride = int64_t(gridDim.x) * EB, strideK = stride % K;
  int64_t e0 = (int64_t(blockIdx.x) * EB) % K;  // be0 mod K, advanced with be0
  for (int64_t be0 = int64_t(blockIdx.x) * EB; be0 < nE; be0 += stride, e0 = e0 + strideK < K ? e0 + strideK : e0 + strideK - K) {
    const int nv = int(nE - be0 < EB ? nE - be0 : EB);
    __syncthreads();
    for (int q = threadIdx.x; q < nv * Np; q += kTetThreads) su[q] = u[be0 * Np + q];
    __syncthreads();
    if (slot < GS) {
      T acc[kR][3];
#pragma unroll
      for (int r = 0; r < kR; ++r) acc[r][0] = acc[r][1] = acc[r][2] = T(0);
#pragma unroll 4
      for (int m = 0; m < Np; ++m) {
        const T d0 = sDT[m * Np + i], d1 = sDT[Np * Np + m * Np + i], d2 = sDT[2 * Np * Np + m * Np + i];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          const T um = su[(slot + GS * r) * Np + m];
          acc[r][0] += d0 * um;
          acc[r][1] += d1 * um;
          acc[r][2] += d2 * um;
        }
      }
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int g = slot + GS * r;
        if (g >= nv) continue;
        const int64_t be = be0 + g, e = tet_elem(e0, g, K);
        const T* G = geo + e * kGeo + 1;  // rr rs rt ss st tt
        sub[(g * 3 + 0) * Np + i] = acc[r][0];
        sub[(g * 3 + 1) * Np + i] = acc[r][1];
        sub[(g * 3 + 2) * Np + i] = acc[r][2];
        T* wo = w + be * 3 * Np;
        wo[i] = G[0] * acc[r][0] + G[1] * acc[r][1] + G[2] * acc[r][2];
        wo[Np + i] = G[1] * acc[r][0] + G[3] * acc[r][1] + G[4] * acc[r][2];
        wo[2 * Np + i] = G[2] * acc[r][0] + G[4] * acc[r][1] + G[5] * acc[r][2];
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv * NF; q += kTetThreads) {
      const int g = q / NF, fj = q - g * NF, f = fj / D::Nfp;
      const int k = fmask[fj];
      const int64_t e = tet_elem(e0, g, K);
      const T* nr = geo + e * kGeo + 7 + 8 * f;
      const T* ub = sub + g * 3 * Np;
      T* t2 = tr + ((be0 + g) * NF + fj) * 2;
      t2[0] = su[g * Np + k];
      t2[1] = nr[0] * ub[k] + nr[1] * ub[Np + k] + nr[2] * ub[2 * Np + k];
    }
  }
}

// Second kernel of the apply: per element the face jumps and averages from the
// traces (own and neighbour's), the face-mass products F1 = -sJ Mf (avg + tau jump)
// and F2 = sJ Mf jump / 2, then per node
//   z_b = J M w_b + y_b,  y_b[k] = sum over the face nodes (f, j) at node k of nr_fb F2_fj,
//   (A u)_i = sum_b (D_b^T z_b)_i + sum over (f, j) at node i of F1_fj [+ lambda J (M u)_i]
// (B_b = D_b^T M, so the volume term and the lift of the jump share one product).
template <typename T, int N, bool HELM>
__global__ void __launch_bounds__(kTetThreads) tet_lift(int64_t K, int64_t nE, OpsLayout L, const T* __restrict__ ops,
                                                        const int* __restrict__ nfs, const T* __restrict__ geo,
                                                        const int* __restrict__ conn, const int* __restrict__ mapJ,
                                                        T lambda, const T* __restrict__ u, const T* __restrict__ w,
                                                        const T* __restrict__ tr, T* __restrict__ Au) {
  using D = TetDims<N>;
  constexpr int Np = D::Np, Nfp = D::Nfp, NF = D::NF, EB = D::EB, GS = D::GS;
  extern __shared__ __align__(16) unsigned char tet_smem[];
  T* sD = reinterpret_cast<T*>(tet_smem);  // [3][m][i] = D_b[m][i]
  T* sM = sD + 3 * Np * Np;                 // [m][i]
  T* sMf = sM + Np * Np;                    // [4][l][j]
  T* su = sMf + 4 * Nfp * Nfp;              // [EB][Np]
  T* sw = su + EB * Np;                     // [EB][3][Np]
  T* sz = sw + EB * 3 * Np;                 // [EB][3][Np]
  T* sJm = sz + EB * 3 * Np;                // [EB][NF]
  T* sAv = sJm + EB * NF;
  T* sF1 = sAv + EB * NF;
  T* sF2 = sF1 + EB * NF;
  for (int q = threadIdx.x; q < 3 * Np * Np; q += kTetThreads) {
    const int b = q / (Np * Np);
    sD[q] = ops[L.D[b] + (q - b * Np * Np)];
  }
  for (int q = threadIdx.x; q < Np * Np; q += kTetThreads) sM[q] = ops[L.M + q];
  for (int q = threadIdx.x; q < 4 * Nfp * Nfp; q += kTetThreads) {
    const int f = q / (Nfp * Nfp);
    sMf[q] = ops[L.Mf[f] + (q - f * Nfp * Nfp)];
  }
  const int slot = threadIdx.x / Np, i = threadIdx.x - slot * Np;
  const int64_t stride = int64_t(gridDim.x) * EB, strideK = stride % K;
  int64_t e0 = (int64_t(blockIdx.x) * EB) % K;  // be0 mod K, advanced with be0
  for (int64_t be0 = int64_t(blockIdx.x) * EB; be0 < nE; be0 += stride, e0 = e0 + strideK < K ? e0 + strideK : e0 + strideK - K) {
    const int nv = int(nE - be0 < EB ? nE - be0 : EB);
    __syncthreads();
    if (HELM)
      for (int q = threadIdx.x; q < nv * Np; q += kTetThreads) su[q] = u[be0 * Np + q];
    for (int q = threadIdx.x; q < nv * 3 * Np; q += kTetThreads) sw[q] = w[be0 * 3 * Np + q];
    for (int q = threadIdx.x; q < nv * NF; q += kTetThreads) {  // jumps and averages
      const int g = q / NF, fj = q - g * NF, f = fj / Nfp;
      const int64_t be = be0 + g, e = tet_elem(e0, g, K);
      const int c = conn[4 * e + f];
      const T* own = tr + (be * NF + fj) * 2;
      T jm = T(0), av = T(0);
      if (c >= 0) {
        const T* nb = tr + ((be - e + c) * NF + mapJ[e * NF + fj]) * 2;
        jm = nb[0] - own[0];
        av = T(0.5) * (own[1] - nb[1]);  // the neighbour's trace carries its own (opposite) normal
      } else if (c == -2) {              // Dirichlet ghost: u+ = -u-, grad u+ = grad u-
        jm = T(-2) * own[0];
        av = own[1];
      }
      sJm[g * NF + fj] = jm;
      sAv[g * NF + fj] = av;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nv * NF; q += kTetThreads) {  // face-mass products
      const int g = q / NF, fj = q - g * NF, f = fj / Nfp, j = fj - f * Nfp;
      const int64_t e = tet_elem(e0, g, K);
      const T* gf = geo + e * kGeo + 7 + 8 * f;
      const T sJ = gf[6], tau = gf[7];
      const T* Mf = sMf + f * Nfp * Nfp;
      const T* jf = sJm + g * NF + f * Nfp;
      const T* af = sAv + g * NF + f * Nfp;
      T m1 = T(0), m2 = T(0);
#pragma unroll 4
      for (int l = 0; l < Nfp; ++l) {
        const T mf = Mf[l * Nfp + j];
        m1 += mf * (af[l] + tau * jf[l]);
        m2 += mf * jf[l];
      }
      sF1[g * NF + fj] = -sJ * m1;
      sF2[g * NF + fj] = T(0.5) * sJ * m2;
    }
    __syncthreads();
    T extra[kR] = {};
    if (slot < GS) {
      T z[kR][3], h[kR];
#pragma unroll
      for (int r = 0; r < kR; ++r) z[r][0] = z[r][1] = z[r][2] = h[r] = T(0);
#pragma unroll 4
      for (int m = 0; m < Np; ++m) {
        const T mv = sM[m * Np + i];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          const T* wg = sw + (slot + GS * r) * 3 * Np;
          z[r][0] += mv * wg[m];
          z[r][1] += mv * wg[Np + m];
          z[r][2] += mv * wg[2 * Np + m];
          if (HELM) h[r] += mv * su[(slot + GS * r) * Np + m];
        }
      }
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int g = slot + GS * r;
        extra[r] = T(0);
        if (g >= nv) continue;
        const int64_t e = tet_elem(e0, g, K);
        const T* ge = geo + e * kGeo;
        const T J = ge[0];
        T y0 = T(0), y1 = T(0), y2 = T(0), f1 = T(0);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const int fj = nfs[i * 3 + s];
          if (fj < 0) continue;
          const T* nr = ge + 7 + 8 * (fj / Nfp);
          const T F2 = sF2[g * NF + fj];
          y0 += nr[0] * F2;
          y1 += nr[1] * F2;
          y2 += nr[2] * F2;
          f1 += sF1[g * NF + fj];
        }
        T* zg = sz + g * 3 * Np;
        zg[i] = J * z[r][0] + y0;
        zg[Np + i] = J * z[r][1] + y1;
        zg[2 * Np + i] = J * z[r][2] + y2;
        extra[r] = HELM ? f1 + lambda * J * h[r] : f1;
      }
    }
    __syncthreads();
    if (slot < GS) {
      T o[kR];
#pragma unroll
      for (int r = 0; r < kR; ++r) o[r] = T(0);
#pragma unroll 4
      for (int m = 0; m < Np; ++m) {
        const T d0 = sD[m * Np + i], d1 = sD[Np * Np + m * Np + i], d2 = sD[2 * Np * Np + m * Np + i];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          const T* zg = sz + (slot + GS * r) * 3 * Np;
          o[r] += d0 * zg[m] + d1 * zg[Np + m] + d2 * zg[2 * Np + m];
        }
      }
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int g = slot + GS * r;
        if (g < nv) Au[(be0 + g) * Np + i] = o[r] + extra[r];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 apply with its dense products on the tensor cores (exactly sliced FP64
// GEMMs, out[r] = A X[r]): UB = [Dr; Ds; Dt] u, FM_f = diag(Mf_f, Mf_f) [avg +
// tau jump | jump] per local face f, MW = M [J w_0; J w_1; J w_2; lambda J u] and
// Au += [Dr^T Ds^T Dt^T] z, with the pointwise stages between them on CUDA cores:
//   tet64_point1: W = J G UB (and lambda J u), face traces (u, n.grad u);
//   tet64_jumps:  jumps and averages from the element's and the neighbours' traces;
//   tet64_point2: F1 = -sJ FM, F2 = sJ FM / 2; z_b = MW_b + y_b (y_b the lifted F2),
//                 Au = sum of F1 at the node [+ lambda J M u], which the last
//                 product adds D_b^T z_b to.
// The same operator as tet_grad / tet_lift, with the FP64 products no longer on
// the FP64 pipe.
// exponent e with |v| < 2^e (-1100 for zero and subnormals), the row bound the
// sliced products take
__device__ __forceinline__ int exp_bound(double v) {
  const int E = int((__double_as_longlong(v) >> 52) & 0x7ff);
  return E == 0 ? -1100 : E - 1022;
}

// The largest exponent over the lanes of the warp that share `key` (lanes of one
// row), which the lowest of them adds to ex[row] by an atomic maximum; ex starts
// below every exponent, so each row ends at its exact bound.
__device__ __forceinline__ void row_exp_max(int* ex, int64_t row, unsigned peers, int v) {
  const int m = __reduce_max_sync(peers, v);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(ex + row, m);
}

template <int N>
__global__ void __launch_bounds__(256) tet64_point1(int64_t K, int64_t nE, int R4, double lambda,
                                                    const int* __restrict__ fmask, const double* __restrict__ geo,
                                                    const double* __restrict__ u, const double* __restrict__ UB,
                                                    double* __restrict__ W, int* __restrict__ exW,
                                                    double2* __restrict__ tr) {
  constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2, NF = 4 * Nfp;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nE * Np; q += stride) {
    const int64_t be = q / Np, e = be < K ? be : be % K;
    const int i = int(q - be * Np);
    const double* g = geo + e * kGeo;
    const double J = g[0];
    const double* ub = UB + be * 3 * Np;
    const double a0 = ub[i], a1 = ub[Np + i], a2 = ub[2 * Np + i];
    double* wo = W + be * R4 * Np;
    const double w0 = J * (g[1] * a0 + g[2] * a1 + g[3] * a2);
    const double w1 = J * (g[2] * a0 + g[4] * a1 + g[5] * a2);
    const double w2 = J * (g[3] * a0 + g[5] * a1 + g[6] * a2);
    wo[i] = w0;
    wo[Np + i] = w1;
    wo[2 * Np + i] = w2;
    const unsigned peers = __match_any_sync(__activemask(), static_cast<unsigned long long>(be));
    row_exp_max(exW, be * R4, peers, exp_bound(w0));
    row_exp_max(exW, be * R4 + 1, peers, exp_bound(w1));
    row_exp_max(exW, be * R4 + 2, peers, exp_bound(w2));
    if (R4 == 4) {
      const double w3 = lambda * J * u[q];
      wo[3 * Np + i] = w3;
      row_exp_max(exW, be * R4 + 3, peers, exp_bound(w3));
    }
  }
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nE * NF; q += stride) {
    const int64_t be = q / NF, e = be < K ? be : be % K;
    const int fj = int(q - be * NF), k = fmask[fj];
    const double* nr = geo + e * kGeo + 7 + 8 * (fj / Nfp);
    const double* ub = UB + be * 3 * Np;
    tr[q] = make_double2(u[be * Np + k], nr[0] * ub[k] + nr[1] * ub[Np + k] + nr[2] * ub[2 * Np + k]);
  }
}

// Per element and face: the rows [avg + tau jump | jump] at the face nodes
// ([nE][4][2 Nfp]) that the face-mass products take.
template <int N>
__global__ void __launch_bounds__(256) tet64_jumps(int64_t K, int64_t nE, const double* __restrict__ geo,
                                                   const int* __restrict__ conn, const int* __restrict__ mapJ,
                                                   const double2* __restrict__ tr, double* __restrict__ XF,
                                                   int* __restrict__ exF) {
  constexpr int Nfp = (N + 1) * (N + 2) / 2, NF = 4 * Nfp;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nE * NF; q += stride) {
    const int64_t be = q / NF, e = be < K ? be : be % K;
    const int fj = int(q - be * NF), f = fj / Nfp, j = fj - f * Nfp;
    const int c = conn[4 * e + f];
    const double2 own = tr[q];
    double jm = 0.0, av = 0.0;
    if (c >= 0) {
      const double2 nb = tr[(be - e + c) * NF + mapJ[e * NF + fj]];
      jm = nb.x - own.x;
      av = 0.5 * (own.y - nb.y);  // the neighbour's trace carries its own (opposite) normal
    } else if (c == -2) {         // Dirichlet ghost: u+ = -u-, grad u+ = grad u-
      jm = -2.0 * own.x;
      av = own.y;
    }
    const double tau = geo[e * kGeo + 7 + 8 * f + 7];
    double* x = XF + (be * 4 + f) * 2 * Nfp;
    const double v1 = av + tau * jm;
    x[j] = v1;
    x[Nfp + j] = jm;
    const int64_t row = be * 4 + f;
    const unsigned peers = __match_any_sync(__activemask(), static_cast<unsigned long long>(row));
    row_exp_max(exF, row, peers, max(exp_bound(v1), exp_bound(jm)));
  }
}

// FM ([nE][4][2 Nfp]): the face-mass products Mf [avg + tau jump | jump] per face
// (with face 0's matrix for every face when they share it, fr[f] the area ratio);
// F1 = -sJ fr[f] FM[f][j], F2 = sJ fr[f] FM[f][Nfp + j] / 2.
struct FaceRatio {
  double r[4];
};
template <int N>
__global__ void __launch_bounds__(256) tet64_point2(int64_t K, int64_t nE, int R4, const int* __restrict__ nfs,
                                                    const double* __restrict__ geo, const double* __restrict__ FM,
                                                    FaceRatio fr, double* __restrict__ MW, int* __restrict__ exZ,
                                                    double* __restrict__ Au) {
  constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2, NF = 4 * Nfp;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nE * Np; q += stride) {
    const int64_t be = q / Np, e = be < K ? be : be % K;
    const int i = int(q - be * Np);
    const double* ge = geo + e * kGeo;
    const double* fm = FM + be * 2 * NF;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0, f1 = 0.0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int fj = nfs[i * 3 + s];
      if (fj < 0) continue;
      const int f = fj / Nfp, j = fj - f * Nfp;
      const double* gf = ge + 7 + 8 * f;
      const double sJ = gf[6] * fr.r[f];
      const double F2 = 0.5 * sJ * fm[f * 2 * Nfp + Nfp + j];
      y0 += gf[0] * F2;
      y1 += gf[1] * F2;
      y2 += gf[2] * F2;
      f1 -= sJ * fm[f * 2 * Nfp + j];
    }
    double* mw = MW + be * R4 * Np;
    const double z0 = mw[i] + y0, z1 = mw[Np + i] + y1, z2 = mw[2 * Np + i] + y2;
    mw[i] = z0;
    mw[Np + i] = z1;
    mw[2 * Np + i] = z2;
    Au[q] = R4 == 4 ? f1 + mw[3 * Np + i] : f1;
    const unsigned peers = __match_any_sync(__activemask(), static_cast<unsigned long long>(be));
    row_exp_max(exZ, be, peers, max(exp_bound(z0), max(exp_bound(z1), exp_bound(z2))));
  }
}

// diag(A) per node of one right-hand side ([K][Np], FP64).
__global__ void tet_diag(int N, int64_t K, OpsLayout L, const double* __restrict__ ops, const int* __restrict__ fmask,
                         const double* __restrict__ geo, const int* __restrict__ conn, double lambda,
                         double* __restrict__ diag) {
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= K * Np) return;
  const int64_t e = idx / Np;
  const int i = int(idx - e * Np);
  const double* g = geo + e * kGeo;
  const double J = g[0];
  const double c[6] = {1, 2, 2, 1, 2, 1};
  double d = 0.0;
  for (int q = 0; q < 6; ++q) d += c[q] * g[1 + q] * ops[L.dS[q] + i];
  d = J * d + lambda * J * ops[L.dM + i];
  for (int f = 0; f < 4; ++f) {
    const int cf = conn[4 * e + f];
    if (!(cf >= 0 || cf == -2)) continue;
    const double w = cf >= 0 ? 1.0 : 2.0;
    const double* gf = g + 7 + 8 * f;
    for (int j = 0; j < Nfp; ++j) {
      if (fmask[f * Nfp + j] != i) continue;
      const double a1 = gf[6] * (gf[0] * ops[L.fc[0][f] + j] + gf[1] * ops[L.fc[1][f] + j] + gf[2] * ops[L.fc[2][f] + j]);
      const double a2 = gf[6] * ops[L.Mf[f] + j * Nfp + j];
      d += w * (-a1 + gf[7] * a2);
    }
  }
  diag[idx] = d;
}

// b = J M f - L(g) for B right-hand sides: L(g)_i = sum over Dirichlet faces of
// (n.grad l_i, g) - 2 tau (l_i, g), g the nodal trace.
__global__ void tet_rhs(int N, int64_t K, int64_t nE, OpsLayout L, const double* __restrict__ ops,
                        const int* __restrict__ fmask, const double* __restrict__ geo, const int* __restrict__ conn,
                        const double* __restrict__ f, const double* __restrict__ gd, double* __restrict__ b) {
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= nE * Np) return;
  const int64_t be = idx / Np;
  const int i = int(idx - be * Np);
  const int64_t e = be % K;
  const double* g = geo + e * kGeo;
  double o = 0.0;
  for (int m = 0; m < Np; ++m) o += ops[L.M + i * Np + m] * f[be * Np + m];
  o *= g[0];
  for (int fc = 0; fc < 4; ++fc) {
    if (conn[4 * e + fc] != -2) continue;
    const double* gf = g + 7 + 8 * fc;
    for (int j = 0; j < Nfp; ++j) {  // (Mf g)_j, then its two uses
      double mg = 0.0;
      for (int l = 0; l < Nfp; ++l) mg += ops[L.Mf[fc] + j * Nfp + l] * gd[be * Np + fmask[fc * Nfp + l]];
      mg *= gf[6];
      const int k = fmask[fc * Nfp + j];
      const double dn = gf[0] * ops[L.D[0] + k * Np + i] + gf[1] * ops[L.D[1] + k * Np + i] +
                        gf[2] * ops[L.D[2] + k * Np + i];
      o -= dn * mg;
      if (k == i) o += 2.0 * gf[7] * mg;
    }
  }
  b[idx] = o;
}

// --- Jacobi-PCG vector kernels ([B][n] vectors, fixed-order reductions)
constexpr int kRB = 256;  // reduction blocks per right-hand side

__global__ void k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                       double* __restrict__ partial) {
  __shared__ double sh[256];
  const int rhs = blockIdx.y;
  const double* x = a + int64_t(rhs) * n;
  const double* y = b + int64_t(rhs) * n;
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    s += x[i] * y[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[rhs * kRB + blockIdx.x] = sh[0];
}
__global__ void k_sum(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[kRB];
  sh[threadIdx.x] = partial[blockIdx.x * kRB + threadIdx.x];
  __syncthreads();
  for (int w = kRB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}
// y[rhs] = a[rhs] * x[rhs] + y[rhs] (coefficients per right-hand side, device)
__global__ void k_axpy(int64_t n, int B, const double* __restrict__ coef, int sign, const double* __restrict__ x,
                       double* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * B; i += int64_t(gridDim.x) * blockDim.x) {
    const double a = coef[i / n];
    y[i] += sign * a * x[i];
  }
}
// p = z + beta p
__global__ void k_xpay(int64_t n, int B, const double* __restrict__ beta, const double* __restrict__ z,
                       double* __restrict__ p) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * B; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = z[i] + beta[i / n] * p[i];
}
// z = dinv r (dinv shared by the right-hand sides); r = b - Ax when ax is given
__global__ void k_jac(int64_t n, int B, const double* __restrict__ dinv, const double* __restrict__ b,
                      const double* __restrict__ ax, double* __restrict__ r, double* __restrict__ z) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * B; i += int64_t(gridDim.x) * blockDim.x) {
    const double ri = ax ? b[i] - ax[i] : r[i];
    r[i] = ri;
    z[i] = dinv[i % n] * ri;
  }
}
__global__ void k_recip(int64_t n, double* __restrict__ d) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    d[i] = 1.0 / d[i];
}
inline unsigned grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16)));
}

}  // namespace tet
}  // namespace dgx

namespace dgx {
namespace tet {

dg_status fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace tet
}  // namespace dgx

using namespace dgx;
using namespace dgx::tet;

namespace {
// Per-instantiation launch data: the dynamic shared-memory limit raised once per
// device, and the resident blocks per SM at the kernel's shared-memory size.
struct TetKernelInfo {
  std::atomic<uint64_t> ready{0};
  std::atomic<int> occ{1};
};

template <typename Kern>
cudaError_t tet_prepare(Kern k, size_t smem, TetKernelInfo& info, int dev, int* occ) {
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(info.ready.load() & bit)) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int o = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, kTetThreads, smem);
    if (e != cudaSuccess) return e;
    info.occ.store(o > 0 ? o : 1);
    info.ready.fetch_or(bit);
  }
  *occ = info.occ.load();
  return cudaSuccess;
}

template <typename T, int N, bool HELM>
cudaError_t tet_apply_n(const dg_tet_mesh* m, int64_t nE, T lambda, const T* ops, const T* geo, const T* u, T* Au,
                        T* w, T* tr, cudaStream_t st) {
  static TetKernelInfo info_g, info_l;
  const size_t sg = size_t(tet_grad_words<N>()) * sizeof(T), sl = size_t(tet_lift_words<N>()) * sizeof(T);
  int dev = 0, sms = 0, og = 1, ol = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = tet_prepare(tet_grad<T, N>, sg, info_g, dev, &og);
  if (e == cudaSuccess) e = tet_prepare(tet_lift<T, N, HELM>, sl, info_l, dev, &ol);
  if (e != cudaSuccess) return e;
  // one resident wave of blocks, each loading the operators once and striding over element batches
  const int64_t batches = (nE + TetDims<N>::EB - 1) / TetDims<N>::EB;
  const unsigned gg = unsigned(std::min<int64_t>(batches, int64_t(sms) * og));
  const unsigned gl = unsigned(std::min<int64_t>(batches, int64_t(sms) * ol));
  tet_grad<T, N><<<gg, kTetThreads, sg, st>>>(m->K, nE, m->L, ops, m->fmask, geo, u, w, tr);
  note_launch();
  tet_lift<T, N, HELM><<<gl, kTetThreads, sl, st>>>(m->K, nE, m->L, ops, m->nfs, geo, m->conn, m->mapJ, lambda, u, w,
                                                    tr, Au);
  note_launch();
  return cudaGetLastError();
}

template <int N>
cudaError_t tet64_tc_n(const dg_tet_mesh* m, int64_t nE, double lambda, const double* u, double* Au, cudaStream_t st) {
  constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2, NF = 4 * Nfp;
  const int R4 = lambda != 0.0 ? 4 : 3;
  auto even = [](size_t n) { return (n + 1) & ~size_t(1); };  // keeps the traces 16-byte aligned
  const size_t nUB = even(size_t(nE) * 3 * Np), nW = even(size_t(nE) * R4 * Np);
  const size_t nEx = even((size_t(nE) * (R4 + 4 + 1) + 1) / 2);  // row exponents (ints), in doubles
  const size_t words = nUB + 2 * nW + size_t(nE) * NF * 2 + 2 * size_t(nE) * 2 * NF + nEx;
  if (m->t64scr_bytes < words * sizeof(double)) {
    cudaFree(m->t64scr);
    m->t64scr = nullptr;
    m->t64scr_bytes = 0;
    const cudaError_t e = cudaMalloc(&m->t64scr, words * sizeof(double));
    if (e != cudaSuccess) return e;
    m->t64scr_bytes = words * sizeof(double);
  }
  double* UB = m->t64scr;
  double* W = UB + nUB;
  double* MW = W + nW;
  double2* tr = reinterpret_cast<double2*>(MW + nW);
  double* XF = reinterpret_cast<double*>(tr + size_t(nE) * NF);  // [nE][4][2 Nfp]
  double* FM = XF + size_t(nE) * 2 * NF;
  int* exW = reinterpret_cast<int*>(FM + size_t(nE) * 2 * NF);  // [nE R4]
  int* exF = exW + size_t(nE) * R4;                              // [nE 4]
  int* exZ = exF + size_t(nE) * 4;                               // [nE]
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned gp = unsigned(std::min<int64_t>((nE * Np + 255) / 256, int64_t(sms) * 16));
  const unsigned gf = unsigned(std::min<int64_t>((nE * NF + 255) / 256, int64_t(sms) * 16));
  // row exponents start below every exponent (0x80808080); the producers raise them
  e = cudaMemsetAsync(exW, 0x80, size_t(nE) * (R4 + 4 + 1) * sizeof(int), st);
  if (e == cudaSuccess) e = tc64_gemm_launch(m->t64_grad, nE, u, Np, UB, 3 * Np, st);
  if (e != cudaSuccess) return e;
  tet64_point1<N><<<gp, 256, 0, st>>>(m->K, nE, R4, lambda, m->fmask, m->geo64, u, UB, W, exW, tr);
  note_launch();
  tet64_jumps<N><<<gf, 256, 0, st>>>(m->K, nE, m->geo64, m->conn, m->mapJ, tr, XF, exF);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (m->face_shared) {  // FM = diag(Mf_0, Mf_0) XF over the rows of all faces
    e = tc64_gemm_launch(m->t64_face[0], nE * 4, XF, 2 * Nfp, FM, 2 * Nfp, st, 0, exF);
  } else {
    for (int f = 0; f < 4 && e == cudaSuccess; ++f)  // FM[f] = diag(Mf, Mf) XF[f], the rows of face f
      e = tc64_gemm_launch(m->t64_face[f], nE, XF + f * 2 * Nfp, 2 * NF, FM + f * 2 * Nfp, 2 * NF, st);
  }
  FaceRatio fr;
  for (int f = 0; f < 4; ++f) fr.r[f] = m->face_shared ? m->face_ratio[f] : 1.0;
  if (e == cudaSuccess) e = tc64_gemm_launch(m->t64_mass, nE * R4, W, Np, MW, Np, st, 0, exW);
  if (e != cudaSuccess) return e;
  tet64_point2<N><<<gp, 256, 0, st>>>(m->K, nE, R4, m->nfs, m->geo64, FM, fr, MW, exZ, Au);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return tc64_gemm_launch(m->t64_out, nE, MW, int64_t(R4) * Np, Au, Np, st, 1, exZ);
}

// FP64 on the tensor cores (the default) or, with pipe set, on the FP64 pipe.
cudaError_t tet64_apply(const dg_tet_mesh* m, int B, double lambda, const double* u, double* Au, bool pipe,
                        cudaStream_t st);

template <typename T>
cudaError_t tet_apply_launch(const dg_tet_mesh* m, int B, double lambda, const T* u, T* Au, cudaStream_t st) {
  const bool f64 = sizeof(T) == 8;
  const T* ops = f64 ? reinterpret_cast<const T*>(m->ops64) : reinterpret_cast<const T*>(m->ops32);
  const T* geo = f64 ? reinterpret_cast<const T*>(m->geo64) : reinterpret_cast<const T*>(m->geo32);
  const int64_t nE = int64_t(B) * m->K;
  const size_t need = size_t(nE) * size_t(3 * m->Np + 8 * m->Nfp) * sizeof(T);
  if (m->ascr_bytes < need) {
    cudaFree(m->ascr);
    m->ascr = nullptr;
    m->ascr_bytes = 0;
    const cudaError_t e = cudaMalloc(&m->ascr, need);
    if (e != cudaSuccess) return e;
    m->ascr_bytes = need;
  }
  T* w = static_cast<T*>(m->ascr);
  T* tr = w + nE * 3 * m->Np;
  const T lam = T(lambda);
  const bool helm = lambda != 0.0;
  switch (m->N) {
#define TET_CASE(NN)                                                                           \
  case NN:                                                                                     \
    return helm ? tet_apply_n<T, NN, true>(m, nE, lam, ops, geo, u, Au, w, tr, st)             \
                : tet_apply_n<T, NN, false>(m, nE, lam, ops, geo, u, Au, w, tr, st);
    TET_CASE(1)
    TET_CASE(2)
    TET_CASE(3)
    TET_CASE(4)
    TET_CASE(5)
#undef TET_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t tet64_apply(const dg_tet_mesh* m, int B, double lambda, const double* u, double* Au, bool pipe,
                        cudaStream_t st) {
  // at degrees 1 and 2 the products are too small for the tensor cores to pay
  // (196,608 elements, N = 1: 0.25 ms on the FP64 pipe against 0.54 ms)
  if (pipe || !m->t64_grad.blocks || m->N <= 2) return tet_apply_launch<double>(m, B, lambda, u, Au, st);
  const int64_t nE = int64_t(B) * m->K;
  switch (m->N) {
    case 1: return tet64_tc_n<1>(m, nE, lambda, u, Au, st);
    case 2: return tet64_tc_n<2>(m, nE, lambda, u, Au, st);
    case 3: return tet64_tc_n<3>(m, nE, lambda, u, Au, st);
    case 4: return tet64_tc_n<4>(m, nE, lambda, u, Au, st);
    case 5: return tet64_tc_n<5>(m, nE, lambda, u, Au, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

extern "C" {

dg_status dg_tet_mesh_destroy(dg_tet_mesh* m) {
  if (!m) return DG_OK;
  for (void* p : {static_cast<void*>(m->ops64), static_cast<void*>(m->ops32), static_cast<void*>(m->fmask),
                  static_cast<void*>(m->geo64), static_cast<void*>(m->geo32), static_cast<void*>(m->conn),
                  static_cast<void*>(m->mapJ), static_cast<void*>(m->nfs), static_cast<void*>(m->xyz),
                  static_cast<void*>(m->work), m->ascr, static_cast<void*>(m->t64scr)})
    cudaFree(p);
  tc64_op_free(&m->t64_grad);
  tc64_op_free(&m->t64_mass);
  tc64_op_free(&m->t64_out);
  for (dgx::Tc64Op& op : m->t64_face) tc64_op_free(&op);
  delete m;
  return DG_OK;
}

dg_status dg_tet_mesh_setup(int N, int64_t Nv, const double* VX, const double* VY, const double* VZ, int64_t K,
                            const int32_t* EToV, const int8_t* bc, void* stream, dg_tet_mesh** out) {
  (void)stream;
  if (!out || !VX || !VY || !VZ || !EToV || !bc) { set_error("NULL argument"); return DG_ERR_ARG; }
  *out = nullptr;
  if (N < 1 || N > kMaxTetN) { set_error("tetrahedral degree N must be in 1..5"); return DG_ERR_ARG; }
  if (K < 1 || Nv < 4 || K * np3(N) >= (int64_t(1) << 31)) { set_error("bad tetrahedral mesh size"); return DG_ERR_ARG; }
  for (int64_t i = 0; i < 4 * K; ++i)
    if (EToV[i] < 0 || EToV[i] >= Nv) { set_error("EToV index out of range"); return DG_ERR_MESH; }
  dg_tet_mesh* m = new dg_tet_mesh();
  try {
    m->N = N;
    m->K = K;
    m->ref = build_tet(N);
  } catch (const std::exception& ex) {
    delete m;
    set_error(ex.what());
    return DG_ERR_ARG;
  }
  const TetRef& R = m->ref;
  const int Np = R.Np, Nfp = R.Nfp;
  m->Np = Np;
  m->Nfp = Nfp;
  // element geometry
  std::vector<double> jinv(size_t(K) * 9), Jd(K), vol(K), nrm(size_t(K) * 12), area(size_t(K) * 4);
  for (int64_t e = 0; e < K; ++e) {
    double P[4][3];
    for (int v = 0; v < 4; ++v) {
      const int32_t g = EToV[4 * e + v];
      P[v][0] = VX[g], P[v][1] = VY[g], P[v][2] = VZ[g];
    }
    double A[3][3];  // columns x_r, x_s, x_t
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) A[d][c] = 0.5 * (P[c + 1][d] - P[0][d]);
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(det > 0)) {
      dg_tet_mesh_destroy(m);
      set_error("tetrahedron with non-positive Jacobian");
      return DG_ERR_MESH;
    }
    // inverse: rows grad r, grad s, grad t
    double* I = &jinv[size_t(e) * 9];
    I[0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    I[1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    I[2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    I[3] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    I[4] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    I[5] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    I[6] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    I[7] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    I[8] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    Jd[e] = det;
    vol[e] = det * 4.0 / 3.0;
    double cen[3] = {0, 0, 0};
    for (int v = 0; v < 4; ++v)
      for (int d = 0; d < 3; ++d) cen[d] += 0.25 * P[v][d];
    for (int f = 0; f < 4; ++f) {
      const double* a = P[kFaceVerts[f][0]];
      const double* b = P[kFaceVerts[f][1]];
      const double* c = P[kFaceVerts[f][2]];
      const double u1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, u2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double n[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
      const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int d = 0; d < 3; ++d) n[d] /= len;
      if (n[0] * (a[0] - cen[0]) + n[1] * (a[1] - cen[1]) + n[2] * (a[2] - cen[2]) < 0)
        for (int d = 0; d < 3; ++d) n[d] = -n[d];
      for (int d = 0; d < 3; ++d) nrm[size_t(e) * 12 + 3 * f + d] = n[d];
      area[size_t(e) * 4 + f] = 0.5 * len;
    }
  }
  // face connectivity by the sorted vertex triple
  std::vector<int> nbE(size_t(K) * 4, -1), nbF(size_t(K) * 4, -1);
  {
    std::map<std::array<int32_t, 3>, std::pair<int64_t, int>> open;
    for (int64_t e = 0; e < K; ++e)
      for (int f = 0; f < 4; ++f) {
        std::array<int32_t, 3> key = {EToV[4 * e + kFaceVerts[f][0]], EToV[4 * e + kFaceVerts[f][1]],
                                      EToV[4 * e + kFaceVerts[f][2]]};
        std::sort(key.begin(), key.end());
        auto it = open.find(key);
        if (it == open.end()) {
          open[key] = {e, f};
        } else {
          const int64_t e2 = it->second.first;
          const int f2 = it->second.second;
          nbE[4 * e + f] = int(e2), nbF[4 * e + f] = f2;
          nbE[4 * e2 + f2] = int(e), nbF[4 * e2 + f2] = f;
          open.erase(it);
        }
      }
  }
  std::vector<int> conn(size_t(K) * 4);
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 4; ++f) {
      if (nbE[4 * e + f] >= 0) {
        conn[4 * e + f] = nbE[4 * e + f];
      } else {
        const int tag = bc[4 * e + f];
        if (tag != 1 && tag != 2) {
          dg_tet_mesh_destroy(m);
          set_error("a face without a neighbour needs boundary tag 1 (Dirichlet) or 2 (Neumann)");
          return DG_ERR_MESH;
        }
        conn[4 * e + f] = -1 - tag;
      }
    }
  // node coordinates and the neighbour's node at each face node
  std::vector<double> xyz(size_t(3) * K * Np);
  for (int64_t e = 0; e < K; ++e) {
    const int32_t* ev = &EToV[4 * e];
    for (int k = 0; k < Np; ++k) {
      const double w[3] = {0.5 * (R.r[k] + 1.0), 0.5 * (R.s[k] + 1.0), 0.5 * (R.t[k] + 1.0)};
      const double* V[3] = {VX, VY, VZ};
      for (int d = 0; d < 3; ++d) {
        const double x0 = V[d][ev[0]];
        xyz[(size_t(d) * K + e) * Np + k] =
            x0 + w[0] * (V[d][ev[1]] - x0) + w[1] * (V[d][ev[2]] - x0) + w[2] * (V[d][ev[3]] - x0);
      }
    }
  }
  std::vector<int> mapJ(size_t(K) * 4 * Nfp, -1);
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 4; ++f) {
      const int e2 = nbE[4 * e + f], f2 = nbF[4 * e + f];
      if (e2 < 0) continue;
      const double hscale = std::cbrt(vol[e]);
      for (int j = 0; j < Nfp; ++j) {
        const int k = R.fmask[f][j];
        int best = -1, bestj = -1;
        for (int j2 = 0; j2 < Nfp; ++j2) {
          const int k2 = R.fmask[f2][j2];
          double d2 = 0.0;
          for (int d = 0; d < 3; ++d) {
            const double dx = xyz[(size_t(d) * K + e) * Np + k] - xyz[(size_t(d) * K + e2) * Np + k2];
            d2 += dx * dx;
          }
          if (std::sqrt(d2) < 1e-8 * hscale) best = k2, bestj = j2;
        }
        if (best < 0) {
          dg_tet_mesh_destroy(m);
          set_error("non-conforming tetrahedral faces (face nodes do not match)");
          return DG_ERR_MESH;
        }
        mapJ[(size_t(e) * 4 + f) * Nfp + j] = f2 * Nfp + bestj;
      }
    }
  // per-element geometry words
  const double cpen = double((N + 1) * (N + 3)) / 3.0;
  std::vector<double> geo(size_t(K) * kGeo, 0.0);
  for (int64_t e = 0; e < K; ++e) {
    double* g = &geo[size_t(e) * kGeo];
    const double* I = &jinv[size_t(e) * 9];
    g[0] = Jd[e];
    const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q)
      g[1 + q] = I[3 * pa[q]] * I[3 * pb[q]] + I[3 * pa[q] + 1] * I[3 * pb[q] + 1] + I[3 * pa[q] + 2] * I[3 * pb[q] + 2];
    for (int f = 0; f < 4; ++f) {
      double* gf = g + 7 + 8 * f;
      const double* n = &nrm[size_t(e) * 12 + 3 * f];
      for (int b = 0; b < 3; ++b) gf[b] = n[0] * I[3 * b] + n[1] * I[3 * b + 1] + n[2] * I[3 * b + 2];
      const int e2 = nbE[4 * e + f];
      if (e2 >= 0) {
        const double* I2 = &jinv[size_t(e2) * 9];
        for (int b = 0; b < 3; ++b) gf[3 + b] = n[0] * I2[3 * b] + n[1] * I2[3 * b + 1] + n[2] * I2[3 * b + 2];
      }
      gf[6] = area[size_t(e) * 4 + f] / R.face_area[f];
      double ih = area[size_t(e) * 4 + f] / vol[e];
      if (e2 >= 0) ih = std::max(ih, area[size_t(e2) * 4 + nbF[4 * e + f]] / vol[e2]);
      gf[7] = cpen * ih;
    }
  }
  // reference data, both precisions
  m->L = ops_layout(Np, Nfp);
  std::vector<double> ops(m->L.total, 0.0);
  for (int b = 0; b < 3; ++b) {
    std::copy(R.D[b].begin(), R.D[b].end(), ops.begin() + m->L.D[b]);
    std::copy(R.Bm[b].begin(), R.Bm[b].end(), ops.begin() + m->L.B[b]);
  }
  std::copy(R.M.begin(), R.M.end(), ops.begin() + m->L.M);
  for (int f = 0; f < 4; ++f) std::copy(R.Mf[f].begin(), R.Mf[f].end(), ops.begin() + m->L.Mf[f]);
  for (int q = 0; q < 6; ++q) std::copy(R.dS[q].begin(), R.dS[q].end(), ops.begin() + m->L.dS[q]);
  std::copy(R.dM.begin(), R.dM.end(), ops.begin() + m->L.dM);
  for (int b = 0; b < 3; ++b)
    for (int f = 0; f < 4; ++f) std::copy(R.fc[b][f].begin(), R.fc[b][f].end(), ops.begin() + m->L.fc[b][f]);
  std::vector<int> fm(size_t(4) * Nfp), nfs(size_t(Np) * 3, -1);
  for (int f = 0; f < 4; ++f)
    for (int j = 0; j < Nfp; ++j) {
      const int k = R.fmask[f][j];
      fm[size_t(f) * Nfp + j] = k;
      int s = 0;
      while (s < 3 && nfs[size_t(k) * 3 + s] >= 0) ++s;
      if (s == 3) {  // a node of a tetrahedron lies on at most three faces
        dg_tet_mesh_destroy(m);
        set_error("tetrahedron node on more than three faces");
        return DG_ERR_ARG;
      }
      nfs[size_t(k) * 3 + s] = f * Nfp + j;
    }
  const std::vector<float> ops32(ops.begin(), ops.end()), geo32(geo.begin(), geo.end());
  cudaError_t ce = upload(&m->ops64, ops);
  if (ce == cudaSuccess) ce = upload(&m->ops32, ops32);
  if (ce == cudaSuccess) ce = upload(&m->fmask, fm);
  if (ce == cudaSuccess) ce = upload(&m->geo64, geo);
  if (ce == cudaSuccess) ce = upload(&m->geo32, geo32);
  if (ce == cudaSuccess) ce = upload(&m->conn, conn);
  if (ce == cudaSuccess) ce = upload(&m->mapJ, mapJ);
  if (ce == cudaSuccess) ce = upload(&m->nfs, nfs);
  if (ce == cudaSuccess) ce = upload(&m->xyz, xyz);
  if (ce == cudaSuccess) {  // the FP64 tensor-core operators
    std::vector<double> A1(size_t(3) * Np * Np), A3(size_t(Np) * 3 * Np);
    for (int b = 0; b < 3; ++b)
      for (int i = 0; i < Np; ++i)
        for (int q = 0; q < Np; ++q) {
          A1[(size_t(b) * Np + i) * Np + q] = R.D[b][size_t(i) * Np + q];
          A3[size_t(i) * 3 * Np + size_t(b) * Np + q] = R.D[b][size_t(q) * Np + i];
        }
    ce = tc64_op_create(A1, 3 * Np, Np, &m->t64_grad);
    if (ce == cudaSuccess) ce = tc64_op_create(R.M, Np, Np, &m->t64_mass);
    if (ce == cudaSuccess) ce = tc64_op_create(A3, Np, 3 * Np, &m->t64_out);
    m->face_shared = true;
    for (int f = 0; f < 4; ++f) {
      m->face_ratio[f] = R.face_area[f] / R.face_area[0];
      double dmax = 0.0, amax = 0.0;
      for (size_t q = 0; q < R.Mf[f].size(); ++q) {
        dmax = std::max(dmax, std::fabs(R.Mf[f][q] - m->face_ratio[f] * R.Mf[0][q]));
        amax = std::max(amax, std::fabs(R.Mf[f][q]));
      }
      if (dmax > 1e-13 * amax) m->face_shared = false;
    }
    for (int f = 0; f < (m->face_shared ? 1 : 4) && ce == cudaSuccess; ++f) {  // diag(Mf, Mf) per reference face
      std::vector<double> A4(size_t(4) * Nfp * Nfp, 0.0);
      for (int j = 0; j < Nfp; ++j)
        for (int l = 0; l < Nfp; ++l) {
          A4[size_t(j) * 2 * Nfp + l] = R.Mf[f][size_t(j) * Nfp + l];
          A4[size_t(Nfp + j) * 2 * Nfp + Nfp + l] = R.Mf[f][size_t(j) * Nfp + l];
        }
      ce = tc64_op_create(A4, 2 * Nfp, 2 * Nfp, &m->t64_face[f]);
    }
  }
  if (ce != cudaSuccess) {
    dg_tet_mesh_destroy(m);
    return fail(ce, "dg_tet_mesh_setup");
  }
  *out = m;
  return DG_OK;
}

dg_status dg_tet_mesh_info(const dg_tet_mesh* m, int* N, int64_t* K, int* Np) {
  if (!m) { set_error("NULL mesh"); return DG_ERR_ARG; }
  if (N) *N = m->N;
  if (K) *K = m->K;
  if (Np) *Np = m->Np;
  return DG_OK;
}

dg_status dg_tet_mesh_nodes(const dg_tet_mesh* m, double* x, double* y, double* z, void* stream) {
  if (!m || !x || !y || !z) { set_error("NULL argument"); return DG_ERR_ARG; }
  const size_t n = size_t(m->K) * m->Np * sizeof(double);
  cudaStream_t st = (cudaStream_t)stream;
  double* dst[3] = {x, y, z};
  for (int d = 0; d < 3; ++d) {
    const cudaError_t e = cudaMemcpyAsync(dst[d], m->xyz + size_t(d) * m->K * m->Np, n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(e, "dg_tet_mesh_nodes");
  }
  return DG_OK;
}



dg_status dg_tet_apply(const dg_tet_mesh* m, dg_prec prec, int B, double lambda, const void* u, void* Au,
                       void* stream) {
  if (!m || !u || !Au) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (B < 1 || B > DG_MAX_BATCH) { set_error("batch must be in 1..64"); return DG_ERR_ARG; }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (prec == DG_F32)
    e = tet_apply_launch<float>(m, B, lambda, static_cast<const float*>(u), static_cast<float*>(Au), st);
  else if (prec == DG_F64 || prec == DG_F64_DFMA)
    e = tet64_apply(m, B, lambda, static_cast<const double*>(u), static_cast<double*>(Au), prec == DG_F64_DFMA, st);
  else {
    set_error("unknown precision");
    return DG_ERR_ARG;
  }
  return e == cudaSuccess ? DG_OK : fail(e, "dg_tet_apply");
}

dg_status dg_tet_rhs(const dg_tet_mesh* m, int B, const double* f, const double* g, double* b, void* stream) {
  if (!m || !f || !g || !b) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (B < 1 || B > DG_MAX_BATCH) { set_error("batch must be in 1..64"); return DG_ERR_ARG; }
  const int64_t nE = int64_t(B) * m->K, n = nE * m->Np;
  tet_rhs<<<unsigned((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(m->N, m->K, nE, m->L, m->ops64, m->fmask,
                                                                       m->geo64, m->conn, f, g, b);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : fail(e, "dg_tet_rhs");
}

dg_status dg_tet_pcg_jacobi_solve(dg_tet_mesh* m, int B, double lambda, double tol, int max_iter, const double* b,
                                  double* x, dg_solve_info* info, void* stream) {
  if (!m || !b || !x) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (B < 1 || B > DG_MAX_BATCH) { set_error("batch must be in 1..64"); return DG_ERR_ARG; }
  if (!(tol > 0.0) || max_iter < 0) { set_error("tol must be > 0 and max_iter >= 0"); return DG_ERR_ARG; }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = m->K * m->Np;
  const size_t nt = size_t(n) * B;
  // workspace: r, z, p, Ap (nt each), dinv (n), partials (B kRB), scalars (4 B)
  const size_t words = 4 * nt + size_t(n) + size_t(B) * kRB + 4 * size_t(B);
  if (m->work_cap < words) {
    cudaFree(m->work);
    m->work = nullptr;
    m->work_cap = 0;
    const cudaError_t e = cudaMalloc(&m->work, words * sizeof(double));
    if (e != cudaSuccess) return fail(e, "dg_tet_pcg_jacobi_solve");
    m->work_cap = words;
  }
  double *r = m->work, *z = r + nt, *p = z + nt, *Ap = p + nt, *dinv = Ap + nt, *part = dinv + n, *sc = part + size_t(B) * kRB;
  double* coefd = sc + B;  // B coefficients uploaded per step
  const dim3 rg(kRB, unsigned(B));
  const unsigned gv = grid_of(int64_t(nt)), gn = grid_of(n);
  std::vector<double> hb(B), hrz(B), hd(B), coef(B), active(B, 1.0);
  auto dot = [&](const double* a, const double* c, double* host) -> cudaError_t {
    k_dot2<<<rg, 256, 0, st>>>(n, a, c, part); note_launch();
    k_sum<<<unsigned(B), kRB, 0, st>>>(part, sc); note_launch();
    cudaError_t e = cudaMemcpyAsync(host, sc, sizeof(double) * B, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  };
  auto setc = [&](const std::vector<double>& c) {
    return cudaMemcpyAsync(coefd, c.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st);
  };
#define TCK(expr)                                          \
  do {                                                     \
    const cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return fail(e_, "dg_tet_pcg_jacobi_solve"); \
  } while (0)
  tet_diag<<<unsigned((n + 255) / 256), 256, 0, st>>>(m->N, m->K, m->L, m->ops64, m->fmask, m->geo64, m->conn, lambda,
                                                      dinv);
  note_launch();
  k_recip<<<gn, 256, 0, st>>>(n, dinv); note_launch();
  TCK(tet64_apply(m, B, lambda, x, Ap, false, st));
  k_jac<<<gv, 256, 0, st>>>(n, B, dinv, b, Ap, r, z); note_launch();
  TCK(cudaMemcpyAsync(p, z, nt * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TCK(dot(b, b, hb.data()));
  std::vector<double> hrr(B);
  TCK(dot(r, r, hrr.data()));
  TCK(dot(r, z, hrz.data()));
  for (int k = 0; k < B; ++k) {
    hb[k] = std::sqrt(hb[k]);
    if (hb[k] == 0.0 || std::sqrt(hrr[k]) <= tol * hb[k]) active[k] = 0.0;
  }
  int it = 0;
  dg_status status = DG_OK;
  std::vector<int> iters(B, 0);
  auto any_active = [&]() {
    for (int k = 0; k < B; ++k)
      if (active[k] != 0.0) return true;
    return false;
  };
  while (any_active() && it < max_iter) {
    TCK(tet64_apply(m, B, lambda, p, Ap, false, st));
    TCK(dot(p, Ap, hd.data()));
    for (int k = 0; k < B; ++k) {
      if (active[k] != 0.0 && !(hd[k] > 0.0)) {
        status = DG_ERR_BREAKDOWN;
        active[k] = 0.0;
      }
      coef[k] = active[k] != 0.0 ? hrz[k] / hd[k] : 0.0;
    }
    TCK(setc(coef));
    k_axpy<<<gv, 256, 0, st>>>(n, B, coefd, 1, p, x); note_launch();
    k_axpy<<<gv, 256, 0, st>>>(n, B, coefd, -1, Ap, r); note_launch();
    ++it;
    TCK(dot(r, r, hrr.data()));
    for (int k = 0; k < B; ++k)
      if (active[k] != 0.0) {
        iters[k] = it;
        if (std::sqrt(hrr[k]) <= tol * hb[k]) active[k] = 0.0;
      }
    if (!any_active() || it >= max_iter) break;
    k_jac<<<gv, 256, 0, st>>>(n, B, dinv, nullptr, nullptr, r, z); note_launch();
    std::vector<double> rzn(B);
    TCK(dot(r, z, rzn.data()));
    for (int k = 0; k < B; ++k) {
      coef[k] = (active[k] != 0.0 && hrz[k] != 0.0) ? rzn[k] / hrz[k] : 0.0;
      hrz[k] = rzn[k];
    }
    TCK(setc(coef));
    k_xpay<<<gv, 256, 0, st>>>(n, B, coefd, z, p); note_launch();
  }
#undef TCK
  if (status == DG_OK && any_active()) status = DG_ERR_NOT_CONVERGED;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int k = 0; k < B; ++k) {
      info->iters[k] = iters[k];
      info->relres[k] = hb[k] > 0.0 ? std::sqrt(hrr[k]) / hb[k] : 0.0;
    }
    info->total_iters = it;
  }
  return status;
}

}  // extern "C"
