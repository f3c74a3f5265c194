// Reference-element data for the nodal DG triangle (host, FP64).
//
// Section 2.1: the basis of P_N on each triangle is the set of Lagrange
// polynomials through the Warp & Blend nodes (Warburton 2006). Section 5.2
// (Eq. elMass, elStiff, elLift, elementOps) builds everything from reference
// operators on the bi-unit triangle: mass M, differentiation Dr, Ds and the
// face mass used by the lift. They are formed here from the orthonormal
// (Dubiner) modal basis: M = (V V^T)^{-1}, Dr = V_r V^{-1}, Ds = V_s V^{-1},
// face mass Mf = (V1 V1^T)^{-1} with the 1-D Legendre Vandermonde V1 at the
// Gauss-Lobatto face nodes.
#include "dg_internal.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace dgx {

// Optimised Warp & Blend blend parameters alpha(N), N = 1..15 (Warburton 2006).
static const double kAlphaOpt[15] = {0.0000, 0.0000, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
                                     1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258};

// Recurrence coefficients of the orthonormal Jacobi polynomials:
//   x p_n = a_{n+1} p_{n+1} + b_n p_n + a_n p_{n-1}.
static double rec_a(int n, double a, double b) {
  const double h = 2.0 * n + a + b;
  return 2.0 / h * std::sqrt(n * (n + a + b) * (n + a) * (n + b) / ((h - 1.0) * (h + 1.0)));
}
static double rec_b(int n, double a, double b) {
  if (n == 0) return (b - a) / (a + b + 2.0);
  const double h = 2.0 * n + a + b;
  return (b * b - a * a) / (h * (h + 2.0));
}
static double norm0(double a, double b) {
  // integral of (1-x)^a (1+x)^b over [-1,1]
  return std::exp((a + b + 1.0) * std::log(2.0) + std::lgamma(a + 1.0) + std::lgamma(b + 1.0) -
                  std::lgamma(a + b + 2.0));
}

double jacobi_p(double x, double a, double b, int n) {
  double pm1 = 0.0, p = 1.0 / std::sqrt(norm0(a, b));
  for (int k = 0; k < n; ++k) {
    const double pn = ((x - rec_b(k, a, b)) * p - (k > 0 ? rec_a(k, a, b) * pm1 : 0.0)) / rec_a(k + 1, a, b);
    pm1 = p;
    p = pn;
  }
  return p;
}

double jacobi_dp(double x, double a, double b, int n) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + a + b + 1.0)) * jacobi_p(x, a + 1.0, b + 1.0, n - 1);
}

// Symmetric eigenvalue decomposition by cyclic Jacobi rotations (small n).
// A (n x n, row-major) is overwritten; eigenvalues in w, eigenvectors in columns of Q.
static void sym_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& Q) {
  Q.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-32) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

// Gauss-Jacobi rule by Golub-Welsch: nodes = eigenvalues of the Jacobi matrix,
// weights = mu_0 * (first eigenvector component)^2. Sorted ascending.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& wts) {
  std::vector<double> T(n * n, 0.0), w, Q;
  for (int i = 0; i < n; ++i) {
    T[i * n + i] = rec_b(i, a, b);
    if (i + 1 < n) T[i * n + i + 1] = T[(i + 1) * n + i] = rec_a(i + 1, a, b);
  }
  sym_eig(n, T, w, Q);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return w[i] < w[j]; });
  x.resize(n);
  wts.resize(n);
  const double mu0 = norm0(a, b);
  for (int k = 0; k < n; ++k) {
    x[k] = w[idx[k]];
    wts[k] = mu0 * Q[0 * n + idx[k]] * Q[0 * n + idx[k]];
  }
}

std::vector<double> lobatto_points(int N) {
  std::vector<double> t(N + 1);
  t[0] = -1.0;
  t[N] = 1.0;
  if (N >= 2) {
    std::vector<double> x, w;
    gauss_jacobi(N - 1, 1.0, 1.0, x, w);
    for (int i = 0; i < N - 1; ++i) t[i + 1] = x[i];
  }
  return t;
}

// 1-D warp: interpolant through equispaced points of (Lobatto - equispaced),
// divided by 1 - r^2 away from the end points.
static double warp(int N, double rr, const std::vector<double>& lgl) {
  double v = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double ri = -1.0 + 2.0 * i / N;
    double li = 1.0;
    for (int j = 0; j <= N; ++j)
      if (j != i) li *= (rr - (-1.0 + 2.0 * j / N)) / (ri - (-1.0 + 2.0 * j / N));
    v += li * (lgl[i] - ri);
  }
  if (std::fabs(rr) < 1.0 - 1e-10) return v / (1.0 - rr * rr);
  return 0.0;
}

void warp_blend_nodes(int N, std::vector<double>& r, std::vector<double>& s) {
  const double alpha = N <= 15 ? kAlphaOpt[N - 1] : 5.0 / 3.0;
  const std::vector<double> lgl = lobatto_points(N);
  const double sq3 = std::sqrt(3.0);
  r.clear();
  s.clear();
  for (int row = 0; row <= N; ++row) {
    for (int m = 0; m <= N - row; ++m) {
      const double L1 = double(row) / N, L3 = double(m) / N, L2 = 1.0 - L1 - L3;
      double X = -L2 + L3, Y = (-L2 - L3 + 2.0 * L1) / sq3;
      const double d1 = 4 * L2 * L3 * warp(N, L3 - L2, lgl) * (1 + (alpha * L1) * (alpha * L1));
      const double d2 = 4 * L1 * L3 * warp(N, L1 - L3, lgl) * (1 + (alpha * L2) * (alpha * L2));
      const double d3 = 4 * L1 * L2 * warp(N, L2 - L1, lgl) * (1 + (alpha * L3) * (alpha * L3));
      const double c2 = std::cos(2 * M_PI / 3), c3 = std::cos(4 * M_PI / 3);
      const double s2 = std::sin(2 * M_PI / 3), s3 = std::sin(4 * M_PI / 3);
      X += d1 + c2 * d2 + c3 * d3;
      Y += s2 * d2 + s3 * d3;
      const double l1 = (sq3 * Y + 1.0) / 3.0;
      const double l2 = (-3.0 * X - sq3 * Y + 2.0) / 6.0;
      const double l3 = (3.0 * X - sq3 * Y + 2.0) / 6.0;
      r.push_back(-l2 + l3 - l1);
      s.push_back(-l2 - l3 + l1);
    }
  }
}

// Orthonormal simplex basis psi_{ij} and its (r, s) gradient at one point.
static void simplex_eval(int i, int j, double r, double s, double* psi, double* dr, double* ds) {
  double a = (std::fabs(1.0 - s) < 1e-14) ? -1.0 : 2.0 * (1.0 + r) / (1.0 - s) - 1.0;
  const double b = s;
  const double fa = jacobi_p(a, 0, 0, i), dfa = jacobi_dp(a, 0, 0, i);
  const double gb = jacobi_p(b, 2.0 * i + 1, 0, j), dgb = jacobi_dp(b, 2.0 * i + 1, 0, j);
  const double sq2 = std::sqrt(2.0);
  if (psi) *psi = sq2 * fa * gb * std::pow(1.0 - b, i);
  if (dr || ds) {
    double vr, vs;
    if (i == 0) {
      vr = 0.0;
      vs = fa * dgb;
    } else {
      const double t = std::pow(1.0 - b, i - 1);
      vr = 2.0 * dfa * gb * t;
      vs = (1.0 + a) * dfa * gb * t + fa * (dgb * std::pow(1.0 - b, i) - i * gb * t);
    }
    if (dr) *dr = sq2 * vr;
    if (ds) *ds = sq2 * vs;
  }
}

void vandermonde2d(int N, const std::vector<double>& r, const std::vector<double>& s, std::vector<double>& V,
                   std::vector<double>* Vr, std::vector<double>* Vs) {
  const int Np = (N + 1) * (N + 2) / 2, n = int(r.size());
  V.assign(size_t(n) * Np, 0.0);
  if (Vr) Vr->assign(size_t(n) * Np, 0.0);
  if (Vs) Vs->assign(size_t(n) * Np, 0.0);
  for (int q = 0; q < n; ++q) {
    int k = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N - i; ++j, ++k) {
        double p, dr, ds;
        simplex_eval(i, j, r[q], s[q], &p, &dr, &ds);
        V[size_t(q) * Np + k] = p;
        if (Vr) (*Vr)[size_t(q) * Np + k] = dr;
        if (Vs) (*Vs)[size_t(q) * Np + k] = ds;
      }
  }
}

// Inverse of a dense n x n matrix by Gauss-Jordan elimination with partial pivoting.
std::vector<double> invert(int n, std::vector<double> A) {
  std::vector<double> I(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) I[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(A[size_t(i) * n + c]) > std::fabs(A[size_t(piv) * n + c])) piv = i;
    if (std::fabs(A[size_t(piv) * n + c]) < 1e-300) throw std::runtime_error("singular matrix");
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[size_t(c) * n + k], A[size_t(piv) * n + k]);
        std::swap(I[size_t(c) * n + k], I[size_t(piv) * n + k]);
      }
    const double d = 1.0 / A[size_t(c) * n + c];
    for (int k = 0; k < n; ++k) {
      A[size_t(c) * n + k] *= d;
      I[size_t(c) * n + k] *= d;
    }
    for (int i = 0; i < n; ++i)
      if (i != c) {
        const double f = A[size_t(i) * n + c];
        if (f == 0.0) continue;
        for (int k = 0; k < n; ++k) {
          A[size_t(i) * n + k] -= f * A[size_t(c) * n + k];
          I[size_t(i) * n + k] -= f * I[size_t(c) * n + k];
        }
      }
  }
  return I;
}

static std::vector<double> matmul(int n, int m, int p, const std::vector<double>& A, const std::vector<double>& B) {
  std::vector<double> C(size_t(n) * p, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < m; ++k) {
      const double a = A[size_t(i) * m + k];
      for (int j = 0; j < p; ++j) C[size_t(i) * p + j] += a * B[size_t(k) * p + j];
    }
  return C;
}

static std::vector<double> transpose(int n, int m, const std::vector<double>& A) {
  std::vector<double> T(size_t(m) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) T[size_t(j) * n + i] = A[size_t(i) * m + j];
  return T;
}

int face_node(int N, int f, int j) {
  // counter-clockwise: face 0 v0->v1 (first row), face 1 v1->v2 (last node of
  // each row, upward), face 2 v2->v0 (first node of each row, downward)
  auto row_start = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  if (f == 0) return j;
  if (f == 1) return row_start(j) + (N - j);
  return row_start(N - j);
}

RefElem build_reference(int N) {
  if (N < 1 || N > kMaxN) throw std::invalid_argument("degree out of range");
  RefElem R;
  R.N = N;
  R.Np = (N + 1) * (N + 2) / 2;
  R.Nfp = N + 1;
  const int Np = R.Np, Nfp = R.Nfp;
  warp_blend_nodes(N, R.r, R.s);
  std::vector<double> V, Vr, Vs;
  vandermonde2d(N, R.r, R.s, V, &Vr, &Vs);
  R.Vinv = invert(Np, V);
  R.M = invert(Np, matmul(Np, Np, Np, V, transpose(Np, Np, V)));
  R.Dr = matmul(Np, Np, Np, Vr, R.Vinv);
  R.Ds = matmul(Np, Np, Np, Vs, R.Vinv);
  R.Br = matmul(Np, Np, Np, transpose(Np, Np, R.Dr), R.M);
  R.Bs = matmul(Np, Np, Np, transpose(Np, Np, R.Ds), R.M);
  const std::vector<double> t = lobatto_points(N);
  std::vector<double> V1(size_t(Nfp) * Nfp);
  for (int i = 0; i < Nfp; ++i)
    for (int k = 0; k < Nfp; ++k) V1[size_t(i) * Nfp + k] = jacobi_p(t[i], 0, 0, k);
  R.Mf = invert(Nfp, matmul(Nfp, Nfp, Nfp, V1, transpose(Nfp, Nfp, V1)));
  R.fmask.resize(3 * Nfp);
  for (int f = 0; f < 3; ++f)
    for (int j = 0; j < Nfp; ++j) R.fmask[f * Nfp + j] = face_node(N, f, j);
  // diagonal data for the Jacobi preconditioner:
  //   S_ab = D_a^T M D_b (stiffness pieces), and per face node the Mf-weighted
  //   face-row sums of Dr/Ds at that node.
  const std::vector<double> Srr = matmul(Np, Np, Np, R.Br, R.Dr);
  const std::vector<double> Srs = matmul(Np, Np, Np, R.Br, R.Ds);
  const std::vector<double> Sss = matmul(Np, Np, Np, R.Bs, R.Ds);
  R.diag_rr.resize(Np);
  R.diag_rs.resize(Np);
  R.diag_ss.resize(Np);
  R.diag_m.resize(Np);
  for (int i = 0; i < Np; ++i) {
    R.diag_rr[i] = Srr[size_t(i) * Np + i];
    R.diag_rs[i] = 2.0 * Srs[size_t(i) * Np + i];
    R.diag_ss[i] = Sss[size_t(i) * Np + i];
    R.diag_m[i] = R.M[size_t(i) * Np + i];
  }
  R.face_cr.resize(3 * Nfp);
  R.face_cs.resize(3 * Nfp);
  for (int f = 0; f < 3; ++f)
    for (int a = 0; a < Nfp; ++a) {
      const int i = R.fmask[f * Nfp + a];
      double cr = 0.0, cs = 0.0;
      for (int b = 0; b < Nfp; ++b) {
        const int kb = R.fmask[f * Nfp + b];
        cr += R.Mf[size_t(a) * Nfp + b] * R.Dr[size_t(kb) * Np + i];
        cs += R.Mf[size_t(a) * Nfp + b] * R.Ds[size_t(kb) * Np + i];
      }
      R.face_cr[f * Nfp + a] = cr;
      R.face_cs[f * Nfp + a] = cs;
    }
  return R;
}

std::vector<double> interpolation_matrix(int Nf, int Nc) {
  RefElem F = build_reference(Nf), C = build_reference(Nc);
  std::vector<double> Vcf;
  vandermonde2d(Nc, F.r, F.s, Vcf, nullptr, nullptr);
  return matmul(F.Np, C.Np, C.Np, Vcf, C.Vinv);
}

}  // namespace dgx
