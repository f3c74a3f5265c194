// Algebraic multigrid for the coarsest p-multigrid degree (Section 3).
//
// The paper finishes its p-multigrid hierarchy with algebraic multigrid on the
// degree-1 matrix (pMG-AMG): aggregation of the matrix graph, degree-2
// Chebyshev smoothing. Here the coarsest SIPDG matrix is first assembled from
// the library's own GPU operator by probing: with a distance-2 colouring of
// the element graph, the operator applied to one unit nodal function per
// element of a colour returns disjoint element blocks, so Np x (colours)
// batched applies give every matrix entry exactly. The hierarchy (host, FP64)
// uses strength-of-connection aggregation and a damped-Jacobi-smoothed
// prolongator (smoothed aggregation; the paper's unsmoothed aggregation needs
// a K-cycle to converge, the smoothed prolongator converges with a plain
// V-cycle), Galerkin coarse matrices R A P with R = P^T, and a dense inverse
// at the bottom. The V-cycle runs on the GPU: CSR products, Chebyshev-Jacobi
// smoothing of degree 2 on the interval [rho/10, 1.1 rho].
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "dg_internal.h"

namespace dgx {

struct Csr {
  int64_t n = 0, m = 0;  // rows, cols
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

struct DevCsr {
  int64_t n = 0, nnz = 0;
  int64_t* ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
};

struct AmgLevel {
  DevCsr A, P, R;      // P: n x n_next, R = P^T
  double* dinv = nullptr;
  double rho = 1.0;    // largest eigenvalue estimate of D^{-1} A
  double *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *t = nullptr;  // [B][n]
};

struct Amg {
  int B = 0;
  DevCsr A0;               // the probed fine matrix (also level 0 of L when L is not empty)
  std::vector<AmgLevel> L;
  double* cinv = nullptr;  // dense inverse of the coarsest matrix
  int64_t nc = 0;
  double *cb = nullptr, *cx = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;  // device bytes held in allocs
};

void amg_free(Amg* a) {
  if (!a) return;
  for (void* p : a->allocs) cudaFree(p);
  delete a;
}

namespace {

// ------------------------------------------------------------------ host CSR
Csr transpose(const Csr& A) {
  Csr T;
  T.n = A.m;
  T.m = A.n;
  T.ptr.assign(T.n + 1, 0);
  for (int32_t c : A.col) T.ptr[c + 1]++;
  for (int64_t i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int64_t> pos(T.ptr.begin(), T.ptr.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      const int64_t p = pos[A.col[k]]++;
      T.col[p] = int32_t(i);
      T.val[p] = A.val[k];
    }
  return T;
}

// C = A B (Gustavson, dense marker per row)
Csr spgemm(const Csr& A, const Csr& Bm) {
  Csr C;
  C.n = A.n;
  C.m = Bm.m;
  C.ptr.assign(C.n + 1, 0);
  std::vector<int64_t> mark(Bm.m, -1);
  std::vector<double> acc(Bm.m, 0.0);
  std::vector<int32_t> cols;
  for (int64_t i = 0; i < A.n; ++i) {
    cols.clear();
    for (int64_t ka = A.ptr[i]; ka < A.ptr[i + 1]; ++ka) {
      const int32_t k = A.col[ka];
      const double a = A.val[ka];
      for (int64_t kb = Bm.ptr[k]; kb < Bm.ptr[k + 1]; ++kb) {
        const int32_t j = Bm.col[kb];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * Bm.val[kb];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      C.col.push_back(j);
      C.val.push_back(acc[j]);
    }
    C.ptr[i + 1] = int64_t(C.col.size());
  }
  return C;
}

std::vector<double> diag_of(const Csr& A) {
  std::vector<double> d(A.n, 0.0);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (A.col[k] == i) d[i] = A.val[k];
  return d;
}

void spmv_h(const Csr& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign(A.n, 0.0);
  for (int64_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
    y[i] = s;
  }
}

// largest eigenvalue of D^{-1}A by power iteration from a seeded start
double rho_dinv_a(const Csr& A, const std::vector<double>& d, int steps) {
  std::vector<double> v(A.n), w;
  std::mt19937_64 rng(777);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (auto& e : v) e = nd(rng);
  double lam = 1.0;
  for (int s = 0; s < steps; ++s) {
    double nv = 0.0;
    for (double e : v) nv += e * e;
    nv = std::sqrt(nv);
    for (auto& e : v) e /= nv;
    spmv_h(A, v, w);
    double nw = 0.0;
    for (int64_t i = 0; i < A.n; ++i) {
      w[i] /= d[i];
      nw += w[i] * w[i];
    }
    lam = std::sqrt(nw);
    v.swap(w);
  }
  return lam;
}

// Strength-of-connection aggregation (three passes): returns agg[i] and count.
int64_t aggregate(const Csr& A, const std::vector<double>& d, double theta, std::vector<int64_t>& agg) {
  const int64_t n = A.n;
  agg.assign(n, -1);
  auto strong = [&](int64_t i, int64_t k) {
    const int32_t j = A.col[k];
    return j != i && std::fabs(A.val[k]) >= theta * std::sqrt(std::fabs(d[i] * d[j]));
  };
  int64_t na = 0;
  for (int64_t i = 0; i < n; ++i) {  // pass 1: root + whole free strong neighbourhood
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1] && free_nb; ++k)
      if (strong(i, k) && agg[A.col[k]] >= 0) free_nb = false;
    if (!free_nb) continue;
    agg[i] = na;
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (strong(i, k)) agg[A.col[k]] = na;
    ++na;
  }
  std::vector<int64_t> agg1 = agg;
  for (int64_t i = 0; i < n; ++i) {  // pass 2: join a strongly connected aggregate
    if (agg[i] >= 0) continue;
    double best = -1.0;
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (strong(i, k) && agg1[A.col[k]] >= 0 && std::fabs(A.val[k]) > best) {
        best = std::fabs(A.val[k]);
        agg[i] = agg1[A.col[k]];
      }
  }
  for (int64_t i = 0; i < n; ++i) {  // pass 3: leftovers form their own aggregates
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
      if (agg[A.col[k]] < 0) agg[A.col[k]] = na;
    ++na;
  }
  return na;
}

// ------------------------------------------------------------------ device
__global__ void k_probe_vec(int64_t K, int Np, int ncol0, int nvec, const int32_t* __restrict__ color,
                            double* __restrict__ v) {
  // v[p][e][i] = 1 if color[e]*Np + i == ncol0 + p
  const int64_t total = int64_t(nvec) * K * Np;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = idx / (K * Np);
    const int64_t rem = idx - p * K * Np;
    const int64_t e = rem / Np;
    const int i = int(rem - e * Np);
    v[idx] = (int64_t(color[e]) * Np + i == ncol0 + p) ? 1.0 : 0.0;
  }
}

// y[b] = alpha A x[b] + beta y[b]  (one row per thread group of 4 lanes)
__global__ void k_spmv(int64_t n, int64_t xs, int64_t ys, int B, const int64_t* __restrict__ ptr,
                       const int32_t* __restrict__ col, const double* __restrict__ val, const double* __restrict__ x,
                       double* __restrict__ y, double alpha, double beta) {
  const int64_t g = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 2;
  const int lane = threadIdx.x & 3;
  const int b = blockIdx.y;
  const bool valid = g < n;  // every lane stays for the shuffles below
  const double* xb = x + size_t(b) * xs;
  double s = 0.0;
  if (valid)
    for (int64_t k = ptr[g] + lane; k < ptr[g + 1]; k += 4) s += val[k] * xb[col[k]];
  s += __shfl_down_sync(0xffffffffu, s, 2, 4);
  s += __shfl_down_sync(0xffffffffu, s, 1, 4);
  if (valid && lane == 0) {
    double* yb = y + size_t(b) * ys;
    yb[g] = alpha * s + (beta != 0.0 ? beta * yb[g] : 0.0);
  }
}

// Chebyshev pieces on [B][n] vectors, dinv shared across the batch
__global__ void k_cheb0(int64_t n, int B, const double* __restrict__ dinv, const double* __restrict__ res,
                        double* __restrict__ d, double* __restrict__ x, double c0, int zero_x) {
  const int64_t tot = n * B;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot; i += int64_t(gridDim.x) * blockDim.x) {
    const double di = c0 * dinv[i % n] * res[i];
    d[i] = di;
    x[i] = zero_x ? di : x[i] + di;
  }
}
__global__ void k_cheb1(int64_t n, int B, const double* __restrict__ dinv, const double* __restrict__ Ad,
                        double* __restrict__ res, double* __restrict__ d, double* __restrict__ x, double c1,
                        double c2) {
  const int64_t tot = n * B;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot; i += int64_t(gridDim.x) * blockDim.x) {
    const double r = res[i] - Ad[i];
    res[i] = r;
    const double di = c1 * d[i] + c2 * dinv[i % n] * r;
    d[i] = di;
    x[i] += di;
  }
}
__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = a[i];
}
// y[b] = Minv x[b] (dense, n <= a few thousand)
__global__ void k_dense(int64_t n, const double* __restrict__ M, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= n) return;
  const double* xb = x + size_t(b) * n;
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j) s += M[size_t(i) * n + j] * xb[j];
  y[size_t(b) * n + i] = s;
}

inline int eg(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return int(b < 1 ? 1 : b);
}

#define ACK(x)                         \
  do {                                 \
    cudaError_t e_ = (x);              \
    if (e_ != cudaSuccess) return e_;  \
  } while (0)

cudaError_t upload(Amg* a, const Csr& h, DevCsr& d) {
  d.n = h.n;
  d.nnz = int64_t(h.col.size());
  ACK(cudaMalloc(&d.ptr, sizeof(int64_t) * (h.n + 1)));
  a->allocs.push_back(d.ptr);
  ACK(cudaMalloc(&d.col, sizeof(int32_t) * std::max<int64_t>(d.nnz, 1)));
  a->allocs.push_back(d.col);
  ACK(cudaMalloc(&d.val, sizeof(double) * std::max<int64_t>(d.nnz, 1)));
  a->allocs.push_back(d.val);
  a->bytes += sizeof(int64_t) * (h.n + 1) + (sizeof(int32_t) + sizeof(double)) * std::max<int64_t>(d.nnz, 1);
  ACK(cudaMemcpy(d.ptr, h.ptr.data(), sizeof(int64_t) * (h.n + 1), cudaMemcpyHostToDevice));
  if (d.nnz) {
    ACK(cudaMemcpy(d.col, h.col.data(), sizeof(int32_t) * d.nnz, cudaMemcpyHostToDevice));
    ACK(cudaMemcpy(d.val, h.val.data(), sizeof(double) * d.nnz, cudaMemcpyHostToDevice));
  }
  return cudaSuccess;
}

cudaError_t spmv(const DevCsr& A, int B, int64_t xs, int64_t ys, const double* x, double* y, double alpha,
                 double beta, cudaStream_t st) {
  const int64_t threads = A.n * 4;
  dim3 grid(unsigned((threads + 255) / 256), unsigned(B));
  k_spmv<<<grid, 256, 0, st>>>(A.n, xs, ys, B, A.ptr, A.col, A.val, x, y, alpha, beta);
  note_launch();
  return cudaGetLastError();
}

// Assemble the SIPDG matrix of the given degree by probing the GPU operator.
cudaError_t probe_matrix(dg_mesh* m, int degree, double lambda, Csr& A, cudaStream_t st) {
  const int64_t K = m->K;
  const int Np = (degree + 1) * (degree + 2) / 2;
  // distance-2 colouring of the element graph
  std::vector<int32_t> color(K, -1);
  int ncolor = 0;
  std::vector<int> stamp(64, -1);
  for (int64_t e = 0; e < K; ++e) {
    std::vector<int64_t> near;
    for (int f = 0; f < 3; ++f) {
      const int32_t c = m->conn_h[3 * e + f];
      if (c < 0) continue;
      const int64_t nb = c >> 2;
      near.push_back(nb);
      for (int g = 0; g < 3; ++g) {
        const int32_t c2 = m->conn_h[3 * nb + g];
        if (c2 >= 0 && (c2 >> 2) != e) near.push_back(c2 >> 2);
      }
    }
    for (int64_t x : near)
      if (color[x] >= 0) stamp[color[x]] = int(e & 0x7fffffff);
    int c = 0;
    while (c < 64 && stamp[c] == int(e & 0x7fffffff)) ++c;
    if (c >= 64) return cudaErrorInvalidValue;  // cannot happen for a triangle mesh
    color[e] = c;
    ncolor = std::max(ncolor, c + 1);
  }
  // CSR structure: row block e holds dense Np x Np blocks for e and its neighbours (sorted)
  std::vector<std::array<int64_t, 4>> blk(K);
  std::vector<int> nblk(K);
  A.n = A.m = int64_t(K) * Np;
  A.ptr.assign(A.n + 1, 0);
  for (int64_t e = 0; e < K; ++e) {
    int c = 0;
    blk[e][c++] = e;
    for (int f = 0; f < 3; ++f)
      if (m->conn_h[3 * e + f] >= 0) blk[e][c++] = m->conn_h[3 * e + f] >> 2;
    std::sort(blk[e].begin(), blk[e].begin() + c);
    nblk[e] = c;
    for (int i = 0; i < Np; ++i) A.ptr[e * Np + i + 1] = A.ptr[e * Np + i] + int64_t(c) * Np;
  }
  A.col.resize(A.ptr[A.n]);
  A.val.assign(A.ptr[A.n], 0.0);
  for (int64_t e = 0; e < K; ++e)
    for (int i = 0; i < Np; ++i) {
      int64_t q = A.ptr[e * Np + i];
      for (int b = 0; b < nblk[e]; ++b)
        for (int j = 0; j < Np; ++j) A.col[q++] = int32_t(blk[e][b] * Np + j);
    }
  // elements of each colour
  std::vector<std::vector<int64_t>> members(ncolor);
  for (int64_t e = 0; e < K; ++e) members[color[e]].push_back(e);
  int32_t* dcolor = nullptr;
  ACK(cudaMalloc(&dcolor, sizeof(int32_t) * K));
  ACK(cudaMemcpy(dcolor, color.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice));
  const int nprobe = ncolor * Np;
  const int chunk = 16;
  const size_t n1 = size_t(K) * Np;
  double *v = nullptr, *w = nullptr;
  ACK(cudaMalloc(&v, sizeof(double) * n1 * chunk));
  ACK(cudaMalloc(&w, sizeof(double) * n1 * chunk));
  ACK(poison(v, sizeof(double) * n1 * chunk, POISON_AMG));
  ACK(poison(w, sizeof(double) * n1 * chunk, POISON_AMG));
  std::vector<double> res(size_t(chunk) * n1);
  ACK(ensure_ops(m, degree));
  for (int p0 = 0; p0 < nprobe; p0 += chunk) {
    const int nv = std::min(chunk, nprobe - p0);
    k_probe_vec<<<eg(int64_t(nv) * n1), 256, 0, st>>>(K, Np, p0, nv, dcolor, v);
    note_launch();
    ACK(launch_apply(m, degree, DG_F64, nv, lambda, v, w, st));
    ACK(cudaMemcpyAsync(res.data(), w, sizeof(double) * n1 * nv, cudaMemcpyDeviceToHost, st));
    ACK(cudaStreamSynchronize(st));
    for (int pp = 0; pp < nv; ++pp) {
      const int p = p0 + pp, c = p / Np, j = p % Np;
      const double* rp = res.data() + size_t(pp) * n1;
      for (int64_t x : members[c])
        for (int b = 0; b < nblk[x]; ++b) {
          const int64_t ep = blk[x][b];  // rows of element ep see column (x, j)
          int pos = 0;
          while (blk[ep][pos] != x) ++pos;
          for (int i = 0; i < Np; ++i) A.val[A.ptr[ep * Np + i] + int64_t(pos) * Np + j] = rp[ep * Np + i];
        }
    }
  }
  cudaFree(v);
  cudaFree(w);
  cudaFree(dcolor);
  return cudaSuccess;
}

}  // namespace

// Build the hierarchy for the degree-`degree` operator at lambda, batch B.
cudaError_t amg_build(dg_mesh* m, int degree, double lambda, int B, Amg** out, cudaStream_t st) {
  Amg* a = new Amg();
  *out = a;
  a->B = B;
  Csr A;
  ACK(probe_matrix(m, degree, lambda, A, st));
  ACK(upload(a, A, a->A0));
  const int64_t coarse_max = 400;
  for (int lev = 0; lev < 12; ++lev) {
    AmgLevel L;
    const std::vector<double> d = diag_of(A);
    L.rho = rho_dinv_a(A, d, 15);
    if (A.n <= coarse_max || lev == 11) {
      // coarsest: dense inverse
      const int64_t n = A.n;
      std::vector<double> Dn(size_t(n) * n, 0.0);
      for (int64_t i = 0; i < n; ++i)
        for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) Dn[size_t(i) * n + A.col[k]] = A.val[k];
      const std::vector<double> inv = invert(int(n), Dn);
      a->nc = n;
      ACK(cudaMalloc(&a->cinv, sizeof(double) * n * n));
      a->allocs.push_back(a->cinv);
      ACK(cudaMemcpy(a->cinv, inv.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice));
      ACK(cudaMalloc(&a->cb, sizeof(double) * n * B));
      ACK(poison(a->cb, sizeof(double) * n * B, POISON_AMG));
      a->allocs.push_back(a->cb);
      ACK(cudaMalloc(&a->cx, sizeof(double) * n * B));
      ACK(poison(a->cx, sizeof(double) * n * B, POISON_AMG));
      a->allocs.push_back(a->cx);
      a->bytes += sizeof(double) * (size_t(n) * n + 2 * size_t(n) * B);
      break;
    }
    std::vector<int64_t> agg;
    const int64_t na = aggregate(A, d, 0.08, agg);
    // tentative prolongator (normalised indicator columns), then one damped
    // Jacobi smoothing step: P = (I - w D^{-1} A) T, w = 4 / (3 rho)
    std::vector<int64_t> cnt(na, 0);
    for (int64_t i = 0; i < A.n; ++i) cnt[agg[i]]++;
    Csr T;
    T.n = A.n;
    T.m = na;
    T.ptr.resize(A.n + 1);
    for (int64_t i = 0; i <= A.n; ++i) T.ptr[i] = i;
    T.col.resize(A.n);
    T.val.resize(A.n);
    for (int64_t i = 0; i < A.n; ++i) {
      T.col[i] = int32_t(agg[i]);
      T.val[i] = 1.0 / std::sqrt(double(cnt[agg[i]]));
    }
    Csr AT = spgemm(A, T);
    const double w = 4.0 / (3.0 * L.rho);
    Csr P;
    P.n = A.n;
    P.m = na;
    P.ptr.assign(A.n + 1, 0);
    for (int64_t i = 0; i < A.n; ++i) {
      bool has_diag = false;
      for (int64_t k = AT.ptr[i]; k < AT.ptr[i + 1]; ++k) {
        double v = -w / d[i] * AT.val[k];
        if (AT.col[k] == T.col[i]) {
          v += T.val[i];
          has_diag = true;
        }
        P.col.push_back(AT.col[k]);
        P.val.push_back(v);
      }
      if (!has_diag) {
        P.col.push_back(T.col[i]);
        P.val.push_back(T.val[i]);
      }
      P.ptr[i + 1] = int64_t(P.col.size());
    }
    Csr R = transpose(P);
    Csr Ac = spgemm(R, spgemm(A, P));
    if (lev == 0) L.A = a->A0;  // the probed matrix, already on the device
    else ACK(upload(a, A, L.A));
    ACK(upload(a, P, L.P));
    ACK(upload(a, R, L.R));
    std::vector<double> di(A.n);
    for (int64_t i = 0; i < A.n; ++i) di[i] = 1.0 / d[i];
    ACK(cudaMalloc(&L.dinv, sizeof(double) * A.n));
    a->allocs.push_back(L.dinv);
    a->bytes += sizeof(double) * A.n * (1 + 5 * size_t(B));  // dinv and the five level vectors
    ACK(cudaMemcpy(L.dinv, di.data(), sizeof(double) * A.n, cudaMemcpyHostToDevice));
    for (double** p : {&L.x, &L.b, &L.r, &L.d, &L.t}) {
      ACK(cudaMalloc(p, sizeof(double) * A.n * B));
      ACK(poison(*p, sizeof(double) * A.n * B, POISON_AMG));
      a->allocs.push_back(*p);
    }
    a->L.push_back(L);
    A = std::move(Ac);
  }
  return cudaSuccess;
}

namespace {

// Chebyshev smoothing on level l (degree 2), x either zero or given
cudaError_t smooth(Amg* a, int l, int B, bool zero_x, cudaStream_t st) {
  AmgLevel& L = a->L[l];
  const int64_t n = L.A.n;
  const double lmin = L.rho / 10.0, lmax = 1.1 * L.rho;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rk = 1.0 / sigma;
  if (zero_x) {
    k_copy<<<eg(n * B), 256, 0, st>>>(n * B, L.b, L.r);
    note_launch();
  } else {
    k_copy<<<eg(n * B), 256, 0, st>>>(n * B, L.b, L.r);
    note_launch();
    ACK(spmv(L.A, B, n, n, L.x, L.r, -1.0, 1.0, st));
  }
  k_cheb0<<<eg(n * B), 256, 0, st>>>(n, B, L.dinv, L.r, L.d, L.x, 1.0 / theta, zero_x ? 1 : 0);
  note_launch();
  const double rnew = 1.0 / (2.0 * sigma - rk);
  ACK(spmv(L.A, B, n, n, L.d, L.t, 1.0, 0.0, st));
  k_cheb1<<<eg(n * B), 256, 0, st>>>(n, B, L.dinv, L.t, L.r, L.d, L.x, rnew * rk, 2.0 * rnew / delta);
  note_launch();
  return cudaGetLastError();
}

cudaError_t vcyc(Amg* a, int l, int B, cudaStream_t st) {
  if (l == int(a->L.size())) {
    dim3 grid(unsigned((a->nc + 127) / 128), unsigned(B));
    k_dense<<<grid, 128, 0, st>>>(a->nc, a->cinv, a->cb, a->cx);
    note_launch();
    return cudaGetLastError();
  }
  AmgLevel& L = a->L[l];
  const int64_t n = L.A.n;
  ACK(smooth(a, l, B, true, st));
  // residual after pre-smoothing, restricted to the next level
  k_copy<<<eg(n * B), 256, 0, st>>>(n * B, L.b, L.r);
  note_launch();
  ACK(spmv(L.A, B, n, n, L.x, L.r, -1.0, 1.0, st));
  const bool last = (l + 1 == int(a->L.size()));
  const int64_t nn = last ? a->nc : a->L[l + 1].A.n;
  double* nb = last ? a->cb : a->L[l + 1].b;
  double* nx = last ? a->cx : a->L[l + 1].x;
  ACK(spmv(L.R, B, n, nn, L.r, nb, 1.0, 0.0, st));
  ACK(vcyc(a, l + 1, B, st));
  ACK(spmv(L.P, B, nn, n, nx, L.x, 1.0, 1.0, st));
  ACK(smooth(a, l, B, false, st));
  return cudaGetLastError();
}

}  // namespace

// x = V(b), one V-cycle for B right-hand sides ([B][n] each, n = rows of level 0)
cudaError_t amg_vcycle(Amg* a, const double* b, double* x, cudaStream_t st) {
  if (a->L.empty()) {  // tiny problem: dense solve only
    k_copy<<<eg(a->nc * a->B), 256, 0, st>>>(a->nc * a->B, b, a->cb);
    note_launch();
    dim3 grid(unsigned((a->nc + 127) / 128), unsigned(a->B));
    k_dense<<<grid, 128, 0, st>>>(a->nc, a->cinv, a->cb, x);
    note_launch();
    return cudaGetLastError();
  }
  AmgLevel& L0 = a->L[0];
  const int64_t n = L0.A.n;
  k_copy<<<eg(n * a->B), 256, 0, st>>>(n * a->B, b, L0.b);
  note_launch();
  ACK(vcyc(a, 0, a->B, st));
  k_copy<<<eg(n * a->B), 256, 0, st>>>(n * a->B, L0.x, x);
  note_launch();
  return cudaGetLastError();
}

int amg_levels(const Amg* a) { return a ? int(a->L.size()) + 1 : 0; }
size_t amg_bytes(const Amg* a) { return a ? a->bytes : 0; }

// y = A0 x for the Amg's batch of right-hand sides
cudaError_t amg_apply_fine(Amg* a, const double* x, double* y, cudaStream_t st) {
  return spmv(a->A0, a->B, a->A0.n, a->A0.n, x, y, 1.0, 0.0, st);
}

}  // namespace dgx
