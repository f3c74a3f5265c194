// Semi-implicit incompressible Navier-Stokes step with semi-Lagrangian
// subcycling (Section 2.2 Eq. INS_TD_3; Section 2.3; Section 5.3).
//
// Per macro step:
//   (i)   advection: each history field U^{n-i} is advected to t^{n+1} with
//         LSERK(5,4) substeps of dU~/dt = -N~(Ubar, U~), where N~ is the weak DG
//         advection operator of Eq. INS_CUB_N evaluated with cubature (the
//         volume term of Eq. KSS_3 through combined differentiation/projection
//         operators P_r, P_s, the surface term through a cubature lift) and
//         the local Lax-Friedrichs flux; Ubar is the linear extrapolant
//         through U^n and U^{n-1}; U^ = sum beta_i U~^{n-i};
//   (ii)  both velocity components in one batched Helmholtz PCG;
//   (iii) the pressure-increment Poisson PCG;
//   (iv)  the pressure-gradient correction.
// At degrees 1-2 one advection kernel computes volume and surface terms
// together and applies the LSERK stage update, ping-ponging U~ between two
// buffers so neighbours always read the previous stage. From degree 3 the
// stage's two dense contractions (cubature interpolation, projection with the
// lift) run as exactly sliced FP64 products on the tensor cores, around an
// FP64 kernel for the fluxes at the cubature points.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dgx {

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage Runge-Kutta.
static const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
static const double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                               2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

// Cubature operators of one degree (device, FP64), offsets into one buffer.
struct AdvLayout {
  int N = 0, Np = 0, Nfp = 0, nc = 0, Nc = 0;
  size_t Iq = 0, Pr = 0, Ps = 0, I1 = 0, Lc = 0, M = 0, Minv = 0, Dr = 0, Ds = 0, Mf = 0, total = 0;
};

struct InsWorkspace {
  int64_t K = 0;
  int N = 0;
  AdvLayout L;
  double* ops = nullptr;
  // tensor-core advection (degree >= 3): the cubature interpolation Iq and the
  // projection blocks Pr, Ps, -Lc as sliced FP64 operators, with their row
  // buffers (the projection is split at its blocks so that every sliced product
  // sums at most 256 terms, which keeps its FP32 group sums exact)
  bool tensor = false;
  SlicedOp opIq, opPr, opPs, opLc;
  double *X = nullptr, *W = nullptr, *Y = nullptr, *R = nullptr;
  double *Ut0 = nullptr, *Ut1 = nullptr, *res = nullptr, *Uhat = nullptr, *Uhh = nullptr, *bu = nullptr,
         *G = nullptr, *bp = nullptr, *dP = nullptr, *tmp = nullptr;
  double *gts = nullptr, *zero = nullptr;  // time-dependent data: velocity data at a stage time; zeros
  std::vector<void*> allocs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

void free_ins_workspace(dg_mesh* m) {
  InsWorkspace* w = m->ins;
  if (!w) return;
  for (void* p : w->allocs) cudaFree(p);
  sliced_op_free(&w->opIq);
  sliced_op_free(&w->opPr);
  sliced_op_free(&w->opPs);
  sliced_op_free(&w->opLc);
  if (w->ev0) cudaEventDestroy(w->ev0);
  if (w->ev1) cudaEventDestroy(w->ev1);
  delete w;
  m->ins = nullptr;
}

namespace {

__host__ __device__ inline int row_start_i(int N, int row) { return row * (N + 1) - row * (row - 1) / 2; }
__host__ __device__ inline int fnode_i(int N, int f, int j) {
  return f == 0 ? j : (f == 1 ? row_start_i(N, j) + (N - j) : row_start_i(N, N - j));
}

// Build the cubature operators on the host (FP64).
std::vector<double> build_adv_ops(const RefElem& R, AdvLayout& L) {
  const int N = R.N, Np = R.Np, Nfp = R.Nfp;
  const int nc = (3 * N + 2) / 2;  // ceil((3N+1)/2): exact for degree 3N
  L.N = N;
  L.Np = Np;
  L.Nfp = Nfp;
  L.nc = nc;
  L.Nc = nc * nc;
  std::vector<double> xa, wa, xb, wb;
  gauss_jacobi(nc, 0.0, 0.0, xa, wa);
  gauss_jacobi(nc, 1.0, 0.0, xb, wb);
  std::vector<double> rq, sq, wq;
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) {
      rq.push_back(0.5 * (1.0 + xa[i]) * (1.0 - xb[j]) - 1.0);
      sq.push_back(xb[j]);
      wq.push_back(0.5 * wa[i] * wb[j]);
    }
  const int Nc = L.Nc;
  std::vector<double> Vq, Vrq, Vsq;
  vandermonde2d(N, rq, sq, Vq, &Vrq, &Vsq);
  auto mm = [](int n, int k, int p, const std::vector<double>& A, const std::vector<double>& B) {
    std::vector<double> C(size_t(n) * p, 0.0);
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < k; ++q) {
        const double a = A[size_t(i) * k + q];
        for (int j = 0; j < p; ++j) C[size_t(i) * p + j] += a * B[size_t(q) * p + j];
      }
    return C;
  };
  const std::vector<double> Iq = mm(Nc, Np, Np, Vq, R.Vinv);
  const std::vector<double> Lr = mm(Nc, Np, Np, Vrq, R.Vinv);
  const std::vector<double> Ls = mm(Nc, Np, Np, Vsq, R.Vinv);
  const std::vector<double> Minv = invert(Np, R.M);
  std::vector<double> Pr(size_t(Np) * Nc), Ps(size_t(Np) * Nc);
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < Nc; ++q) {
      double a = 0.0, b = 0.0;
      for (int m = 0; m < Np; ++m) {
        a += Minv[size_t(i) * Np + m] * Lr[size_t(q) * Np + m];
        b += Minv[size_t(i) * Np + m] * Ls[size_t(q) * Np + m];
      }
      Pr[size_t(i) * Nc + q] = a * wq[q];
      Ps[size_t(i) * Nc + q] = b * wq[q];
    }
  // face cubature: Gauss-Legendre in the face parameter t, interpolated from the
  // Gauss-Lobatto face nodes
  const std::vector<double> t = lobatto_points(N);
  std::vector<double> tk, wk;
  gauss_jacobi(nc, 0.0, 0.0, tk, wk);
  std::vector<double> I1(size_t(nc) * Nfp);
  for (int k = 0; k < nc; ++k)
    for (int a = 0; a < Nfp; ++a) {
      double l = 1.0;
      for (int b = 0; b < Nfp; ++b)
        if (b != a) l *= (tk[k] - t[b]) / (t[a] - t[b]);
      I1[size_t(k) * Nfp + a] = l;
    }
  std::vector<double> Lc(size_t(Np) * 3 * nc, 0.0);
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < nc; ++k)
      for (int a = 0; a < Nfp; ++a) {
        const int node = R.fmask[f * Nfp + a];
        for (int i = 0; i < Np; ++i)
          Lc[size_t(i) * 3 * nc + f * nc + k] += Minv[size_t(i) * Np + node] * I1[size_t(k) * Nfp + a] * wk[k];
      }
  std::vector<double> buf;
  auto put = [&](size_t& off, const std::vector<double>& v) {
    off = buf.size();
    buf.insert(buf.end(), v.begin(), v.end());
  };
  put(L.Iq, Iq);
  put(L.Pr, Pr);
  put(L.Ps, Ps);
  put(L.I1, I1);
  put(L.Lc, Lc);
  put(L.M, R.M);
  put(L.Minv, Minv);
  put(L.Dr, R.Dr);
  put(L.Ds, R.Ds);
  put(L.Mf, R.Mf);
  L.total = buf.size();
  return buf;
}

struct GeoF {
  double rx, sx, ry, sy, J;
};

__device__ __forceinline__ GeoF load_geo(const double* geo, int64_t e) {
  GeoF g;
  g.rx = geo[4 * e + 0];
  g.sx = geo[4 * e + 1];
  g.ry = geo[4 * e + 2];
  g.sy = geo[4 * e + 3];
  g.J = 1.0 / (g.rx * g.sy - g.ry * g.sx);
  return g;
}

// outward unit normal and sJ/J of face f (affine triangle)
__device__ __forceinline__ void face_n(const GeoF& g, int f, double& nx, double& ny, double& sjj) {
  double gx, gy;
  if (f == 0) { gx = -g.sx; gy = -g.sy; }
  else if (f == 1) { gx = g.rx + g.sx; gy = g.ry + g.sy; }
  else { gx = -g.rx; gy = -g.ry; }
  sjj = sqrt(gx * gx + gy * gy);
  nx = gx / sjj;
  ny = gy / sjj;
}

constexpr int kAdvThreads = 256;

// Advection right-hand side -N~(Ubar, U~) and one LSERK stage:
//   res = a res + dts * rhs;  Ut_out = Ut_in + b res.
// Ubar = ca U^n + cb U^{n-1}. Fields are [2][K][Np].
template <int N>
__global__ void __launch_bounds__(kAdvThreads)
    advect_kernel(int64_t K, const double* __restrict__ geo, const int32_t* __restrict__ conn,
                  const double* __restrict__ ops, AdvLayout L, const double* __restrict__ Un,
                  const double* __restrict__ Unm1, double ca, double cb, const double* __restrict__ Ut_in,
                  double* __restrict__ Ut_out, double* __restrict__ res, const double* __restrict__ gU, double a,
                  double b, double dts) {
  constexpr int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1;
  constexpr int nc = (3 * N + 2) / 2, Nc = nc * nc;
  constexpr int E = (2 * Nc) >= 512 ? 1 : (512 / (2 * Nc) < 1 ? 1 : 512 / (2 * Nc));
  __shared__ double sf[E][4][Np];          // ubar, vbar, ut, vt
  __shared__ double sp[E][4][3 * Nfp];     // exterior traces of the same four fields
  __shared__ double sA[E][4][Nc];          // Au, Bu, Av, Bv at cubature points
  __shared__ double sF[E][2][3 * nc];      // (sJ/J) n.F* at face cubature points
  __shared__ GeoF sg[E];
  const size_t fs = size_t(K) * Np;        // component stride
  const int tid = threadIdx.x;
  const int64_t e0 = int64_t(blockIdx.x) * E;
  const int ne = int((K - e0) < E ? (K - e0) : E);
  if (ne <= 0) return;
  for (int idx = tid; idx < ne * 4 * Np; idx += kAdvThreads) {
    const int e = idx / (4 * Np), r = idx - e * 4 * Np, c = r / Np, i = r - c * Np;
    const size_t gi = size_t(e0 + e) * Np + i;
    double v;
    if (c < 2) v = ca * Un[c * fs + gi] + (cb != 0.0 ? cb * Unm1[c * fs + gi] : 0.0);
    else v = Ut_in[(c - 2) * fs + gi];
    sf[e][c][i] = v;
  }
  for (int e = tid; e < ne; e += kAdvThreads) sg[e] = load_geo(geo, e0 + e);
  for (int idx = tid; idx < ne * 3 * Nfp; idx += kAdvThreads) {
    const int e = idx / (3 * Nfp), q = idx - e * 3 * Nfp, f = q / Nfp, j = q - f * Nfp;
    const int64_t ge = e0 + e;
    const int code = conn[3 * ge + f];
    const int kl = fnode_i(N, f, j);
    double v[4];
    if (code >= 0) {
      const int64_t nb = code >> 2;
      const int kn = fnode_i(N, code & 3, Nfp - 1 - j);
      const size_t gi = size_t(nb) * Np + kn;
      for (int c = 0; c < 2; ++c) v[c] = ca * Un[c * fs + gi] + (cb != 0.0 ? cb * Unm1[c * fs + gi] : 0.0);
      for (int c = 0; c < 2; ++c) v[2 + c] = Ut_in[c * fs + gi];
    } else if (code == -2) {  // velocity Dirichlet: exterior state is the boundary datum
      const size_t gi = size_t(ge) * Np + kl;
      v[0] = v[2] = gU[gi];
      v[1] = v[3] = gU[fs + gi];
    } else {                  // Neumann: exterior = interior
      const size_t gi = size_t(ge) * Np + kl;
      for (int c = 0; c < 2; ++c) v[c] = ca * Un[c * fs + gi] + (cb != 0.0 ? cb * Unm1[c * fs + gi] : 0.0);
      for (int c = 0; c < 2; ++c) v[2 + c] = Ut_in[c * fs + gi];
    }
    for (int c = 0; c < 4; ++c) sp[e][c][q] = v[c];
  }
  __syncthreads();
  const double* Iq = ops + L.Iq;
  const double* I1 = ops + L.I1;
  // volume fluxes at the cubature points, already combined with G^e
  for (int idx = tid; idx < ne * (Nc + 3 * nc); idx += kAdvThreads) {
    if (idx < ne * Nc) {
      const int e = idx / Nc, q = idx - e * Nc;
      double w[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j = 0; j < Np; ++j) {
        const double iq = __ldg(Iq + size_t(q) * Np + j);
        for (int c = 0; c < 4; ++c) w[c] += iq * sf[e][c][j];
      }
      const GeoF g = sg[e];
      for (int c = 0; c < 2; ++c) {
        const double Fx = w[0] * w[2 + c], Fy = w[1] * w[2 + c];
        sA[e][2 * c + 0][q] = g.rx * Fx + g.ry * Fy;
        sA[e][2 * c + 1][q] = g.sx * Fx + g.sy * Fy;
      }
    } else {
      const int r = idx - ne * Nc;
      const int e = r / (3 * nc), q = r - e * 3 * nc, f = q / nc, k = q - f * nc;
      double m[4] = {0, 0, 0, 0}, p[4] = {0, 0, 0, 0};
      for (int a2 = 0; a2 < Nfp; ++a2) {
        const double i1 = __ldg(I1 + size_t(k) * Nfp + a2);
        const int kl = fnode_i(N, f, a2);
        for (int c = 0; c < 4; ++c) {
          m[c] += i1 * sf[e][c][kl];
          p[c] += i1 * sp[e][c][f * Nfp + a2];
        }
      }
      double nx, ny, sjj;
      face_n(sg[e], f, nx, ny, sjj);
      const double unm = nx * m[0] + ny * m[1], unp = nx * p[0] + ny * p[1];
      const double lam = fmax(fabs(unm), fabs(unp));
      for (int c = 0; c < 2; ++c)
        sF[e][c][q] = sjj * (0.5 * (unm * m[2 + c] + unp * p[2 + c]) + 0.5 * lam * (m[2 + c] - p[2 + c]));
    }
  }
  __syncthreads();
  const double* Pr = ops + L.Pr;
  const double* Ps = ops + L.Ps;
  const double* Lc = ops + L.Lc;
  for (int idx = tid; idx < ne * Np; idx += kAdvThreads) {
    const int e = idx / Np, i = idx - e * Np;
    double r0 = 0.0, r1 = 0.0;
    for (int q = 0; q < Nc; ++q) {
      const double pr = __ldg(Pr + size_t(i) * Nc + q), ps = __ldg(Ps + size_t(i) * Nc + q);
      r0 += pr * sA[e][0][q] + ps * sA[e][1][q];
      r1 += pr * sA[e][2][q] + ps * sA[e][3][q];
    }
    for (int q = 0; q < 3 * nc; ++q) {
      const double lc = __ldg(Lc + size_t(i) * 3 * nc + q);
      r0 -= lc * sF[e][0][q];
      r1 -= lc * sF[e][1][q];
    }
    const size_t gi = size_t(e0 + e) * Np + i;
    const double s0 = a * res[gi] + dts * r0;
    const double s1 = a * res[fs + gi] + dts * r1;
    res[gi] = s0;
    res[fs + gi] = s1;
    Ut_out[gi] = Ut_in[gi] + b * s0;
    Ut_out[fs + gi] = Ut_in[fs + gi] + b * s1;
  }
}

// Weak gradient (two components) or weak divergence with central fluxes.
// mode 0: out[c] = (l_i, d_c p) + 1/2 (l_i, n_c [p]);  p* = g on Dirichlet, p- on Neumann faces.
// mode 1: out    = (l_i, div U) + 1/2 (l_i, n.[U]);     u* = g on Dirichlet, u- on Neumann faces.
__global__ void grad_div_kernel(int mode, int N, int64_t K, const double* __restrict__ geo,
                                const int32_t* __restrict__ conn, const double* __restrict__ ops, AdvLayout L,
                                const double* __restrict__ in, const double* __restrict__ g,
                                double* __restrict__ out) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1;
  const int64_t e = blockIdx.x;
  const int i = threadIdx.x;
  const size_t fs = size_t(K) * Np;
  extern __shared__ double sh[];
  double* s_in = sh;            // [2][Np]
  double* s_d = sh + 2 * Np;    // [2][Np]: mode 0: px, py; mode 1: div (first row)
  const int ncomp = mode == 0 ? 1 : 2;
  if (i < Np)
    for (int c = 0; c < ncomp; ++c) s_in[c * Np + i] = in[c * fs + size_t(e) * Np + i];
  __syncthreads();
  const GeoF gf = load_geo(geo, e);
  const double* Dr = ops + L.Dr;
  const double* Ds = ops + L.Ds;
  const double* M = ops + L.M;
  const double* Mf = ops + L.Mf;
  if (i < Np) {
    double ar[2] = {0, 0}, as[2] = {0, 0};
    for (int j = 0; j < Np; ++j)
      for (int c = 0; c < ncomp; ++c) {
        ar[c] += Dr[size_t(i) * Np + j] * s_in[c * Np + j];
        as[c] += Ds[size_t(i) * Np + j] * s_in[c * Np + j];
      }
    if (mode == 0) {
      s_d[i] = gf.rx * ar[0] + gf.sx * as[0];
      s_d[Np + i] = gf.ry * ar[0] + gf.sy * as[0];
    } else {
      s_d[i] = gf.rx * ar[0] + gf.sx * as[0] + gf.ry * ar[1] + gf.sy * as[1];
    }
  }
  __syncthreads();
  if (i >= Np) return;
  double w[2] = {0, 0};
  for (int j = 0; j < Np; ++j) {
    w[0] += M[size_t(i) * Np + j] * s_d[j];
    if (mode == 0) w[1] += M[size_t(i) * Np + j] * s_d[Np + j];
  }
  w[0] *= gf.J;
  w[1] *= gf.J;
  // face terms on the faces this node lies on
  int row = 0, rs = 0;
  while (i >= rs + (N + 1 - row)) {
    rs += N + 1 - row;
    ++row;
  }
  const int col = i - rs;
  for (int f = 0; f < 3; ++f) {
    int a = -1;
    if (f == 0 && row == 0) a = col;
    if (f == 1 && col == N - row) a = row;
    if (f == 2 && col == 0) a = N - row;
    if (a < 0) continue;
    const int code = conn[3 * e + f];
    if (code == -3) continue;  // Neumann: p* = p-, u* = u-: no jump
    double nx, ny, sjj;
    face_n(gf, f, nx, ny, sjj);
    const double sJ = sjj * gf.J;
    double acc[2] = {0, 0};
    for (int b = 0; b < Nfp; ++b) {
      const int kl = fnode_i(N, f, b);
      double jmp[2];
      for (int c = 0; c < ncomp; ++c) {
        const double vm = s_in[c * Np + kl];
        if (code >= 0) {
          const int kn = fnode_i(N, code & 3, Nfp - 1 - b);
          jmp[c] = in[c * fs + size_t(code >> 2) * Np + kn] - vm;
        } else {  // Dirichlet: value* = g  ->  exterior = 2 g - interior
          jmp[c] = 2.0 * (g[c * fs + size_t(e) * Np + kl] - vm);
        }
      }
      const double mfab = Mf[size_t(a) * Nfp + b];
      if (mode == 0) acc[0] += mfab * jmp[0];
      else acc[0] += mfab * (nx * jmp[0] + ny * jmp[1]);
    }
    if (mode == 0) {
      w[0] += 0.5 * sJ * nx * acc[0];
      w[1] += 0.5 * sJ * ny * acc[0];
    } else {
      w[0] += 0.5 * sJ * acc[0];
    }
  }
  out[size_t(e) * Np + i] = w[0];
  if (mode == 0) out[fs + size_t(e) * Np + i] = w[1];
}

// out[c] = (J M)^{-1} w[c] per element, for nc components
__global__ void strong_kernel(int Np, int64_t K, int ncomp, const double* __restrict__ geo,
                              const double* __restrict__ Minv, const double* __restrict__ w, double* __restrict__ out) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(ncomp) * K * Np) return;
  const int64_t ce = idx / Np;
  const int i = int(idx - ce * Np);
  const int64_t e = ce % K;
  const double J = 1.0 / (geo[4 * e] * geo[4 * e + 3] - geo[4 * e + 2] * geo[4 * e + 1]);
  const double* we = w + ce * Np;
  double acc = 0.0;
  for (int j = 0; j < Np; ++j) acc += Minv[size_t(i) * Np + j] * we[j];
  out[idx] = acc / J;
}

// y = a x + b y (n entries); with x2: y = a x + b y + c x2
// y = a x + b y + c x2; with b = 0 the old y is not read (it may be uninitialised)
__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y,
                             double c, const double* __restrict__ x2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = a * x[i] + (b != 0.0 ? b * y[i] : 0.0) + (x2 ? c * x2[i] : 0.0);
}

inline int eg(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return int(b < 1 ? 1 : b);
}

template <int N>
cudaError_t launch_advect_n(const dg_mesh* m, InsWorkspace* w, const double* Un, const double* Unm1, double ca,
                            double cb, const double* Ut_in, double* Ut_out, const double* gU, double a, double b,
                            double dts, cudaStream_t st) {
  constexpr int nc = (3 * N + 2) / 2, Nc = nc * nc;
  constexpr int E = (2 * Nc) >= 512 ? 1 : (512 / (2 * Nc) < 1 ? 1 : 512 / (2 * Nc));
  const int blocks = int((m->K + E - 1) / E);
  advect_kernel<N><<<blocks, kAdvThreads, 0, st>>>(m->K, m->geo64, m->conn, w->ops, w->L, Un, Unm1, ca, cb, Ut_in,
                                                   Ut_out, w->res, gU, a, b, dts);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_advect(const dg_mesh* m, InsWorkspace* w, const double* Un, const double* Unm1, double ca,
                          double cb, const double* Ut_in, double* Ut_out, const double* gU, double a, double b,
                          double dts, cudaStream_t st) {
  switch (m->N) {
#define CASE(n) \
  case n: return launch_advect_n<n>(m, w, Un, Unm1, ca, cb, Ut_in, Ut_out, gU, a, b, dts, st);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------- tensor-core advection stage
// The stage of advect_kernel split at its two dense contractions, which run as
// sliced FP64 products on the tensor cores (sliced_gemm):
//   X = [Ubar_x; Ubar_y; Ut_x; Ut_y]            rows (c K + e), Np each
//   W = Iq X                                     rows (c K + e), Nc each
//   Y = [ G.F at the volume points | (sJ/J) n.F* at the face points ]   rows (c K + e)
//   R = Pr Y_r + Ps Y_s - Lc Y_F                 rows (c K + e), Np each: the rhs
//       (three sliced products, summed in FP64 by the update)
// then the LSERK update. Arithmetic and layout as in advect_kernel.
__global__ void k_adv_gather(int64_t n1, const double* __restrict__ Un, const double* __restrict__ Unm1, double ca,
                             double cb, const double* __restrict__ Ut_in, double* __restrict__ X) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < 4 * n1; i += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(i / n1);
    const int64_t j = i - c * n1;
    X[i] = c < 2 ? ca * Un[c * n1 + j] + (cb != 0.0 ? cb * Unm1[c * n1 + j] : 0.0) : Ut_in[(c - 2) * n1 + j];
  }
}

// one thread per volume cubature point (e, q) or face cubature point (e, f, k)
__global__ void k_adv_flux(int N, int64_t K, const double* __restrict__ geo, const int32_t* __restrict__ conn,
                           const double* __restrict__ I1, const double* __restrict__ X, const double* __restrict__ W,
                           const double* __restrict__ gU, double* __restrict__ Y) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, nc = (3 * N + 2) / 2, Nc = nc * nc;
  const int KY = 2 * Nc + 3 * nc;
  const int64_t nvol = K * Nc, total = nvol + K * 3 * nc;
  const size_t fsX = size_t(K) * Np, fsW = size_t(K) * Nc, fsY = size_t(K) * KY;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    if (idx < nvol) {
      const int64_t e = idx / Nc;
      const int q = int(idx - e * Nc);
      const GeoF g = load_geo(geo, e);
      double w[4];
      for (int c = 0; c < 4; ++c) w[c] = W[c * fsW + size_t(e) * Nc + q];
      for (int c = 0; c < 2; ++c) {
        const double Fx = w[0] * w[2 + c], Fy = w[1] * w[2 + c];
        Y[c * fsY + size_t(e) * KY + q] = g.rx * Fx + g.ry * Fy;
        Y[c * fsY + size_t(e) * KY + Nc + q] = g.sx * Fx + g.sy * Fy;
      }
    } else {
      const int64_t r = idx - nvol;
      const int64_t e = r / (3 * nc);
      const int q = int(r - e * 3 * nc), f = q / nc, k = q - f * nc;
      const GeoF g = load_geo(geo, e);
      const int code = conn[3 * e + f];
      double m[4] = {0, 0, 0, 0}, p[4] = {0, 0, 0, 0};
      for (int a2 = 0; a2 < Nfp; ++a2) {
        const double i1 = I1[size_t(k) * Nfp + a2];
        const int kl = fnode_i(N, f, a2);
        double vm[4], vp[4];
        for (int c = 0; c < 4; ++c) vm[c] = X[c * fsX + size_t(e) * Np + kl];
        if (code >= 0) {
          const int64_t nb = code >> 2;
          const int kn = fnode_i(N, code & 3, Nfp - 1 - a2);
          for (int c = 0; c < 4; ++c) vp[c] = X[c * fsX + size_t(nb) * Np + kn];
        } else if (code == -2) {  // velocity Dirichlet: exterior state is the boundary datum
          const size_t gi = size_t(e) * Np + kl;
          vp[0] = vp[2] = gU[gi];
          vp[1] = vp[3] = gU[fsX + gi];
        } else {                  // Neumann: exterior = interior
          for (int c = 0; c < 4; ++c) vp[c] = vm[c];
        }
        for (int c = 0; c < 4; ++c) {
          m[c] += i1 * vm[c];
          p[c] += i1 * vp[c];
        }
      }
      double nx, ny, sjj;
      face_n(g, f, nx, ny, sjj);
      const double unm = nx * m[0] + ny * m[1], unp = nx * p[0] + ny * p[1];
      const double lam = fmax(fabs(unm), fabs(unp));
      for (int c = 0; c < 2; ++c)
        Y[c * fsY + size_t(e) * KY + 2 * Nc + q] =
            sjj * (0.5 * (unm * m[2 + c] + unp * p[2 + c]) + 0.5 * lam * (m[2 + c] - p[2 + c]));
    }
  }
}

// rhs = R_r + R_s + R_lift (the three projection blocks, each n entries);
// res = a res + dts rhs; Ut_out = Ut_in + b res  (n = 2 K Np)
__global__ void k_adv_update(int64_t n, const double* __restrict__ R, double a, double dts, double b,
                             const double* __restrict__ Ut_in, double* __restrict__ res, double* __restrict__ Ut_out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double r = a * res[i] + dts * (R[i] + R[n + i] + R[2 * n + i]);
    res[i] = r;
    Ut_out[i] = Ut_in[i] + b * r;
  }
}

#define ICK(x)                         \
  do {                                 \
    cudaError_t e_ = (x);              \
    if (e_ != cudaSuccess) return e_;  \
  } while (0)

cudaError_t setup_ins(dg_mesh* m) {
  if (m->ins) return cudaSuccess;
  InsWorkspace* w = new InsWorkspace();
  m->ins = w;
  w->K = m->K;
  w->N = m->N;
  const std::vector<double> h = build_adv_ops(m->ref[m->N], w->L);
  auto al = [&](double** p, size_t n) -> cudaError_t {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(double));
    if (e == cudaSuccess) w->allocs.push_back(*p);
    return e;
  };
  const size_t n1 = size_t(m->K) * ((m->N + 1) * (m->N + 2) / 2);
  ICK(al(&w->ops, h.size()));
  ICK(cudaMemcpy(w->ops, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  ICK(al(&w->Ut0, 2 * n1));
  ICK(al(&w->Ut1, 2 * n1));
  ICK(al(&w->res, 2 * n1));
  ICK(al(&w->Uhat, 2 * n1));
  ICK(al(&w->Uhh, 2 * n1));
  ICK(al(&w->bu, 2 * n1));
  ICK(al(&w->G, 2 * n1));
  ICK(al(&w->bp, n1));
  ICK(al(&w->dP, n1));
  ICK(al(&w->tmp, 2 * n1));
  ICK(al(&w->gts, 2 * n1));
  ICK(al(&w->zero, n1));
  ICK(cudaMemset(w->zero, 0, n1 * sizeof(double)));
  ICK(cudaEventCreate(&w->ev0));
  ICK(cudaEventCreate(&w->ev1));
  // degree >= 3: the stage's dense contractions on the tensor cores
  if (m->N >= 3) {
    const AdvLayout& L = w->L;
    const int Np = L.Np, Nc = L.Nc, nc = L.nc, KY = 2 * Nc + 3 * nc;
    const std::vector<double> Iq(h.begin() + L.Iq, h.begin() + L.Iq + size_t(Nc) * Np);
    const std::vector<double> Pr(h.begin() + L.Pr, h.begin() + L.Pr + size_t(Np) * Nc);
    const std::vector<double> Ps(h.begin() + L.Ps, h.begin() + L.Ps + size_t(Np) * Nc);
    std::vector<double> Lc(h.begin() + L.Lc, h.begin() + L.Lc + size_t(Np) * 3 * nc);
    for (double& v : Lc) v = -v;
    ICK(sliced_op_create(Iq, Nc, Np, &w->opIq));
    ICK(sliced_op_create(Pr, Np, Nc, &w->opPr));
    ICK(sliced_op_create(Ps, Np, Nc, &w->opPs));
    ICK(sliced_op_create(Lc, Np, 3 * nc, &w->opLc));
    ICK(al(&w->X, 4 * n1));
    ICK(al(&w->W, 4 * size_t(m->K) * Nc));
    ICK(al(&w->Y, 2 * size_t(m->K) * KY));
    ICK(al(&w->R, 3 * 2 * n1));  // the three projection blocks' results
    w->tensor = true;
  }
  return cudaSuccess;
}

// One LSERK stage of the advection on the tensor cores (see k_adv_gather).
cudaError_t advect_stage_tensor(const dg_mesh* m, InsWorkspace* w, const double* Un, const double* Unm1, double ca,
                                double cb, const double* Ut_in, double* Ut_out, const double* gU, double a, double b,
                                double dts, cudaStream_t st) {
  const AdvLayout& L = w->L;
  const int Np = L.Np, Nc = L.Nc, nc = L.nc, KY = 2 * Nc + 3 * nc;
  const int64_t K = m->K, n1 = K * Np;
  k_adv_gather<<<eg(4 * n1), 256, 0, st>>>(n1, Un, Unm1, ca, cb, Ut_in, w->X);
  note_launch();
  ICK(sliced_gemm(w->opIq, 4 * K, w->X, Np, w->W, Nc, st));
  k_adv_flux<<<eg(K * (Nc + 3 * nc)), 256, 0, st>>>(m->N, K, m->geo64, m->conn, w->ops + L.I1, w->X, w->W, gU, w->Y);
  note_launch();
  ICK(sliced_gemm(w->opPr, 2 * K, w->Y, KY, w->R, Np, st));
  ICK(sliced_gemm(w->opPs, 2 * K, w->Y + Nc, KY, w->R + 2 * n1, Np, st));
  ICK(sliced_gemm(w->opLc, 2 * K, w->Y + 2 * Nc, KY, w->R + 4 * n1, Np, st));
  k_adv_update<<<eg(2 * n1), 256, 0, st>>>(2 * n1, w->R, a, dts, b, Ut_in, w->res, Ut_out);
  note_launch();
  return cudaGetLastError();
}

// Advect U0 (given at t0) to t0 + nsub*dts with LSERK(5,4); result in the
// returned buffer (one of Ut0/Ut1). Ubar(t) = U^n + (t - tn)/dt (U^n - U^{n-1}).
cudaError_t advect_field(const dg_mesh* m, InsWorkspace* w, const dg_ins_state* s, const double* U0, double t0,
                         int nsub, double tn, bool extrap, double** result, cudaStream_t st) {
  const size_t n2 = 2 * size_t(m->K) * ((m->N + 1) * (m->N + 2) / 2);
  const double dts = s->dt / s->Ns;
  ICK(cudaMemcpyAsync(w->Ut0, U0, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ICK(cudaMemsetAsync(w->res, 0, n2 * sizeof(double), st));
  double* cur = w->Ut0;
  double* nxt = w->Ut1;
  double t = t0;
  for (int k = 0; k < nsub; ++k) {
    for (int stg = 0; stg < 5; ++stg) {
      const double ts = t + kRkC[stg] * dts;
      double ca = 1.0, cb = 0.0;
      if (extrap) {
        const double th = (ts - tn) / s->dt;
        ca = 1.0 + th;
        cb = -th;
      }
      const double* g = s->gU;
      if (s->gU_hist) {  // the velocity data at ts, interpolated through t^{n-1}, t^n, t^{n+1}
        const double tau = (ts - tn) / s->dt;
        const double* gn = s->gU_hist;
        if (s->step == 0) {  // t^n, t^{n+1}: linear
          axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, tau, s->gU, 0.0, w->gts, 1.0 - tau, gn); note_launch();
        } else {
          axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, 0.5 * tau * (tau + 1.0), s->gU, 0.0, w->gts, 1.0 - tau * tau, gn);
          note_launch();
          axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, 0.5 * tau * (tau - 1.0), gn + n2, 1.0, w->gts, 0.0, nullptr);
          note_launch();
        }
        g = w->gts;
      }
      if (w->tensor)
        ICK(advect_stage_tensor(m, w, s->U, s->Uold, ca, cb, cur, nxt, g, kRkA[stg], kRkB[stg], dts, st));
      else
        ICK(launch_advect(m, w, s->U, s->Uold, ca, cb, cur, nxt, g, kRkA[stg], kRkB[stg], dts, st));
      std::swap(cur, nxt);
    }
    t += dts;
  }
  *result = cur;
  return cudaSuccess;
}

}  // namespace

cudaError_t ins_run(dg_mesh* mu, dg_mesh* mp, dg_ins_state* s, int nsteps, cudaStream_t st, dg_status& status) {
  status = DG_OK;
  ICK(setup_ins(mu));
  InsWorkspace* w = mu->ins;
  const int Np = (mu->N + 1) * (mu->N + 2) / 2;
  const unsigned gd_threads = unsigned((Np + 31) / 32 * 32);  // grad_div_kernel: one thread per node
  const int64_t K = mu->K;
  const size_t n1 = size_t(K) * Np, n2 = 2 * n1;
  const AdvLayout& L = w->L;
  ICK(cudaEventRecord(w->ev0, st));
  for (int it = 0; it < nsteps; ++it) {
    const int n = s->step;
    const double dt = s->dt, nu = s->nu;
    const double tn = n * dt;
    double gamma;
    // (i) advection of the history into U^
    double* Ut = nullptr;
    if (n == 0) {
      gamma = 1.0;
      ICK(advect_field(mu, w, s, s->U, tn, s->Ns, tn, false, &Ut, st));
      ICK(cudaMemcpyAsync(w->Uhat, Ut, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      gamma = 1.5;
      ICK(advect_field(mu, w, s, s->U, tn, s->Ns, tn, true, &Ut, st));
      axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, 2.0, Ut, 0.0, w->Uhat, 0.0, nullptr); note_launch();
      ICK(advect_field(mu, w, s, s->Uold, tn - dt, 2 * s->Ns, tn, true, &Ut, st));
      axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, -0.5, Ut, 1.0, w->Uhat, 0.0, nullptr); note_launch();
    }
    // (ii) velocity Helmholtz: b = J M U^/(nu dt) - L(gU) - (1/nu) G P^n
    axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, 1.0 / (nu * dt), w->Uhat, 0.0, w->tmp, 0.0, nullptr); note_launch();
    ICK(launch_rhs(mu, 2, w->tmp, s->gU, w->bu, st));
    grad_div_kernel<<<unsigned(K), gd_threads, 4 * Np * sizeof(double), st>>>(0, mu->N, K, mu->geo64, mp->conn, w->ops, L,
                                                                       s->P, s->gU_hist ? s->gP_n : s->gP, w->G);
    note_launch();
    axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, -1.0 / nu, w->G, 1.0, w->bu, 0.0, nullptr); note_launch();
    ICK(cudaMemcpyAsync(w->Uhh, s->U, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    const double lam = gamma / (nu * dt);
    dg_solve_info info;
    dg_status sv = dg_pcg_solve(mu, &s->vel_opts, 2, lam, w->bu, w->Uhh, &info, st);
    s->vel_iters[0] = info.iters[0];
    s->vel_iters[1] = info.iters[1];
    if (sv != DG_OK) {
      status = sv;
      return cudaSuccess;
    }
    // (iii) pressure increment: b = -(gamma/dt) D.U^^ (zero increment on pressure-Dirichlet faces)
    grad_div_kernel<<<unsigned(K), gd_threads, 4 * Np * sizeof(double), st>>>(1, mu->N, K, mu->geo64, mu->conn, w->ops, L,
                                                                       w->Uhh, s->gU, w->bp);
    note_launch();
    axpby_kernel<<<eg(n1), 256, 0, st>>>(n1, 0.0, w->bp, -gamma / dt, w->bp, 0.0, nullptr); note_launch();
    ICK(cudaMemsetAsync(w->dP, 0, n1 * sizeof(double), st));
    if (s->gU_hist) {  // the increment's Dirichlet data gP - gP_n: b -= L(gP - gP_n)
      axpby_kernel<<<eg(n1), 256, 0, st>>>(n1, 1.0, s->gP, 0.0, w->tmp, -1.0, s->gP_n); note_launch();
      ICK(launch_rhs(mp, 1, w->zero, w->tmp, w->G, st));
      axpby_kernel<<<eg(n1), 256, 0, st>>>(n1, 1.0, w->G, 1.0, w->bp, 0.0, nullptr); note_launch();
    } else {
      ICK(cudaMemsetAsync(w->tmp, 0, n1 * sizeof(double), st));
    }
    sv = dg_pcg_solve(mp, &s->pr_opts, 1, 0.0, w->bp, w->dP, &info, st);
    s->pr_iters = info.iters[0];
    if (sv != DG_OK) {
      status = sv;
      return cudaSuccess;
    }
    // (iv) U^{n+1} = U^^ - (dt/gamma) (J M)^{-1} G dP ; P += dP ; history shift
    grad_div_kernel<<<unsigned(K), gd_threads, 4 * Np * sizeof(double), st>>>(0, mu->N, K, mu->geo64, mp->conn, w->ops, L,
                                                                       w->dP, w->tmp, w->G);
    note_launch();
    strong_kernel<<<unsigned((n2 + 255) / 256), 256, 0, st>>>(Np, K, 2, mu->geo64, w->ops + L.Minv, w->G, w->bu);
    note_launch();
    ICK(cudaMemcpyAsync(s->Uold, s->U, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    axpby_kernel<<<eg(n2), 256, 0, st>>>(n2, 1.0, w->Uhh, 0.0, s->U, -dt / gamma, w->bu); note_launch();
    axpby_kernel<<<eg(n1), 256, 0, st>>>(n1, 1.0, w->dP, 1.0, s->P, 0.0, nullptr); note_launch();
    s->step = n + 1;
  }
  ICK(cudaEventRecord(w->ev1, st));
  ICK(cudaEventSynchronize(w->ev1));
  float ms = 0.f;
  ICK(cudaEventElapsedTime(&ms, w->ev0, w->ev1));
  s->ms = ms;
  return cudaGetLastError();
}

}  // namespace dgx

extern "C" dg_status dg_ins_step(dg_mesh* mu, dg_mesh* mp, dg_ins_state* s, int nsteps, void* stream) {
  using namespace dgx;
  if (!mu || !mp || !s) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (!s->U || !s->Uold || !s->P || !s->gU || !s->gP) { set_error("NULL field in dg_ins_state"); return DG_ERR_ARG; }
  if (mu->N != mp->N || mu->K != mp->K || mu->EToV != mp->EToV || mu->geo_h != mp->geo_h) {
    set_error("mesh_u and mesh_p must be the same triangulation and degree");
    return DG_ERR_ARG;
  }
  if (!(s->nu > 0) || !(s->dt > 0) || s->Ns < 1 || s->step < 0 || nsteps < 0) {
    set_error("need nu > 0, dt > 0, Ns >= 1, step >= 0, nsteps >= 0");
    return DG_ERR_ARG;
  }
  if (s->gU_hist && (!s->gP_n || nsteps > 1)) {
    set_error("time-dependent boundary data (gU_hist) need gP_n and one step per call");
    return DG_ERR_ARG;
  }
  try {
    dg_status status = DG_OK;
    cudaError_t e = ins_run(mu, mp, s, nsteps, (cudaStream_t)stream, status);
    if (e != cudaSuccess) {
      set_error(std::string("dg_ins_step: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    }
    return status;
  } catch (const std::exception& ex) {
    set_error(ex.what());
    return DG_ERR_ARG;
  }
}
