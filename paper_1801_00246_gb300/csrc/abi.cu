// C ABI entry points: mesh setup, operator applies, right-hand side, nodes,
// and the small per-element kernels they need (Jacobi diagonal, Dirichlet
// right-hand side). The operator is the SIPDG form of Section 5.2
// (Eq. ellipticOp1, evaluated as Eq. ellipticOp3); the right-hand side carries
// the Dirichlet data of Eq. DirichletBC; the diagonal feeds the Jacobi
// preconditioner of Section 3.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dgx {
bool compute_geometry(dg_mesh* m, std::string& err);
bool compute_connectivity(dg_mesh* m, const int8_t* bc, std::string& err);
bool check_face_matching(const dg_mesh* m, std::string& err);
void node_coordinates(const dg_mesh* m, int degree, std::vector<double>& x, std::vector<double>& y);
const char* last_error();
void free_workspace(dg_mesh* m);
void free_ins_workspace(dg_mesh* m);

size_t ops_count(int N) {
  const size_t Np = size_t(N + 1) * (N + 2) / 2, Nfp = N + 1;
  return 6 * Np * Np + Nfp * Nfp + 4 * Np + 6 * Nfp;
}

// Offsets (in entries) of the pieces of the operator buffer.
struct OpsLayout {
  size_t Dr, Ds, Br, Bs, M, Mf, drr, drs, dss, dm, fcr, fcs, Minv;
  explicit OpsLayout(int N) {
    const size_t Np = size_t(N + 1) * (N + 2) / 2, Nfp = N + 1;
    Dr = 0;
    Ds = Np * Np;
    Br = 2 * Np * Np;
    Bs = 3 * Np * Np;
    M = 4 * Np * Np;
    Mf = 5 * Np * Np;
    drr = Mf + Nfp * Nfp;
    drs = drr + Np;
    dss = drs + Np;
    dm = dss + Np;
    fcr = dm + Np;
    fcs = fcr + 3 * Nfp;
    Minv = fcs + 3 * Nfp;
  }
};

cudaError_t ensure_ops(dg_mesh* m, int degree) {
  if (m->ops64[degree].buf) return cudaSuccess;
  if (m->ref[degree].N == 0) m->ref[degree] = build_reference(degree);
  const RefElem& R = m->ref[degree];
  const OpsLayout L(degree);
  const size_t n = ops_count(degree);
  std::vector<double> h(n, 0.0);
  auto put = [&](size_t off, const std::vector<double>& v) { std::memcpy(&h[off], v.data(), v.size() * sizeof(double)); };
  put(L.Dr, R.Dr);
  put(L.Ds, R.Ds);
  put(L.Br, R.Br);
  put(L.Bs, R.Bs);
  put(L.M, R.M);
  put(L.Mf, R.Mf);
  put(L.drr, R.diag_rr);
  put(L.drs, R.diag_rs);
  put(L.dss, R.diag_ss);
  put(L.dm, R.diag_m);
  put(L.fcr, R.face_cr);
  put(L.fcs, R.face_cs);
  put(L.Minv, invert(R.Np, R.M));
  std::vector<float> hf(n);
  for (size_t i = 0; i < n; ++i) hf[i] = float(h[i]);
  cudaError_t err = cudaMalloc(&m->ops64[degree].buf, n * sizeof(double));
  if (err != cudaSuccess) return err;
  err = cudaMalloc(&m->ops32[degree].buf, n * sizeof(float));
  if (err != cudaSuccess) return err;
  m->ops64[degree].bytes = n * sizeof(double);
  m->ops32[degree].bytes = n * sizeof(float);
  err = cudaMemcpy(m->ops64[degree].buf, h.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return err;
  return cudaMemcpy(m->ops32[degree].buf, hf.data(), n * sizeof(float), cudaMemcpyHostToDevice);
}

namespace {

__device__ __forceinline__ int fnode_rt(int N, int f, int j) {
  auto rs = [N](int row) { return row * (N + 1) - row * (row - 1) / 2; };
  return f == 0 ? j : (f == 1 ? rs(j) + (N - j) : rs(N - j));
}

// Face geometry of face f from the element's (r_x, s_x, r_y, s_y).
template <typename T>
__device__ __forceinline__ void face_geo(const T* g, int f, T& sJ, T& nr, T& ns, T& gn) {
  const T rx = g[0], sx = g[1], ry = g[2], sy = g[3];
  const T J = T(1) / (rx * sy - ry * sx);
  T gx, gy;
  if (f == 0) { gx = -sx; gy = -sy; }
  else if (f == 1) { gx = rx + sx; gy = ry + sy; }
  else { gx = -rx; gy = -ry; }
  gn = sqrt(gx * gx + gy * gy);
  const T nx = gx / gn, ny = gy / gn;
  sJ = J * gn;
  nr = nx * rx + ny * ry;
  ns = nx * sx + ny * sy;
}

template <typename T>
__device__ __forceinline__ T face_tau(const T* geo, const int32_t* conn, int64_t e, int f, T gn, T cpen) {
  const int c = conn[3 * e + f];
  if (c < 0) return cpen * gn;
  T sJ2, nr2, ns2, hn;
  face_geo(geo + 4 * (int64_t(c) >> 2), c & 3, sJ2, nr2, ns2, hn);
  return cpen * (gn > hn ? gn : hn);
}

// diag(A) per node: volume stiffness diagonal + lambda J M_ii + face terms of
// the element's own block (weight 1 interior, 2 Dirichlet, 0 Neumann).
template <typename T>
__global__ void diagonal_kernel(int N, int64_t K, const T* __restrict__ geo, const int32_t* __restrict__ conn,
                                const T* __restrict__ ops, OpsLayout L, T lambda, T* __restrict__ diag) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1;
  const T cpen = T((N + 1) * (N + 2)) / T(2);
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= K * Np) return;
  const int64_t e = idx / Np;
  const int i = int(idx - e * Np);
  const T* g = geo + 4 * e;
  const T rx = g[0], sx = g[1], ry = g[2], sy = g[3];
  const T J = T(1) / (rx * sy - ry * sx);
  T d = J * ((rx * rx + ry * ry) * ops[L.drr + i] + (rx * sx + ry * sy) * ops[L.drs + i] +
             (sx * sx + sy * sy) * ops[L.dss + i]) +
        lambda * J * ops[L.dm + i];
  for (int f = 0; f < 3; ++f)
    for (int a = 0; a < Nfp; ++a) {
      if (fnode_rt(N, f, a) != i) continue;
      const int c = conn[3 * e + f];
      const T w = c >= 0 ? T(1) : (c == -2 ? T(2) : T(0));
      if (w == T(0)) continue;
      T sJ, nr, ns, gn;
      face_geo(g, f, sJ, nr, ns, gn);
      const T tau = face_tau(geo, conn, e, f, gn, cpen);
      d += w * sJ * (-(nr * ops[L.fcr + f * Nfp + a] + ns * ops[L.fcs + f * Nfp + a]) +
                     tau * ops[L.Mf + size_t(a) * Nfp + a]);
    }
  diag[idx] = d;
}

// b = J M f - L(g), L(g)_i = sum_{Dirichlet f} (n.grad l_i, g)_f - 2 tau (l_i, g)_f.
__global__ void rhs_kernel(int N, int64_t K, int B, const double* __restrict__ geo, const int32_t* __restrict__ conn,
                           const double* __restrict__ ops, OpsLayout L, const double* __restrict__ fv,
                           const double* __restrict__ gv, double* __restrict__ bv) {
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1;
  const double cpen = double((N + 1) * (N + 2)) / 2.0;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(B) * K * Np) return;
  const int64_t be = idx / Np;
  const int i = int(idx - be * Np);
  const int64_t e = be % K;
  const double* g = geo + 4 * e;
  const double J = 1.0 / (g[0] * g[3] - g[2] * g[1]);
  const double* fe = fv + be * Np;
  double acc = 0.0;
  for (int j = 0; j < Np; ++j) acc += ops[L.M + size_t(i) * Np + j] * fe[j];
  acc *= J;
  if (gv) {
    const double* ge = gv + be * Np;
    for (int f = 0; f < 3; ++f) {
      if (conn[3 * e + f] != -2) continue;
      double sJ, nr, ns, gn;
      face_geo(g, f, sJ, nr, ns, gn);
      const double tau = cpen * gn;
      for (int a = 0; a < Nfp; ++a) {
        double mg = 0.0;
        for (int c = 0; c < Nfp; ++c) mg += ops[L.Mf + size_t(a) * Nfp + c] * ge[fnode_rt(N, f, c)];
        mg *= sJ;
        const int ka = fnode_rt(N, f, a);
        double lg = (nr * ops[L.Dr + size_t(ka) * Np + i] + ns * ops[L.Ds + size_t(ka) * Np + i]) * mg;
        if (ka == i) lg -= 2.0 * tau * mg;
        acc -= lg;
      }
    }
  }
  bv[idx] = acc;
}

}  // namespace

cudaError_t launch_diagonal(const dg_mesh* m, int degree, dg_prec prec, double lambda, void* diag, cudaStream_t st) {
  const int Np = (degree + 1) * (degree + 2) / 2;
  const int64_t n = m->K * Np;
  const int blocks = int((n + 255) / 256);
  const OpsLayout L(degree);
  if (prec == DG_F64) {
    diagonal_kernel<double><<<blocks, 256, 0, st>>>(degree, m->K, m->geo64, m->conn,
                                                     (const double*)m->ops64[degree].buf, L, lambda, (double*)diag);
  } else {
    diagonal_kernel<float><<<blocks, 256, 0, st>>>(degree, m->K, m->geo32, m->conn,
                                                    (const float*)m->ops32[degree].buf, L, float(lambda), (float*)diag);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rhs(const dg_mesh* m, int B, const double* f, const double* g, double* b, cudaStream_t st) {
  const int Np = (m->N + 1) * (m->N + 2) / 2;
  const int64_t n = int64_t(B) * m->K * Np;
  const OpsLayout L(m->N);
  rhs_kernel<<<int((n + 255) / 256), 256, 0, st>>>(m->N, m->K, B, m->geo64, m->conn, (const double*)m->ops64[m->N].buf,
                                                   L, f, g, b); note_launch();
  return cudaGetLastError();
}

}  // namespace dgx

using namespace dgx;

#define DG_TRY_BEGIN try {
#define DG_TRY_END                                    \
  }                                                   \
  catch (const std::bad_alloc&) {                     \
    set_error("host allocation failed");              \
    return DG_ERR_OOM;                                \
  }                                                   \
  catch (const std::exception& ex) {                  \
    set_error(ex.what());                             \
    return DG_ERR_ARG;                                \
  }

static dg_status cuda_fail(cudaError_t err, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(err));
  return err == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

extern "C" {

uint64_t dg_launch_count(void) { return launch_count(); }

const char* dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_OOM: return "out of memory";
    case DG_ERR_NOT_CONVERGED: return "not converged";
    case DG_ERR_BREAKDOWN: return "Krylov breakdown";
    case DG_ERR_TIMEOUT: return "device wait timed out";
    case DG_ERR_MESH: return "invalid mesh";
  }
  return "unknown status";
}

const char* dg_last_error(void) { return last_error(); }

dg_status dg_mesh_setup(int N, int64_t Nv, const double* VX, const double* VY, int64_t K, const int32_t* EToV,
                        const int8_t* bc, void* stream, dg_mesh** out) {
  (void)stream;
  if (!out) { set_error("out is NULL"); return DG_ERR_ARG; }
  *out = nullptr;
  if (N < 1 || N > kMaxN) { set_error("degree N must be in 1..10"); return DG_ERR_ARG; }
  if (Nv < 3 || K < 1 || !VX || !VY || !EToV || !bc) { set_error("empty mesh or NULL array"); return DG_ERR_ARG; }
  if (K > (int64_t(1) << 29)) { set_error("K too large"); return DG_ERR_ARG; }
  DG_TRY_BEGIN
  for (int64_t i = 0; i < 3 * K; ++i)
    if (EToV[i] < 0 || EToV[i] >= Nv) { set_error("EToV entry out of range"); return DG_ERR_ARG; }
  dg_mesh* m = new dg_mesh();
  m->N = N;
  m->K = K;
  m->Nv = Nv;
  m->VX.assign(VX, VX + Nv);
  m->VY.assign(VY, VY + Nv);
  m->EToV.assign(EToV, EToV + 3 * K);
  std::string err;
  if (!compute_geometry(m, err) || !compute_connectivity(m, bc, err)) {
    delete m;
    set_error(err);
    return DG_ERR_MESH;
  }
  m->ref[N] = build_reference(N);
  if (!check_face_matching(m, err)) {
    delete m;
    set_error(err);
    return DG_ERR_MESH;
  }
  cudaError_t ce = cudaMalloc(&m->geo64, sizeof(double) * 4 * K);
  if (ce == cudaSuccess) ce = cudaMalloc(&m->geo32, sizeof(float) * 4 * K);
  if (ce == cudaSuccess) ce = cudaMalloc(&m->conn, sizeof(int32_t) * 3 * K);
  std::vector<float> g32(m->geo_h.begin(), m->geo_h.end());
  if (ce == cudaSuccess) ce = cudaMemcpy(m->geo64, m->geo_h.data(), sizeof(double) * 4 * K, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(m->geo32, g32.data(), sizeof(float) * 4 * K, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(m->conn, m->conn_h.data(), sizeof(int32_t) * 3 * K, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) {
    // 1/h = |grad of the face's reference coordinate| for affine triangles
    auto inv_h = [&](int64_t e, int f) {
      const double* g = &m->geo_h[4 * e];
      double gx, gy;
      if (f == 0) { gx = -g[1]; gy = -g[3]; }
      else if (f == 1) { gx = g[0] + g[1]; gy = g[2] + g[3]; }
      else { gx = -g[0]; gy = -g[2]; }
      return std::sqrt(gx * gx + gy * gy);
    };
    std::vector<float> ih(size_t(3) * K);
    for (int64_t e = 0; e < K; ++e)
      for (int f = 0; f < 3; ++f) {
        const int32_t c = m->conn_h[3 * e + f];
        double v = inv_h(e, f);
        if (c >= 0) v = std::max(v, inv_h(c >> 2, c & 3));
        ih[3 * e + f] = float(v);
      }
    ce = cudaMalloc(&m->ih32, sizeof(float) * 3 * K);
    if (ce == cudaSuccess) ce = cudaMemcpy(m->ih32, ih.data(), sizeof(float) * 3 * K, cudaMemcpyHostToDevice);
    // derived geometry for the tensor-core applies (FP64 and an FP32 copy)
    std::vector<double> gx(size_t(16) * K);
    for (int64_t e = 0; e < K; ++e) {
      const double* g = &m->geo_h[4 * e];
      const double rx = g[0], sx = g[1], ry = g[2], sy = g[3];
      const double J = 1.0 / (rx * sy - ry * sx);
      double* o = &gx[16 * e];
      o[0] = J;
      o[1] = J * (rx * rx + ry * ry);
      o[2] = J * (rx * sx + ry * sy);
      o[3] = J * (sx * sx + sy * sy);
      for (int f = 0; f < 3; ++f) {
        double fx, fy;
        if (f == 0) { fx = -sx; fy = -sy; }
        else if (f == 1) { fx = rx + sx; fy = ry + sy; }
        else { fx = -rx; fy = -ry; }
        const double gn = std::sqrt(fx * fx + fy * fy), nx = fx / gn, ny = fy / gn;
        const int32_t c = m->conn_h[3 * e + f];
        o[4 + 4 * f + 0] = nx * rx + ny * ry;
        o[4 + 4 * f + 1] = nx * sx + ny * sy;
        o[4 + 4 * f + 2] = J * gn;
        o[4 + 4 * f + 3] = c >= 0 ? std::max(gn, inv_h(c >> 2, c & 3)) : gn;
      }
    }
    if (ce == cudaSuccess) ce = cudaMalloc(&m->geox, sizeof(double) * 16 * K);
    if (ce == cudaSuccess) ce = cudaMemcpy(m->geox, gx.data(), sizeof(double) * 16 * K, cudaMemcpyHostToDevice);
    const std::vector<float> gx32(gx.begin(), gx.end());
    if (ce == cudaSuccess) ce = cudaMalloc(&m->geox32, sizeof(float) * 16 * K);
    if (ce == cudaSuccess) ce = cudaMemcpy(m->geox32, gx32.data(), sizeof(float) * 16 * K, cudaMemcpyHostToDevice);
  }
  if (ce == cudaSuccess) ce = ensure_ops(m, N);
  // the tensor kernels' operator slices of the mesh degree: built here so that
  // an apply at the mesh degree allocates nothing once the mesh exists
  if (ce == cudaSuccess) ce = ensure_tensor_ops(m, N, true);
  if (ce == cudaSuccess) ce = ensure_tensor_ops(m, N, false);
  if (ce == cudaSuccess) ce = ensure_tc64_ops(m, N);
  if (ce != cudaSuccess) {
    dg_mesh_destroy(m);
    return cuda_fail(ce, "dg_mesh_setup");
  }
  *out = m;
  return DG_OK;
  DG_TRY_END
}

dg_status dg_mesh_destroy(dg_mesh* m) {
  if (!m) return DG_OK;
  free_workspace(m);
  free_ins_workspace(m);
  free_host_apply(m);
  cudaFree(m->face32);
  cudaFree(m->oz_scratch);
  cudaFree(m->t64_scratch);
  cudaFree(m->ih32);
  cudaFree(m->geox);
  cudaFree(m->geox32);
  cudaFree(m->geo64);
  cudaFree(m->geo32);
  cudaFree(m->conn);
  for (int d = 0; d <= kMaxN; ++d) {
    cudaFree(m->ops64[d].buf);
    cudaFree(m->ops32[d].buf);
  }
  for (auto& kv : m->transfer) {
    cudaFree(kv.second.P64);
    cudaFree(kv.second.P32);
  }
  delete m;
  return DG_OK;
}

dg_status dg_mesh_info(const dg_mesh* m, int* N, int64_t* K, int* Np) {
  if (!m) { set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (N) *N = m->N;
  if (K) *K = m->K;
  if (Np) *Np = (m->N + 1) * (m->N + 2) / 2;
  return DG_OK;
}

dg_status dg_mesh_nodes(const dg_mesh* mc, int degree, double* x, double* y, void* stream) {
  if (!mc || !x || !y) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (degree == 0) degree = mc->N;
  if (degree < 1 || degree > kMaxN) { set_error("degree must be in 0..10"); return DG_ERR_ARG; }
  DG_TRY_BEGIN
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  if (m->ref[degree].N == 0) m->ref[degree] = build_reference(degree);
  std::vector<double> hx, hy;
  node_coordinates(m, degree, hx, hy);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce == cudaSuccess) ce = cudaMemcpy(x, hx.data(), hx.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(y, hy.data(), hy.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return cuda_fail(ce, "dg_mesh_nodes");
  return DG_OK;
  DG_TRY_END
}

dg_status dg_operator_apply(const dg_mesh* mc, int degree, dg_prec prec, int B, double lambda, const void* u, void* Au,
                            void* stream) {
  if (!mc) { set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (B == 0) return DG_OK;  // empty batch: nothing to read or write
  if (!u || !Au) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (degree == 0) degree = mc->N;
  if (degree < 1 || degree > kMaxN) { set_error("degree must be in 1..10"); return DG_ERR_ARG; }
  if (prec != DG_F64 && prec != DG_F32 && prec != DG_F64_DFMA) { set_error("bad precision"); return DG_ERR_ARG; }
  if (B < 0) { set_error("negative batch"); return DG_ERR_ARG; }
  if (u == Au) { set_error("u and Au must not alias"); return DG_ERR_ARG; }
  if (!std::isfinite(lambda) || lambda < 0) { set_error("lambda must be finite and >= 0"); return DG_ERR_ARG; }
  DG_TRY_BEGIN
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  cudaError_t ce = ensure_ops(m, degree);
  if (ce == cudaSuccess) ce = launch_apply(m, degree, prec, B, lambda, u, Au, (cudaStream_t)stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "dg_operator_apply");
  return DG_OK;
  DG_TRY_END
}

dg_status dg_poisson_apply(const dg_mesh* m, dg_prec prec, int B, const void* u, void* Au, void* stream) {
  return dg_operator_apply(m, 0, prec, B, 0.0, u, Au, stream);
}

dg_status dg_helmholtz_apply(const dg_mesh* m, dg_prec prec, int B, double lambda, const void* u, void* Au,
                             void* stream) {
  return dg_operator_apply(m, 0, prec, B, lambda, u, Au, stream);
}

dg_status dg_operator_diagonal(const dg_mesh* mc, int degree, dg_prec prec, double lambda, void* diag, void* stream) {
  if (!mc || !diag) { set_error("NULL argument"); return DG_ERR_ARG; }
  if (degree == 0) degree = mc->N;
  if (degree < 1 || degree > kMaxN) { set_error("degree must be in 1..10"); return DG_ERR_ARG; }
  if (prec != DG_F64 && prec != DG_F32) { set_error("bad precision"); return DG_ERR_ARG; }
  DG_TRY_BEGIN
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  cudaError_t ce = ensure_ops(m, degree);
  if (ce == cudaSuccess) ce = launch_diagonal(m, degree, prec, lambda, diag, (cudaStream_t)stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "dg_operator_diagonal");
  return DG_OK;
  DG_TRY_END
}

dg_status dg_rhs(const dg_mesh* m, int B, const double* f, const double* g, double* b, void* stream) {
  if (!m) { set_error("mesh is NULL"); return DG_ERR_ARG; }
  if (B < 0) { set_error("negative batch"); return DG_ERR_ARG; }
  if (B == 0) return DG_OK;
  if (!f || !b) { set_error("NULL argument"); return DG_ERR_ARG; }
  cudaError_t ce = launch_rhs(m, B, f, g, b, (cudaStream_t)stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "dg_rhs");
  return DG_OK;
}

dg_status dg_reference_operators(int N, double* r, double* s, double* M, double* Dr, double* Ds, double* Mf,
                                 int32_t* fmask) {
  if (N < 1 || N > kMaxN) { set_error("degree N must be in 1..10"); return DG_ERR_ARG; }
  DG_TRY_BEGIN
  const RefElem R = build_reference(N);
  auto cp = [](double* dst, const std::vector<double>& v) { if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(double)); };
  cp(r, R.r);
  cp(s, R.s);
  cp(M, R.M);
  cp(Dr, R.Dr);
  cp(Ds, R.Ds);
  cp(Mf, R.Mf);
  if (fmask)
    for (size_t i = 0; i < R.fmask.size(); ++i) fmask[i] = R.fmask[i];
  return DG_OK;
  DG_TRY_END
}

dg_status dg_interpolation_matrix(int Nf, int Nc, double* P) {
  if (Nf < 2 || Nf > kMaxN || Nc < 1 || Nc >= Nf || !P) { set_error("need 10 >= Nf > Nc >= 1 and P"); return DG_ERR_ARG; }
  DG_TRY_BEGIN
  const std::vector<double> h = interpolation_matrix(Nf, Nc);
  std::memcpy(P, h.data(), h.size() * sizeof(double));
  return DG_OK;
  DG_TRY_END
}

}  // extern "C"
