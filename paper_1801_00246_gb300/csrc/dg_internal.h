// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "dg.h"

namespace dgx {

constexpr int kMaxN = DG_MAX_DEGREE;

// Host reference-element data for one degree (FP64, row-major matrices).
struct RefElem {
  int N = 0, Np = 0, Nfp = 0;
  std::vector<double> r, s, Vinv, M, Dr, Ds, Br, Bs, Mf;
  std::vector<int> fmask;  // 3 x Nfp, counter-clockwise per face
  // Jacobi-diagonal pieces: S_rr[i][i], (S_rs+S_sr)[i][i], S_ss[i][i], M[i][i]
  std::vector<double> diag_rr, diag_rs, diag_ss, diag_m;
  // per face node a of face f: sum_b Mf[a][b] Dr[k_b][k_a] (and Ds)
  std::vector<double> face_cr, face_cs;
};

RefElem build_reference(int N);
std::vector<double> interpolation_matrix(int Nf, int Nc);
std::vector<double> lobatto_points(int N);
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
double jacobi_p(double x, double a, double b, int n);
int face_node(int N, int f, int j);
std::vector<double> invert(int n, std::vector<double> A);
void vandermonde2d(int N, const std::vector<double>& r, const std::vector<double>& s, std::vector<double>& V,
                   std::vector<double>* Vr, std::vector<double>* Vs);
struct InsWorkspace;
struct Amg;
cudaError_t amg_build(dg_mesh* m, int degree, double lambda, int B, Amg** out, cudaStream_t st);
cudaError_t amg_vcycle(Amg* a, const double* b, double* x, cudaStream_t st);
void amg_free(Amg* a);
int amg_levels(const Amg* a);
size_t amg_bytes(const Amg* a);  // device bytes of the hierarchy (matrices, vectors, coarse inverse)
cudaError_t amg_apply_fine(Amg* a, const double* x, double* y, cudaStream_t st);
void free_ins_workspace(dg_mesh* m);

// Device copy of the reference operators of one degree, in one precision.
// Layout of the single buffer (all row-major, T = double or float):
//   Dr[Np*Np] Ds[Np*Np] Br[Np*Np] Bs[Np*Np] M[Np*Np] Mf[Nfp*Nfp]
//   diag_rr[Np] diag_rs[Np] diag_ss[Np] diag_m[Np] face_cr[3Nfp] face_cs[3Nfp] Minv[Np*Np]
struct DevOps {
  void* buf = nullptr;
  size_t bytes = 0;
};

size_t ops_count(int N);  // number of T entries in the buffer above

// Per-mesh, per-degree p-multigrid transfer P (Np_f x Np_c), FP64 and FP32.
struct DevTransfer {
  double* P64 = nullptr;
  float* P32 = nullptr;
};

// Solver workspace kept with the mesh (FP64 outer vectors + multigrid levels).
struct Workspace;

}  // namespace dgx

// Connectivity word per face: interior  -> (neighbour << 2) | neighbour_face,
//                             boundary  -> -1 - tag (tag 1 Dirichlet, 2 Neumann).
struct dg_mesh {
  int N = 0;
  int64_t K = 0;
  int64_t Nv = 0;
  // host copies
  std::vector<double> VX, VY;
  std::vector<int32_t> EToV;
  std::vector<double> geo_h;  // K x 4: r_x, s_x, r_y, s_y
  std::vector<int32_t> conn_h;
  // device
  double* geo64 = nullptr;   // K x 4
  float* geo32 = nullptr;    // K x 4
  int32_t* conn = nullptr;   // K x 3
  // per face: max(1/h-, 1/h+) (1/h- on boundary faces); the penalty of a
  // degree-d operator is (d+1)(d+2)/2 times this
  float* ih32 = nullptr;     // K x 3
  // FP64 derived geometry [K][16]: J, Grr, Grs, Gss | per face (n.grad r, n.grad s, sJ, max(1/h-,1/h+))
  double* geox = nullptr;
  float* geox32 = nullptr;  // the same 16 words per element in FP32
  dgx::RefElem ref[dgx::kMaxN + 1];
  dgx::DevOps ops64[dgx::kMaxN + 1];
  dgx::DevOps ops32[dgx::kMaxN + 1];
  std::map<std::pair<int, int>, dgx::DevTransfer> transfer;
  dgx::Workspace* ws = nullptr;  // most recently used solver workspace
  std::map<std::string, dgx::Workspace*> ws_cache;  // all workspaces, by configuration
  dgx::InsWorkspace* ins = nullptr;
  // FP32 apply scratch: every element's face traces and outward normal
  // derivatives, [B][K][3][N+1] float2 (grown on demand)
  float2* face32 = nullptr;
  size_t face32_cap = 0;
  // FP64 tensor-core apply scratch: C1, Y and the face buffer (grown on demand)
  double* oz_scratch = nullptr;
  size_t oz_cap = 0;
  // FP64 tcgen05 apply scratch: C1, Y and per-element exponents (grown on demand)
  double* t64_scratch = nullptr;
  size_t t64_cap = 0;
  uint64_t scratch_gen = 0;  // bumped whenever face32, oz_scratch or t64_scratch is reallocated
  int64_t nb_reach = -1;     // largest (neighbour - element) index over interior faces (-1: not computed)
  // apply kernel per [degree][0: FP64, 1: FP32][Helmholtz]; DG_KERNEL_AUTO = built-in choice
  int8_t kern[dgx::kMaxN + 1][2][2] = {};
  uint64_t kern_gen = 0;  // bumped whenever the table changes
  // host-buffer apply (dg_apply_host): device copies of u and Au (grown on demand),
  // its two copy streams and events (chunk inputs, chunk outputs, start, done)
  void* hx_u = nullptr;
  void* hx_out = nullptr;
  size_t hx_cap = 0;
  cudaStream_t hx_in = nullptr, hx_outs = nullptr;
  static constexpr int kHostChunks = 32;
  cudaEvent_t hx_ev[2 * kHostChunks + 2] = {};
};
void free_host_apply(dg_mesh* m);  // host_apply.cu

namespace dgx {

// Launchers (device code in the .cu files). `degree` in 1..kMaxN.
cudaError_t ensure_ops(dg_mesh* m, int degree);
// c1_scratch (optional, FP64 only): device words for the tensor kernels'
// scratch, at least B*K*Np(degree)*(lambda != 0 ? 3 : 2) + 1 of them for the
// mma.sync kernels and tc64_scratch_words(degree, B*K, lambda != 0) for the
// tcgen05 one; null uses the scratch kept with the mesh (grown on demand).
cudaError_t launch_apply(const dg_mesh* m, int degree, dg_prec prec, int B, double lambda, const void* u,
                         void* Au, cudaStream_t st, double* c1_scratch = nullptr);
cudaError_t launch_rhs(const dg_mesh* m, int B, const double* f, const double* g, double* b, cudaStream_t st);
cudaError_t launch_diagonal(const dg_mesh* m, int degree, dg_prec prec, double lambda, void* diag,
                            cudaStream_t st);
int default_kernel(int degree, bool f64);
bool kernel_valid(int kernel, int degree, bool f64);
bool ept_supported(int degree);
cudaError_t launch_apply_ept(dg_mesh* m, int degree, bool f64, int B, double lambda, const void* u, void* Au,
                             cudaStream_t st);
cudaError_t launch_apply_tensor(dg_mesh* m, int degree, bool f64, int B, double lambda, const void* u, void* Au,
                                bool pipe, cudaStream_t st, double* c1_scratch = nullptr);
bool tensor_supported(int degree);  // the mma.sync tensor kernels (N <= 9)
// Builds (once per device, degree and precision) the tensor kernels' operator
// slices on the current device; dg_mesh_setup calls it for the mesh degree.
cudaError_t ensure_tensor_ops(dg_mesh* m, int degree, bool f64);
bool tensor_ops_ready(int degree, bool f64);  // built on the current device (no build)
cudaError_t tensor_pipe_error(int* flag);
// FP32 apply on the tcgen05 tensor cores (apply_tc05.cu); needs 16-byte aligned u and Au
bool tc05_usable(const void* u, const void* Au);
cudaError_t launch_apply_tc05(dg_mesh* m, int degree, int B, double lambda, const float* u, float* Au,
                              cudaStream_t st);
cudaError_t tc05_error(int* flag);  // reads and clears the tcgen05 kernels' timeout flag
cudaError_t launch_wait_selftest(double seconds, int* gave_up_dev, cudaStream_t st);
struct Tc64Op;
cudaError_t tc64_op_create(const std::vector<double>& A, int M, int K, Tc64Op* op);
void tc64_op_free(Tc64Op* op);
// out[r][c] (+)= sum_k A[c][k] X[r][k] (FP64, exact slicing on the tcgen05 tensor cores;
// accum: add to out instead of overwriting it); X row-major with leading dimension ldx.
// ex (optional): per row r an exponent E with |X[r][k]| < 2^E for every k (-1100 for a
// zero row), from the producer of X; without it the product scans each row itself.
cudaError_t tc64_gemm_launch(const Tc64Op& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                             cudaStream_t st, int accum = 0, const int* ex = nullptr);
bool tc64_supported(int degree);
// An apply in chunks of rows (elements x right-hand sides) for callers that move
// the data in and out while it runs: the first phase (gradient product) reads
// only each row's own u, the last (output product) writes each row's Au by
// itself. `before` is enqueued ahead of chunk i's first phase, `after` behind
// chunk i's last; chunk i's neighbour phase runs once the first phase of every
// chunk holding one of its rows' neighbours has been issued.
struct ApplyChunks {
  int n = 0;                        // chunks
  const int64_t* bounds = nullptr;  // chunk c holds rows [bounds[c], bounds[c + 1]); bounds[n] = all rows
  cudaError_t (*before)(void* ctx, int chunk, int64_t r0, int64_t r1) = nullptr;
  cudaError_t (*after)(void* ctx, int chunk, int64_t r0, int64_t r1) = nullptr;
  void* ctx = nullptr;
};
// scratch (optional): tc64_scratch_words(degree, B*K, lambda != 0) device words;
// null uses the scratch kept with the mesh (grown on demand) and builds the
// degree's tables on first use, a given scratch needs them built already
cudaError_t launch_apply_tc64(dg_mesh* m, int degree, int B, double lambda, const double* u, double* Au,
                              cudaStream_t st, double* scratch = nullptr, const ApplyChunks* chunks = nullptr);
// The apply kernel the mesh's table selects (DG_KERNEL_AUTO resolved).
int selected_kernel(const dg_mesh* m, int degree, dg_prec prec, bool helm);
size_t tc64_scratch_words(int degree, int64_t nE, bool helm);
cudaError_t ensure_tc64_ops(dg_mesh* m, int degree);  // dg_mesh_setup builds the mesh degree's tables
bool tc64_ops_ready(int degree);                      // built on the current device (no build)
cudaError_t tc64_error(int* flag);
// FP64 products on the tcgen05 tensor cores with exact integer slicing (apply_tc64.cu):
// an operator A (M x K, K <= 256) cut into 8 slices in blocks of 48 rows x 32 columns
struct Tc64Op {
  int M = 0, K = 0, NCH = 0, KCH = 0;
  uint8_t* blocks = nullptr;
  int* ea = nullptr;
};
// FP64 operator A (M x K, row-major) sliced for the tensor-core products out[r] = A X[r]:
// the mma.sync fragment layout and the tcgen05 block layout (used when built)
struct SlicedOp {
  int M = 0, K = 0, Mt = 0, Kt = 0;
  uint32_t* A = nullptr;
  int* ea = nullptr;
  Tc64Op t64;
};
cudaError_t sliced_op_create(const std::vector<double>& A, int M, int K, SlicedOp* op);
void sliced_op_free(SlicedOp* op);
cudaError_t sliced_gemm(const SlicedOp& op, int64_t rows, const double* X, int64_t ldx, double* out, int64_t ldo,
                        cudaStream_t st);
cudaError_t launch_nodes(const dg_mesh* m, int degree, double* x, double* y, cudaStream_t st);

void set_error(const std::string& msg);

// Guards the process-wide tables built on first use (operator slices, launch
// configurations, constant-memory operators): every lazy build takes it.
std::mutex& table_mutex();

// Running count of kernels this library has launched (all devices, all threads).
void note_launch();
uint64_t launch_count();
void add_launches(int64_t n);
cudaError_t poison(void* p, size_t bytes, int group);  // 0xFF fill when DG_POISON_SCRATCH=1 or =group
enum { POISON_AMG = 2, POISON_SOLVER = 3, POISON_APPLY = 4 };

}  // namespace dgx
