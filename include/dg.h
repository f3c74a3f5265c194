/*
 * dg.h - C ABI of the GB300 SIPDG pressure-Poisson library.
 *
 * The library implements the hot path of the semi-implicit nodal DG
 * incompressible-flow method of Karakus, Chalmers, Swirydowicz & Warburton
 * (arXiv:1801.00246): the matrix-free symmetric-interior-penalty (SIPDG)
 * Laplacian / screened-Poisson operator on affine triangles of degree
 * N = 1..10 (Section 2.1 Eq. INS_SD_5, Section 5.2 Eq. ellipticOp1-3), and
 * its solution by preconditioned conjugate gradients with a degree-coarsening
 * p-multigrid preconditioner (Section 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Reference triangle {r, s >= -1, r + s <= 0}, vertices v0=(-1,-1),
 *    v1=(1,-1), v2=(-1,1). Elements are given counter-clockwise; local face f
 *    joins local vertices f and (f+1) mod 3.
 *  - Nodal fields are contiguous arrays [B][K][Np], Np = (N+1)(N+2)/2, the
 *    nodes being the Warp & Blend nodes (Section 2.1) ordered in rows of
 *    constant s from s = -1 upward, r increasing within a row.
 *  - Operator outputs are WEAK coefficient vectors: (A u)_i = a(u, l_i),
 *    i.e. already multiplied by the mass matrix (Eq. ellipticOp3 carries the
 *    leading M^e).
 *  - Boundary tags per face: 0 interior, 1 Dirichlet, 2 Neumann.
 *    Dirichlet faces use the ghost state u+ = 2g - u-, grad u+ = grad u-
 *    (homogeneous operator: g = 0); Neumann faces u+ = u-, grad u+ = -grad u-.
 *    Penalty per face: tau = (N+1)(N+2)/2 * max(1/h-, 1/h+), h = |E|/|face|
 *    (Eq. PenaltyParameter); boundary faces use h- only.
 *  - Field pointers marked "device" are caller-owned CUDA device memory; the
 *    library never frees them. Host pointers are only read during the call.
 *  - All device work is enqueued on the caller's stream (cudaStream_t passed
 *    as void*; NULL = legacy default stream). Calls that return results to
 *    the host (dg_pcg_solve's info) synchronise that stream.
 *  - Every entry point returns a dg_status; no exception crosses the ABI.
 *    Arguments are validated before any launch. dg_last_error() returns a
 *    human-readable message for the last failing call on this thread.
 *  - Threads: a mesh and its workspaces belong to one host thread at a time
 *    (calls on one mesh from several threads must be serialised by the
 *    caller). Process-wide tables (operator slices, launch configurations,
 *    constant-memory operators) are built under a library lock on first use
 *    of a degree and precision on a device, so meshes on different threads
 *    may meet a new degree at the same time.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, N out of range) */
  DG_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  DG_ERR_OOM = 3,            /* device allocation failed */
  DG_ERR_NOT_CONVERGED = 4,  /* max_iter reached; x holds the last iterate */
  DG_ERR_BREAKDOWN = 5,      /* p^T A p <= 0 or NaN in a Krylov recurrence */
  DG_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  DG_ERR_MESH = 7            /* non-positive Jacobian or non-conforming faces */
} dg_status;

/* DG_F64: FP64 in/out with the mesh's FP64 kernel (DG_KERNEL_* below; built-in:
 *         from degree 3 up the dense products run on the BF16 tensor cores with
 *         exact integer slicing, relative error ~1e-13 of |A||u|; that path scales
 *         each element's data by a power of two and rebuilds results from their
 *         exponent bits, so it takes finite fields whose nonzero element
 *         magnitudes lie between about 1e-250 and 1e250);
 * DG_F32: FP32 in/out with FP32-level accuracy (relative error <= 1e-5), with the
 *         mesh's FP32 kernel: FP32 arithmetic, or on the tensor cores three
 *         round-to-nearest BF16 pieces per operand with FP32 accumulation;
 * DG_F64_DFMA: FP64 in/out, the tile kernel, every operation on the FP64 pipe. */
typedef enum { DG_F64 = 0, DG_F32 = 1, DG_F64_DFMA = 2 } dg_prec;

typedef struct dg_mesh dg_mesh; /* opaque; owned by the library until dg_mesh_destroy */

/* Apply kernels. Every one evaluates the same operator (Eq. ellipticOp3);
 * they differ in how the work maps to the GPU, and results agree to rounding.
 *   DG_KERNEL_AUTO:   the mesh's current choice (built-in per degree, or set
 *                     by dg_autotune / dg_set_apply_kernel)
 *   DG_KERNEL_TILE:   element tiles in shared memory, one thread per node
 *                     (FP64 on the FP64 pipe, or FP32); all degrees (FP32 default at N = 10)
 *   DG_KERNEL_GEMM:   FP32 only: register-blocked small GEMMs over element tiles; degrees 1-9
 *   DG_KERNEL_TENSOR: dense products on the BF16 tensor cores (FP64: exact 7-bit
 *                     integer slicing, 8 slices; FP32: three round-to-nearest BF16
 *                     pieces); degrees 1-9
 *   DG_KERNEL_EPT:    one element per thread, operators in constant memory; degrees 1-3
 *   DG_KERNEL_TENSOR_PIPE: DG_KERNEL_TENSOR with the output product's fill and product
 *                     phases on separate warps, double-buffered through shared memory
 *                     (mbarrier hand-off with bounded waits; see dg_tensor_timeouts)
 *   DG_KERNEL_TC05:   FP32 only: both products on the Blackwell tensor cores (tcgen05,
 *                     operands and accumulators in tensor memory, bulk copies), two FP16
 *                     pieces per operand scaled by powers of two; degrees 1-8. Needs u and
 *                     Au 16-byte aligned (otherwise DG_KERNEL_TENSOR runs instead).
 *   DG_KERNEL_TC64:   FP64 only: both products on the Blackwell tensor cores (tcgen05,
 *                     exact 7-bit integer slicing, 8 slices, accumulators in tensor memory)
 *                     and the pointwise stage in float-float on the FP32 pipe; all degrees.
 *                     Intermediates carry 48 bits (float-float), so where the operator's
 *                     terms cancel strongly (a node next to an element 2^60 larger, at
 *                     N = 10) an entry's error can reach a few 1e-12 of |A||u|.
 *                     Handles finite fields whose magnitudes stay within the double range
 *                     at every stage (about 1e-250..1e250, as DG_KERNEL_TENSOR). */
enum { DG_KERNEL_AUTO = 0, DG_KERNEL_TILE = 1, DG_KERNEL_GEMM = 2, DG_KERNEL_TENSOR = 3, DG_KERNEL_EPT = 4,
       DG_KERNEL_TENSOR_PIPE = 5, DG_KERNEL_TC05 = 6, DG_KERNEL_TC64 = 7 };
#define DG_NUM_KERNELS 8 /* kernel ids 0..7; dg_autotune's times use this many slots per entry */
#define DG_MAX_DEGREE 10 /* degrees 1..10 (Section 5.2 studies the kernels up to N = 10) */

/* Preconditioner choices for dg_pcg_solve (Section 3). DG_PREC_AMG: one
 * smoothed-aggregation V-cycle on the probed matrix of the mesh degree itself
 * (algebraic multigrid alone, the baseline the paper compares pMG-AMG with;
 * flexible CG, as with DG_PREC_PMG). */
enum { DG_PREC_NONE = 0, DG_PREC_JACOBI = 1, DG_PREC_INVMASS = 2, DG_PREC_PMG = 3, DG_PREC_AMG = 4 };

typedef struct {
  double tol;          /* stop when ||b - A x||_2 / ||b||_2 <= tol (per right-hand side) */
  int max_iter;        /* outer iteration cap */
  int precond;         /* DG_PREC_* */
  int nlevels;         /* p-multigrid: number of degrees in `degrees` (2..8) */
  int degrees[8];      /* p-multigrid degrees, degrees[0] = mesh degree, strictly decreasing, last >= 1 */
  int cheb_degree;     /* Chebyshev smoothing degree per pre/post smoothing (>= 1) */
  double coarse_tol;   /* relative tolerance of the CG solve on the coarsest degree */
  int coarse_max_iter; /* iteration cap of that coarse CG */
  int mixed;           /* 1: p-multigrid levels in FP32, outer iteration FP64; 0: all FP64 */
  int power_steps;     /* power iterations for the Chebyshev bound rho(D^{-1}A) */
  int coarse_amg;      /* 1: the coarsest-degree CG is preconditioned by an algebraic-multigrid
                          V-cycle (smoothed aggregation on the probed coarsest matrix, FP64) */
  int graph;           /* 1 (default): the whole solve runs as one CUDA graph whose iteration
                          loops are device-side conditional WHILE nodes (no host round trip
                          per iteration); it is captured on the first solve of a configuration
                          (batch, lambda, options) and replayed afterwards. 0: host-driven
                          loop. Both give bit-identical results. */
} dg_solver_opts;

#define DG_MAX_BATCH 64

typedef struct {
  int iters[DG_MAX_BATCH];      /* outer iterations per right-hand side */
  double relres[DG_MAX_BATCH];  /* final ||b - A x|| / ||b|| from the recurrence residual */
  int total_iters;              /* iterations of the batched loop (max over the batch) */
  float ms;                     /* device time of the solve (CUDA events on the stream) */
  int coarse_iters;             /* coarsest-degree CG iterations summed over the solve */
  double precond_bytes;         /* device bytes of the preconditioner's own data: the p-multigrid
                                   levels' and coarse solve's vectors, the algebraic multigrid's
                                   matrices and vectors (0 for none, Jacobi, inverse mass) */
} dg_solve_info;

/* Default options: tol 1e-10, max_iter 1000, Jacobi, no multigrid. */
void dg_solver_opts_default(dg_solver_opts* opts);

/* Build the discretisation of degree N (1..DG_MAX_DEGREE) on a triangle mesh.
 * VX, VY: host, Nv vertex coordinates. EToV: host, K x 3 vertex indices,
 * counter-clockwise. bc: host, K x 3 tags (0 interior, 1 Dirichlet,
 * 2 Neumann) of face f = (v_f, v_{f+1}); a face with no neighbour must carry
 * a non-zero tag and a shared face must carry 0.
 * Computes on the host: nodes, reference operators (Eq. elMass, elStiff,
 * elLift), geometric factors (Eq. operators2, elementOps), face connectivity;
 * uploads them with stream-ordered copies. Returns DG_ERR_MESH for a
 * non-positive Jacobian, a face shared by more than two elements, or tags
 * that disagree with the connectivity. */
dg_status dg_mesh_setup(int N, int64_t Nv, const double* VX, const double* VY, int64_t K,
                        const int32_t* EToV, const int8_t* bc, void* stream, dg_mesh** out);
dg_status dg_mesh_destroy(dg_mesh* mesh);

/* Degree, element count and nodes per element of a mesh. */
dg_status dg_mesh_info(const dg_mesh* mesh, int* N, int64_t* K, int* Np);

/* Physical coordinates of the degree-`degree` nodes (1..10; 0 = mesh degree):
 * x_dev, y_dev device arrays [K][Np(degree)], FP64. */
dg_status dg_mesh_nodes(const dg_mesh* mesh, int degree, double* x_dev, double* y_dev, void* stream);

/* Poisson operator (Eq. ellipticOp3 with lambda = 0) at the mesh degree:
 * Au[b] = A u[b] for b < B. u, Au: device [B][K][Np] of FP64 (DG_F64) or
 * FP32 (DG_F32); FP32 arithmetic accumulates in FP32. u and Au must not alias.
 * The apply kernels keep scratch with the mesh (the FP32 GEMM kernel's face
 * data, the tensor kernels' gradient rows; allocated or grown on first use),
 * so applies on one mesh must not overlap on the GPU (issue them on one
 * stream, or use one mesh per stream). */
dg_status dg_poisson_apply(const dg_mesh* mesh, dg_prec prec, int B, const void* u, void* Au,
                           void* stream);

/* Screened-Poisson (Helmholtz) operator -L + lambda (Eq. ellipticOp1):
 * Au = A u + lambda J M u. Same layout rules as dg_poisson_apply. */
dg_status dg_helmholtz_apply(const dg_mesh* mesh, dg_prec prec, int B, double lambda,
                             const void* u, void* Au, void* stream);

/* Either operator at any degree 1..10 on the same mesh (p-multigrid levels). */
dg_status dg_operator_apply(const dg_mesh* mesh, int degree, dg_prec prec, int B, double lambda,
                            const void* u, void* Au, void* stream);

/* dg_operator_apply on fields in HOST memory: u_host, Au_host [B][K][Np]
 * (page-locked memory lets the copies overlap the apply; pageable memory
 * works, the copies then serialise). The input is copied to a device buffer
 * kept with the mesh, the operator applied and the result copied back, all
 * enqueued behind the caller's earlier work on `stream`; the caller's later
 * work on `stream` runs after the last copy. With the tcgen05 FP64 kernel (the
 * FP64 default from degree 3) the copies run on two copy streams of the mesh,
 * in chunks of rows: a chunk's gradient product starts once its input has
 * arrived, and a chunk's output copy starts as soon as its output product has
 * written it. The host buffers must stay valid until `stream` has passed the
 * call (synchronise it before reading Au_host). Calls on one mesh must not
 * overlap. Same results as dg_operator_apply on device copies of u. */
dg_status dg_apply_host(const dg_mesh* mesh, int degree, dg_prec prec, int B, double lambda, const void* u_host,
                        void* Au_host, void* stream);

/* Kernel selection has no counterpart in the paper, which tunes its kernels
 * per degree by hand (Section 5.2); it changes how the operator of
 * Eq. ellipticOp3 is computed, never what.
 *
 * The mesh's kernel table: which DG_KERNEL_* the applies (and every solve's
 * applies) of `degree` in `prec` (DG_F64 or DG_F32), Poisson (helmholtz = 0) or
 * Helmholtz (1), use. DG_KERNEL_AUTO restores the built-in choice. A kernel
 * not available for the degree and precision is rejected (DG_ERR_ARG). Not
 * thread-safe against applies in flight on the same mesh from other threads. */
dg_status dg_set_apply_kernel(dg_mesh* mesh, int degree, dg_prec prec, int helmholtz, int kernel);
/* The kernel in use (never DG_KERNEL_AUTO); -1 for bad arguments. */
int dg_get_apply_kernel(const dg_mesh* mesh, int degree, dg_prec prec, int helmholtz);

/* Autotuner: for each degree in [degree_lo, degree_hi] and both precisions,
 * times every available kernel on this mesh with B random right-hand sides
 * (256 MB L2 flush before each of three timed launches, best kept), for the
 * Poisson form and, if lambda > 0, the Helmholtz form (with lambda = 0 the
 * Helmholtz entry takes the Poisson winner), and stores the fastest in the
 * kernel table. times (host, may be NULL): float[DG_MAX_DEGREE + 1][2][2][DG_NUM_KERNELS] milliseconds
 * indexed [degree][0: FP64, 1: FP32][helmholtz][kernel], 0 where not timed.
 * Allocates and frees its own scratch (4 fields of B*K*Np(degree_hi) values
 * plus 256 MB); synchronises `stream`. Solves captured as CUDA graphs before
 * the call are re-captured on their next use. */
dg_status dg_autotune(dg_mesh* mesh, int B, double lambda, int degree_lo, int degree_hi, float* times,
                      void* stream);

/* diag(A) of the operator at `degree` (0 = mesh degree) for the given lambda:
 * diag device [K][Np(degree)] in FP64 or FP32 (Jacobi preconditioner). */
dg_status dg_operator_diagonal(const dg_mesh* mesh, int degree, dg_prec prec, double lambda, void* diag,
                               void* stream);

/* Weak right-hand side of the Dirichlet problem -lap u + lambda u = f,
 * u = g on Dirichlet faces: b = J M f - L(g), L(g)_i = sum over Dirichlet
 * faces of (n.grad l_i, g) - 2 tau (l_i, g). f, g, b: device FP64 [B][K][Np]
 * nodal values (only the face-node values of g are used). */
dg_status dg_rhs(const dg_mesh* mesh, int B, const double* f, const double* g, double* b,
                 void* stream);

/* Preconditioned conjugate gradients on A(lambda) x = b for B right-hand
 * sides at once (Section 3). b, x: device FP64 [B][K][Np]; x holds the
 * initial guess on entry and the solution on exit. With DG_PREC_PMG and
 * opts->mixed the multigrid levels run in FP32 and the outer iteration is
 * flexible CG in FP64; otherwise standard PCG. info (host, may be NULL)
 * receives iterations and residuals after a stream synchronisation.
 * Workspace is allocated by the library on first use and kept with the mesh.
 * Returns DG_ERR_NOT_CONVERGED if any right-hand side misses tol within
 * max_iter (x holds the last iterate), DG_ERR_BREAKDOWN on p^T A p <= 0. */
dg_status dg_pcg_solve(dg_mesh* mesh, const dg_solver_opts* opts, int B, double lambda,
                       const double* b, double* x, dg_solve_info* info, void* stream);

/* State of the semi-implicit incompressible Navier-Stokes stepper
 * (Section 2.2 Eq. INS_TD_3, Section 2.3 subcycling). All field pointers are
 * caller-owned device FP64 arrays; the caller checkpoints by saving them. */
typedef struct {
  double nu;              /* kinematic viscosity */
  double dt;              /* macro time step */
  int Ns;                 /* LSERK(5,4) advection substeps per macro step (dt_s = dt / Ns) */
  int step;               /* completed steps; 0 selects the BDF1/EXT1 start-up step; incremented */
  double* U;              /* [2][K][Np] velocity U^n on entry, U^{n+1} on exit */
  double* Uold;           /* [2][K][Np] U^{n-1} on entry (unused when step == 0), U^n on exit */
  double* P;              /* [K][Np] pressure P^n on entry, P^{n+1} on exit */
  const double* gU;       /* [2][K][Np] steady velocity data on velocity-Dirichlet faces (face nodes used) */
  const double* gP;       /* [K][Np] steady pressure data on pressure-Dirichlet faces (face nodes used) */
  dg_solver_opts vel_opts;   /* the two batched velocity Helmholtz solves (B = 2) */
  dg_solver_opts pr_opts;    /* the pressure-increment Poisson solve */
  int vel_iters[2];       /* out: iterations of the last step's velocity solves */
  int pr_iters;           /* out: iterations of the last step's pressure solve */
  float ms;               /* out: device time of the last call */
  /* Time-dependent boundary data (optional; NULL = steady data in gU, gP).
   * With gU_hist set, gU and gP are the data at t^{n+1} = (step + 1) dt, and a
   * call advances exactly one step (nsteps = 1); the caller supplies each
   * step's data. */
  const double* gU_hist;  /* [2][2][K][Np]: velocity data at t^n, then at t^{n-1} (unused when step == 0) */
  const double* gP_n;     /* [K][Np]: pressure data at t^n (required with gU_hist) */
} dg_ins_state;

/* Advance nsteps macro steps of the algebraic splitting scheme with
 * second-order BDF/EXT coefficients (gamma = 3/2, beta = 2, -1/2; the first
 * step uses BDF1) and a first-order pressure increment:
 *   (i)   U^  = sum_i beta_i U~^{n-i}, each U^{n-i} advected to t^{n+1} by
 *         LSERK(5,4) substeps of the DG advection operator with cubature and
 *         the local Lax-Friedrichs flux (Eq. INS_CUB_N), advecting velocity
 *         the linear extrapolant through U^n, U^{n-1};
 *   (ii)  (-L + gamma/(nu dt)) U^^ = U^/(nu dt) - (1/nu) G P^n, both
 *         components in one batched PCG (vel_opts, lambda = gamma/(nu dt));
 *   (iii) -L dP = -(gamma/dt) D.U^^ (pr_opts);
 *   (iv)  U^{n+1} = U^^ - (dt/gamma) G dP, P^{n+1} = P^n + dP.
 * mesh_u and mesh_p are the same triangulation and degree carrying the
 * velocity and the pressure-increment boundary tags. G uses central fluxes
 * with p* = gP on pressure-Dirichlet faces and p* = p- on the others; D uses
 * u* = gU on velocity-Dirichlet faces and u* = u- on velocity-Neumann faces
 * (Eq. INS_SD_4_1, INS_SD_4_2). With steady boundary data (gU_hist NULL) the
 * pressure increment is zero on pressure-Dirichlet faces. With time-dependent
 * data the advection stages at time t take the velocity data interpolated in
 * time through t^{n-1}, t^n, t^{n+1} (quadratic; linear between t^n and
 * t^{n+1} at step 0), the Helmholtz solve and D take gU at t^{n+1}, G P^n takes
 * gP_n, and the increment takes gP - gP_n on pressure-Dirichlet faces.
 * Workspace is allocated on the first call and kept with mesh_u. Returns the
 * status of a failing solve. */
dg_status dg_ins_step(dg_mesh* mesh_u, dg_mesh* mesh_p, dg_ins_state* state, int nsteps, void* stream);

/* Jacobi-preconditioned CG on A(lambda) x = b that allocates nothing.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run (a host whose memory pool owns
 * the whole GPU, a time-critical loop that must not pay cudaMalloc's implicit
 * synchronisation, or a simulation that must not fail on an allocation
 * midway). Its workspace, including the scratch of the tensor-core apply, is
 * a fixed scratch array of 2^22 doubles (32 MiB) compiled into the library as
 * device memory, which every GPU that loads the library holds until the
 * process exits; the apply's operator tables for the mesh degree are built by
 * dg_mesh_setup. The apply is the kernel dg_pcg_solve would use (the mesh's
 * FP64 kernel choice), so both give the same iterates. b, x: device FP64
 * [B][K][Np] as in dg_pcg_solve (x: initial guess in, solution out); the mesh
 * comes from an earlier dg_mesh_setup on the current device. A call needs
 * (4 B + 1) K Np words for the CG vectors and the Jacobi inverse, a few per
 * right-hand side, and the apply's scratch: B K (2 Np + 15 (N + 1)) words
 * (B K (3 Np + 15 (N + 1)) with lambda != 0) for the tcgen05 FP64 kernel,
 * the default from degree 3, or 2 B K Np (3 B K Np) for the mma.sync ones.
 * At B = 1 and N = 8 that is about K <= 9,200 triangles (lambda = 0) or
 * 8,400; larger problems are rejected with DG_ERR_ARG before any device
 * work. The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture. The call calls no cudaMalloc/cudaFree and no allocating
 * library routine. All calls share the one array and leave their data in it
 * (every word a call reads is written by that call first): two calls whose
 * work overlaps on the GPU (different streams, or different host threads on
 * one device) race and corrupt each other's results; serialise them. info
 * (host, may be NULL) receives iterations and residuals; info->ms is not
 * measured (0). */
dg_status dg_pcg_jacobi_solve_static(const dg_mesh* mesh, int B, double lambda, double tol, int max_iter,
                                     const double* b, double* x, dg_solve_info* info, void* stream);

/* ---------------------------------------------------------------- tetrahedra
 * The same SIPDG operator on affine tetrahedra, the three-dimensional extension
 * the paper names as its next step (Section 6). Readings for three dimensions:
 * penalty tau = (N+1)(N+3)/3 max(1/h-, 1/h+) with h = |E| / |face| (the
 * triangle's (N+1)(N+2)/2 is the d = 2 case of (N+1)(N+d)/d); boundary faces as
 * on triangles; nodes equispaced, (r, s, t) = (-1 + 2i/N, -1 + 2j/N, -1 + 2k/N),
 * i + j + k <= N, ordered by k, then j, then i; degrees 1..5. Reference
 * tetrahedron v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1), v3 = (-1,-1,1);
 * local faces (v0,v1,v2), (v0,v1,v3), (v1,v2,v3), (v0,v2,v3), opposite
 * v3, v2, v0, v1. Fields are device arrays [B][K][Np],
 * Np = (N+1)(N+2)(N+3)/6. */
typedef struct dg_tet_mesh dg_tet_mesh;

/* Build the degree-N discretisation. VX, VY, VZ: host [Nv]; EToV: host [K][4]
 * (positive orientation: det[v1-v0, v2-v0, v3-v0] > 0); bc: host [K][4], tag of
 * face f (0 interior, 1 Dirichlet, 2 Neumann). Faces are matched by their vertex
 * triples and face nodes by coordinates; a boundary face without a tag, a
 * non-positive Jacobian or non-matching face nodes give DG_ERR_MESH. */
dg_status dg_tet_mesh_setup(int N, int64_t Nv, const double* VX, const double* VY, const double* VZ, int64_t K,
                            const int32_t* EToV, const int8_t* bc, void* stream, dg_tet_mesh** mesh);
dg_status dg_tet_mesh_destroy(dg_tet_mesh* mesh);
dg_status dg_tet_mesh_info(const dg_tet_mesh* mesh, int* N, int64_t* K, int* Np);
/* Node coordinates into device [K][Np] arrays x, y, z. */
dg_status dg_tet_mesh_nodes(const dg_tet_mesh* mesh, double* x, double* y, double* z, void* stream);
/* Au = A(lambda) u for B right-hand sides. DG_F64: the dense products ([Dr; Ds;
 * Dt] u, the mass matrix, [Dr^T Ds^T Dt^T]) as exactly sliced FP64 products on
 * the tcgen05 tensor cores, the pointwise and face stages on CUDA cores in FP64;
 * DG_F64_DFMA (and DG_F64 at degrees 1 and 2): everything on the FP64 pipe;
 * DG_F32: FP32. The FP32 and FP64-pipe
 * forms run in two kernels (reference gradient and face traces, then lift and
 * output). The
 * first call at a batch size (and precision) larger than any before allocates
 * the mesh's apply scratch ((3 Np + 8 Nfp) B K words, Nfp = (N+1)(N+2)/2; about
 * (11 Np + 24 Nfp + 5) B K doubles for DG_F64 from degree 3); applies on one mesh
 * must not overlap. */
dg_status dg_tet_apply(const dg_tet_mesh* mesh, dg_prec prec, int B, double lambda, const void* u, void* Au,
                       void* stream);
/* b = J M f - L(g) (the Dirichlet problem's weak right-hand side, as dg_rhs). */
dg_status dg_tet_rhs(const dg_tet_mesh* mesh, int B, const double* f, const double* g, double* b, void* stream);
/* Jacobi-preconditioned CG on A(lambda) x = b in FP64 for B right-hand sides
 * (x: initial guess in, solution out), host-driven (synchronises the stream each
 * iteration); workspace kept with the mesh. info as for dg_pcg_solve. */
dg_status dg_tet_pcg_jacobi_solve(dg_tet_mesh* mesh, int B, double lambda, double tol, int max_iter,
                                  const double* b, double* x, dg_solve_info* info, void* stream);

/* Host-only: the library's own reference data for degree N (1..10), for
 * inspection without a GPU. r, s: Np; M, Dr, Ds: Np x Np row-major;
 * Mf: (N+1) x (N+1); fmask: 3 x (N+1) local node index of face node j of face
 * f in counter-clockwise order. Any pointer may be NULL. */
dg_status dg_reference_operators(int N, double* r, double* s, double* M, double* Dr, double* Ds,
                                 double* Mf, int32_t* fmask);

/* Host-only: p-multigrid interpolation from degree Nc to degree Nf
 * (Nf > Nc >= 1): P[Np(Nf)][Np(Nc)] row-major, the coarse nodal basis
 * evaluated at the fine nodes. */
dg_status dg_interpolation_matrix(int Nf, int Nc, double* P);

/* Waits of the pipelined tensor kernel that gave up (a broken producer/consumer
 * hand-off: the affected apply's output is invalid) since the last call, summed
 * over the current device; reading clears it. Synchronises the device. Returns
 * -1 if the device could not be queried. No counterpart in the paper. */
int dg_tensor_timeouts(void);

/* Diagnostic with no counterpart in the paper: launches one kernel whose
 * warp waits, with the bounded mbarrier wait every tensor-core kernel of the
 * library uses, on a barrier phase that nothing completes. The wait gives up
 * after `seconds` (0 < seconds <= 10), the kernel counts one timeout in
 * dg_tensor_timeouts and returns, and the call returns DG_ERR_TIMEOUT: a
 * device-side wait that cannot finish ends its kernel instead of hanging the
 * GPU, and the context stays usable. Synchronises `stream`. */
dg_status dg_wait_selftest(double seconds, void* stream);

/* Number of kernels this library has launched since it was loaded (all
 * devices and threads); a diagnostic for counting launches in a timed region. */
uint64_t dg_launch_count(void);

const char* dg_status_string(dg_status status);
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
