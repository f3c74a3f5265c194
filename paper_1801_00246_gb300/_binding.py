"""ctypes binding of include/dg.h (argument marshalling only)."""
import ctypes
import os

import numpy as np

from . import build as _build

DG_F64, DG_F32, DG_F64_DFMA = 0, 1, 2
PREC_NONE, PREC_JACOBI, PREC_INVMASS, PREC_PMG, PREC_AMG = 0, 1, 2, 3, 4
(KERNEL_AUTO, KERNEL_TILE, KERNEL_GEMM, KERNEL_TENSOR, KERNEL_EPT, KERNEL_TENSOR_PIPE, KERNEL_TC05,
 KERNEL_TC64) = 0, 1, 2, 3, 4, 5, 6, 7
NUM_KERNELS = 8
MAX_DEGREE = 10  # DG_MAX_DEGREE
DG_MAX_BATCH = 64

_STATUS = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_CUDA", 3: "DG_ERR_OOM", 4: "DG_ERR_NOT_CONVERGED",
           5: "DG_ERR_BREAKDOWN", 6: "DG_ERR_TIMEOUT", 7: "DG_ERR_MESH"}


class DgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = _STATUS.get(status, str(status))


class SolverOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precond", ctypes.c_int),
                ("nlevels", ctypes.c_int), ("degrees", ctypes.c_int * 8), ("cheb_degree", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("coarse_max_iter", ctypes.c_int), ("mixed", ctypes.c_int),
                ("power_steps", ctypes.c_int), ("coarse_amg", ctypes.c_int),
                ("graph", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int * DG_MAX_BATCH), ("relres", ctypes.c_double * DG_MAX_BATCH),
                ("total_iters", ctypes.c_int), ("ms", ctypes.c_float), ("coarse_iters", ctypes.c_int),
                ("precond_bytes", ctypes.c_double)]


class InsState(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("dt", ctypes.c_double), ("Ns", ctypes.c_int), ("step", ctypes.c_int),
                ("U", ctypes.c_void_p), ("Uold", ctypes.c_void_p), ("P", ctypes.c_void_p),
                ("gU", ctypes.c_void_p), ("gP", ctypes.c_void_p), ("vel_opts", SolverOpts),
                ("pr_opts", SolverOpts), ("vel_iters", ctypes.c_int * 2), ("pr_iters", ctypes.c_int),
                ("ms", ctypes.c_float), ("gU_hist", ctypes.c_void_p), ("gP_n", ctypes.c_void_p)]


_lib = None


def lib_path():
    return _build.lib_path()


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pd, pi32 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    sig = {
        "dg_mesh_setup": ([i32, i64, pd, pd, i64, pi32, ctypes.POINTER(ctypes.c_int8), vp, ctypes.POINTER(vp)], i32),
        "dg_mesh_destroy": ([vp], i32),
        "dg_mesh_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)], i32),
        "dg_mesh_nodes": ([vp, i32, vp, vp, vp], i32),
        "dg_poisson_apply": ([vp, i32, i32, vp, vp, vp], i32),
        "dg_helmholtz_apply": ([vp, i32, i32, dbl, vp, vp, vp], i32),
        "dg_operator_apply": ([vp, i32, i32, i32, dbl, vp, vp, vp], i32),
        "dg_apply_host": ([vp, i32, i32, i32, dbl, vp, vp, vp], i32),
        "dg_operator_diagonal": ([vp, i32, i32, dbl, vp, vp], i32),
        "dg_rhs": ([vp, i32, vp, vp, vp, vp], i32),
        "dg_pcg_solve": ([vp, ctypes.POINTER(SolverOpts), i32, dbl, vp, vp, ctypes.POINTER(SolveInfo), vp], i32),
        "dg_solver_opts_default": ([ctypes.POINTER(SolverOpts)], None),
        "dg_ins_step": ([vp, vp, ctypes.POINTER(InsState), i32, vp], i32),
        "dg_pcg_jacobi_solve_static": ([vp, i32, dbl, dbl, i32, vp, vp, ctypes.POINTER(SolveInfo), vp], i32),
        "dg_tet_mesh_setup": ([i32, i64, pd, pd, pd, i64, pi32, ctypes.POINTER(ctypes.c_int8), vp, ctypes.POINTER(vp)],
                              i32),
        "dg_tet_mesh_destroy": ([vp], i32),
        "dg_tet_mesh_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)], i32),
        "dg_tet_mesh_nodes": ([vp, vp, vp, vp, vp], i32),
        "dg_tet_apply": ([vp, i32, i32, dbl, vp, vp, vp], i32),
        "dg_tet_rhs": ([vp, i32, vp, vp, vp, vp], i32),
        "dg_tet_pcg_jacobi_solve": ([vp, i32, dbl, dbl, i32, vp, vp, ctypes.POINTER(SolveInfo), vp], i32),
        "dg_reference_operators": ([i32, pd, pd, pd, pd, pd, pd, pi32], i32),
        "dg_interpolation_matrix": ([i32, i32, pd], i32),
        "dg_status_string": ([i32], ctypes.c_char_p),
        "dg_last_error": ([], ctypes.c_char_p),
        "dg_launch_count": ([], ctypes.c_uint64),
        "dg_set_apply_kernel": ([vp, i32, i32, i32, i32], i32),
        "dg_get_apply_kernel": ([vp, i32, i32, i32], i32),
        "dg_autotune": ([vp, i32, dbl, i32, i32, ctypes.POINTER(ctypes.c_float), vp], i32),
        "dg_tensor_timeouts": ([], i32),
        "dg_wait_selftest": ([dbl, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise DgError(status, lib().dg_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr())


def reference_operators(N):
    """The library's own reference data (host-only call, no GPU needed)."""
    Np = (N + 1) * (N + 2) // 2
    Nfp = N + 1
    r, s = np.zeros(Np), np.zeros(Np)
    M, Dr, Ds = np.zeros((Np, Np)), np.zeros((Np, Np)), np.zeros((Np, Np))
    Mf = np.zeros((Nfp, Nfp))
    fmask = np.zeros((3, Nfp), dtype=np.int32)
    _check(lib().dg_reference_operators(N, _dptr(r), _dptr(s), _dptr(M), _dptr(Dr), _dptr(Ds), _dptr(Mf),
                                        fmask.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return dict(r=r, s=s, M=M, Dr=Dr, Ds=Ds, Mf=Mf, fmask=fmask)


def interpolation_matrix(Nf, Nc):
    P = np.zeros(((Nf + 1) * (Nf + 2) // 2, (Nc + 1) * (Nc + 2) // 2))
    _check(lib().dg_interpolation_matrix(Nf, Nc, _dptr(P)))
    return P


def default_opts(**kw):
    o = SolverOpts()
    lib().dg_solver_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "degrees":
            for i, d in enumerate(v):
                o.degrees[i] = int(d)
            o.nlevels = len(v)
        else:
            setattr(o, k, v)
    return o


class Mesh:
    """A discretisation of degree N on a triangle mesh (owns a dg_mesh*)."""

    def __init__(self, N, VX, VY, EToV, bc):
        self.N = int(N)
        VX = np.ascontiguousarray(VX, dtype=np.float64)
        VY = np.ascontiguousarray(VY, dtype=np.float64)
        EToV = np.ascontiguousarray(EToV, dtype=np.int32)
        bc = np.ascontiguousarray(bc, dtype=np.int8)
        self.K = int(EToV.shape[0])
        self.Np = (self.N + 1) * (self.N + 2) // 2
        h = ctypes.c_void_p()
        _check(lib().dg_mesh_setup(self.N, VX.size, _dptr(VX), _dptr(VY), self.K,
                                   EToV.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), None, ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_inputs(cls, mesh, N):
        return cls(N, mesh.VX, mesh.VY, mesh.EToV, mesh.bc)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dg_mesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def np_of(self, degree):
        d = self.N if degree in (0, None) else degree
        return (d + 1) * (d + 2) // 2

    def nodes(self, degree=0):
        import torch
        n = self.np_of(degree)
        x = torch.empty((self.K, n), dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        _check(lib().dg_mesh_nodes(self._h, int(degree or 0), _tptr(x), _tptr(y), _stream()))
        return x, y

    def apply(self, u, lam=0.0, degree=0, out=None, fp64_pipe=False):
        """A u for u of shape [B][K][Np] or [K][Np] (float64 -> FP64, float32 -> FP32).
        float64 runs the tensor-core product path unless fp64_pipe=True."""
        import torch
        if not u.is_cuda or not u.is_contiguous():
            raise ValueError("u must be a contiguous CUDA tensor")
        prec = {torch.float64: DG_F64, torch.float32: DG_F32}[u.dtype]
        if fp64_pipe and prec == DG_F64:
            prec = DG_F64_DFMA
        B = 1 if u.dim() == 2 else u.shape[0]
        if out is None:
            out = torch.empty_like(u)
        _check(lib().dg_operator_apply(self._h, int(degree or 0), prec, B, float(lam), _tptr(u), _tptr(out),
                                       _stream()))
        return out

    def apply_host(self, u, lam=0.0, degree=0, out=None):
        """A u for a contiguous CPU tensor u ([B][K][Np] or [K][Np], float64 or
        float32; page-locked memory overlaps the copies with the apply), result in
        a CPU tensor (out, page-locked if u is). Enqueued on the current stream;
        synchronise it before reading the result."""
        import torch
        if u.is_cuda or not u.is_contiguous():
            raise ValueError("u must be a contiguous CPU tensor")
        prec = {torch.float64: DG_F64, torch.float32: DG_F32}[u.dtype]
        B = 1 if u.dim() == 2 else u.shape[0]
        if out is None:
            out = torch.empty_like(u, pin_memory=u.is_pinned())
        _check(lib().dg_apply_host(self._h, int(degree or 0), prec, B, float(lam), ctypes.c_void_p(u.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), _stream()))
        return out

    def set_kernel(self, degree, prec, helmholtz, kernel):
        """Choose the apply kernel (KERNEL_*) for a degree, precision (DG_F64 /
        DG_F32) and form (helmholtz 0/1); KERNEL_AUTO restores the built-in one."""
        _check(lib().dg_set_apply_kernel(self._h, int(degree), int(prec), int(bool(helmholtz)), int(kernel)))

    def kernel(self, degree, prec, helmholtz=0):
        return lib().dg_get_apply_kernel(self._h, int(degree), int(prec), int(bool(helmholtz)))

    def kernels_available(self, degree, prec):
        """The KERNEL_* ids the library accepts for a degree and precision (asked
        through the kernel table, whose entry is restored)."""
        L = lib()
        keep = [L.dg_get_apply_kernel(self._h, int(degree), int(prec), h) for h in (0, 1)]
        out = [k for k in range(1, NUM_KERNELS)
               if L.dg_set_apply_kernel(self._h, int(degree), int(prec), 0, k) == 0]
        for h in (0, 1):
            L.dg_set_apply_kernel(self._h, int(degree), int(prec), h, KERNEL_AUTO)
            if keep[h] >= 0 and keep[h] != L.dg_get_apply_kernel(self._h, int(degree), int(prec), h):
                L.dg_set_apply_kernel(self._h, int(degree), int(prec), h, keep[h])
        return out

    def autotune(self, B=1, lam=0.0, degrees=None):
        """Time every available kernel per degree and precision on this mesh and
        keep the fastest; returns {(degree, 'f64'|'f32', helmholtz): {kernel: ms}}."""
        lo, hi = degrees if degrees is not None else (1, self.N)
        times = (ctypes.c_float * ((MAX_DEGREE + 1) * 2 * 2 * NUM_KERNELS))()
        _check(lib().dg_autotune(self._h, int(B), float(lam), int(lo), int(hi), times, _stream()))
        out = {}
        for d in range(lo, hi + 1):
            for p, name in ((0, "f64"), (1, "f32")):
                for h in (0, 1):
                    base = ((d * 2 + p) * 2 + h) * NUM_KERNELS
                    row = {k: times[base + k] for k in range(1, NUM_KERNELS) if times[base + k] > 0}
                    if row:
                        out[(d, name, h)] = row
        return out

    def diagonal(self, lam=0.0, degree=0, dtype=None):
        import torch
        dtype = dtype or torch.float64
        prec = DG_F64 if dtype == torch.float64 else DG_F32
        d = torch.empty((self.K, self.np_of(degree)), dtype=dtype, device="cuda")
        _check(lib().dg_operator_diagonal(self._h, int(degree or 0), prec, float(lam), _tptr(d), _stream()))
        return d

    def rhs(self, f, g=None):
        """b = J M f - L(g) (weak right-hand side with Dirichlet data g)."""
        import torch
        B = 1 if f.dim() == 2 else f.shape[0]
        b = torch.empty_like(f)
        _check(lib().dg_rhs(self._h, B, _tptr(f), _tptr(g) if g is not None else None, _tptr(b), _stream()))
        return b

    def solve_static(self, b, x=None, lam=0.0, tol=1e-10, max_iter=1000, check=True):
        """Jacobi-PCG from the library's fixed device scratch array (no allocation
        inside the call); returns (x, info)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        B = 1 if b.dim() == 2 else b.shape[0]
        info = SolveInfo()
        st = lib().dg_pcg_jacobi_solve_static(self._h, B, float(lam), float(tol), int(max_iter), _tptr(b), _tptr(x),
                                              ctypes.byref(info), _stream())
        if check:
            _check(st)
        return x, dict(iters=list(info.iters[:B]), relres=list(info.relres[:B]), total_iters=info.total_iters,
                       status=_STATUS.get(st, st))

    def solve(self, b, x=None, lam=0.0, opts=None, check=True, **kw):
        """PCG solve A x = b (b, x float64 [B][K][Np] or [K][Np]); returns (x, info, status)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        B = 1 if b.dim() == 2 else b.shape[0]
        o = opts if opts is not None else default_opts(**kw)
        info = SolveInfo()
        st = lib().dg_pcg_solve(self._h, ctypes.byref(o), B, float(lam), _tptr(b), _tptr(x), ctypes.byref(info),
                                _stream())
        if check:
            _check(st)
        res = dict(iters=list(info.iters[:B]), relres=list(info.relres[:B]), total_iters=info.total_iters,
                   ms=info.ms, coarse_iters=info.coarse_iters, precond_bytes=info.precond_bytes,
                   status=_STATUS.get(st, st))
        return x, res


class TetMesh:
    """A degree-N (1..5) discretisation on affine tetrahedra (owns a dg_tet_mesh*):
    VX, VY, VZ vertex coordinates, EToV [K][4], bc [K][4] face tags."""

    def __init__(self, N, VX, VY, VZ, EToV, bc):
        self.N = int(N)
        VX, VY, VZ = (np.ascontiguousarray(v, dtype=np.float64) for v in (VX, VY, VZ))
        EToV = np.ascontiguousarray(EToV, dtype=np.int32)
        bc = np.ascontiguousarray(bc, dtype=np.int8)
        self.K = int(EToV.shape[0])
        self.Np = (self.N + 1) * (self.N + 2) * (self.N + 3) // 6
        h = ctypes.c_void_p()
        _check(lib().dg_tet_mesh_setup(self.N, VX.size, _dptr(VX), _dptr(VY), _dptr(VZ), self.K,
                                       EToV.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), None, ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_inputs(cls, mesh, N):
        return cls(N, mesh.VX, mesh.VY, mesh.VZ, mesh.EToV, mesh.bc)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.dg_tet_mesh_destroy(h)
            self._h = None

    def nodes(self):
        import torch
        x, y, z = (torch.empty((self.K, self.Np), dtype=torch.float64, device="cuda") for _ in range(3))
        _check(lib().dg_tet_mesh_nodes(self._h, _tptr(x), _tptr(y), _tptr(z), _stream()))
        return x, y, z

    def apply(self, u, lam=0.0, out=None, fp64_pipe=False):
        """A(lam) u; u float64 or float32 CUDA [B][K][Np] or [K][Np] (the dtype picks the precision;
        float64 runs its products on the tensor cores unless fp64_pipe=True)."""
        import torch
        u = u.contiguous()
        B = 1 if u.dim() == 2 else u.shape[0]
        out = torch.empty_like(u) if out is None else out
        prec = DG_F64 if u.dtype == torch.float64 else DG_F32
        if fp64_pipe and prec == DG_F64:
            prec = DG_F64_DFMA
        _check(lib().dg_tet_apply(self._h, prec, B, float(lam), _tptr(u), _tptr(out), _stream()))
        return out

    def rhs(self, f, g):
        import torch
        f, g = f.contiguous(), g.contiguous()
        B = 1 if f.dim() == 2 else f.shape[0]
        b = torch.empty_like(f)
        _check(lib().dg_tet_rhs(self._h, B, _tptr(f), _tptr(g), _tptr(b), _stream()))
        return b

    def solve(self, b, x=None, lam=0.0, tol=1e-10, max_iter=5000, check=True):
        """Jacobi-PCG in FP64; returns (x, info)."""
        import torch
        b = b.contiguous()
        x = torch.zeros_like(b) if x is None else x
        B = 1 if b.dim() == 2 else b.shape[0]
        info = SolveInfo()
        st = lib().dg_tet_pcg_jacobi_solve(self._h, B, float(lam), float(tol), int(max_iter), _tptr(b), _tptr(x),
                                           ctypes.byref(info), _stream())
        if check:
            _check(st)
        return x, dict(iters=list(info.iters[:B]), relres=list(info.relres[:B]), total_iters=info.total_iters,
                       status=_STATUS.get(st, st))


class InsStepper:
    """Semi-implicit INS time stepper (dg_ins_step) on a velocity-tagged and a
    pressure-tagged mesh of the same triangulation. U, Uold: float64 CUDA
    [2][K][Np]; P: [K][Np]; gU, gP: steady boundary data as nodal fields, or
    with bc given, time-dependent data: bc(t) -> (gU(t), gP(t)) as CUDA tensors
    of those shapes, sampled at t^{n+1}, t^n and t^{n-1} each step (t^n = n dt)."""

    def __init__(self, mesh_u, mesh_p, nu, dt, Ns, U, P, gU=None, gP=None, vel_opts=None, pr_opts=None, Uold=None,
                 bc=None):
        import torch
        self.mesh_u, self.mesh_p = mesh_u, mesh_p
        self.U = U.contiguous()
        self.Uold = (Uold if Uold is not None else U.clone()).contiguous()
        self.P = P.contiguous()
        self.bc = bc
        if bc is not None:
            g1, p1 = bc(0.0)
            self.gU, self.gP = torch.empty_like(g1).contiguous(), torch.empty_like(p1).contiguous()
            self.gU_hist = torch.empty((2,) + tuple(g1.shape), dtype=g1.dtype, device=g1.device)
            self.gP_n = torch.empty_like(p1).contiguous()
        else:
            self.gU = gU.contiguous()
            self.gP = gP.contiguous()
        self.st = InsState()
        self.st.nu, self.st.dt, self.st.Ns, self.st.step = float(nu), float(dt), int(Ns), 0
        for name in ("U", "Uold", "P", "gU", "gP"):
            setattr(self.st, name, getattr(self, name).data_ptr())
        if bc is not None:
            self.st.gU_hist, self.st.gP_n = self.gU_hist.data_ptr(), self.gP_n.data_ptr()
        self.st.vel_opts = vel_opts if vel_opts is not None else default_opts(precond=PREC_INVMASS, tol=1e-10)
        self.st.pr_opts = pr_opts if pr_opts is not None else default_opts(precond=PREC_JACOBI, tol=1e-10,
                                                                           max_iter=20000)
        del torch

    def step(self, n=1):
        if self.bc is None:
            _check(lib().dg_ins_step(self.mesh_u._h, self.mesh_p._h, ctypes.byref(self.st), int(n), _stream()))
            return dict(step=self.st.step, vel_iters=list(self.st.vel_iters), pr_iters=self.st.pr_iters,
                        ms=self.st.ms)
        ms = 0.0
        for _ in range(int(n)):
            k, dt = self.st.step, self.st.dt
            for dst, t in ((self.gU_hist[0], k * dt), (self.gU_hist[1], (k - 1) * dt)):
                dst.copy_(self.bc(t)[0])
            self.gP_n.copy_(self.bc(k * dt)[1])
            g1, p1 = self.bc((k + 1) * dt)
            self.gU.copy_(g1)
            self.gP.copy_(p1)
            _check(lib().dg_ins_step(self.mesh_u._h, self.mesh_p._h, ctypes.byref(self.st), 1, _stream()))
            ms += self.st.ms
        return dict(step=self.st.step, vel_iters=list(self.st.vel_iters), pr_iters=self.st.pr_iters, ms=ms)
