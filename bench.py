"""Benchmark of the SIPDG pressure-Poisson hot path on one GB300.

Workload (the headline configuration): 512x512 jittered grid split into
524,288 triangles, degree N=8 (Np=45, 23.6M nodes), Dirichlet boundary.
One step = one pass of the hot path over this input:
  * Poisson apply A u in FP64 and in FP32 (U(-1,1) input, seed 1)
  * Helmholtz apply (lambda = 1) in FP64 and in FP32
  * a p-multigrid flexible-CG pressure solve to 1e-10 (V-cycle 8->4->2->1,
    degree-3 Chebyshev-Jacobi smoothing, degree-1 coarse solve by one
    CG pass preconditioned by an algebraic-multigrid V-cycle), mixed precision
    (FP32 multigrid levels, FP64 outer iteration)
  * the same solve in plain FP64 (FP64 multigrid levels)
  * the mixed solve once more with the host-driven loop (the two solves above
    run as one CUDA graph each, loops on the device)
`value` is the FP64 Poisson apply throughput (GDOF/s = K*Np / apply time);
the other pieces are reported beside it. After the timed steps, outside the
timed region: the true residuals of the last solves, the same solves with 4
and 16 right-hand sides in one batched solve, and the split INS step on the
8,192-triangle Kovasznay workload. L2 (135 MB) is flushed by writing a
256 MB buffer before every timed launch; all timing is CUDA events on the
launching stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --sweep     # applies for N = 1..10, FP64/FP32, batch 1/4/16
  python bench.py --tet       # tetrahedral applies for N = 1..5 (196,608 tetrahedra)

`--impl reference` times the FP64 CPU oracle (the method written plainly in
numpy) on a bounded sample of the same workload, on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MESH_NAME = "c5_sweep_524288tri_N8"
METRIC = "Poisson Ax GDOF/s & PCG solve ms (N=8, 524k tri), mixed vs FP64, % HBM roof"
PMG_DEGREES = [8, 4, 2, 1]
CHEB = 3           # Chebyshev-Jacobi smoothing degree per pre/post smoothing
COARSE_PASSES = 1  # degree-1 coarse solve: one AMG-preconditioned CG pass (a scaled AMG V-cycle)
# DRAM bytes per FP64 apply at N=8 from the latest ncu capture of the current
# default kernels (tcgen05: gradient product 0.806 GB, face fill 0.938 GB, output
# product 0.888 GB); None while the kernels differ from that capture
TENSOR_APPLY_TRAFFIC = 2.632e9


# apply kernels by DG_KERNEL_* value
KERNEL_NAMES = {1: "tile (FP64/FP32 pipe)", 2: "gemm (FP32 register GEMMs)",
                3: "tensor (mma.sync BF16 slice products: gradient product, then fused fill + output product)",
                4: "ept (element per thread)", 5: "tensor_pipe",
                6: "tc05 (tcgen05 FP16-piece products, tensor-memory operands: face kernel, then fused apply)",
                7: "tc64 (tcgen05 exactly sliced FP64 products: gradient product, float-float pointwise stage, "
                   "output product)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = 6800.0
    src = "fallback"
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        hbm = float(d.get("hbm_gbs", hbm))
        src = "measured"
    # FP64 CUDA-core peak: the nominal 1.25 TFLOP/s of GB300 (no measured copy in the peaks file)
    bf16 = 1895.5
    if os.path.exists(p):
        bf16 = float(d.get("bf16_tflops", bf16))
    return dict(hbm_gbs=hbm, hbm_src=src, fp64_gflops=1250.0, fp32_gflops=2 * 152 * 128 * 2.07, bf16_tflops=bf16)


def algo_per_element(N, word):
    """Algorithmic bytes and flops per element of one apply (B = 1).

    bytes: read u and write A u (2 Np words) + 4 geometry words + 3 int32
    neighbour words; flops: 10 Np^2 + 24 Np Nfp (gradient, lift of jumps,
    divergence, neighbour normal derivatives, lift of the flux, mass)."""
    Np = (N + 1) * (N + 2) // 2
    Nfp = N + 1
    return 2 * Np * word + 4 * word + 12, 10 * Np * Np + 24 * Np * Nfp


class Clocks:
    """nvidia-smi sampler running during the timed region; the raw samples go to
    $DG_CLOCKS_CSV (default /tmp/dg_clocks.csv; local rank r > 0 appends ".r"), the
    summary into the JSON line."""

    def __init__(self, index):
        self.proc = None
        base = os.environ.get("DG_CLOCKS_CSV", "/tmp/dg_clocks.csv")
        self.path = base if index == 0 else "%s.%d" % (base, index)  # one file per local rank
        self.index = index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": float(np.median(hi)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def ranks_max(vals, device):
    """Max over ranks of each timing: the job takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_gdofs(world, K, Np, ms):
    """Whole-job throughput: every rank applies the operator to its own copy of
    the workload (replicas, weak scaling), so the job processes world * K * Np
    nodes in the slowest rank's time."""
    return world * K * Np / (ms * 1e-3) / 1e9


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def busy_cores(cpu_s, wall_s):
    """Cores the process kept busy over a timed region (CPU time / wall time,
    at least 1): the oracle is plain numpy, but its matrix products may run on
    a multi-threaded BLAS."""
    return max(1, int(round(cpu_s / wall_s))) if wall_s > 0 else 1


def cpu_oracle_sample(N, n_elems, reps=1, seed=1):
    """Time the FP64 oracle apply on a bounded sample of the workload; returns
    the oracle, the wall times and the cores it kept busy."""
    from dg_inputs import config_mesh, uniform_field
    from oracle.sipdg import Sipdg
    m, _ = config_mesh(MESH_NAME)
    ora = Sipdg(m.VX, m.VY, m.EToV, m.bc, N)
    u = uniform_field((m.K, ora.Np), seed=seed)
    elems = np.linspace(0, m.K - 1, n_elems).astype(np.int64)
    ora.apply(u, elems=elems[:64])  # warm caches
    times = []
    c0 = time.process_time()
    for _ in range(reps):
        t0 = time.perf_counter()
        ora.apply(u, elems=elems)
        times.append(time.perf_counter() - t0)
    return ora, times, busy_cores(time.process_time() - c0, sum(times))


def cpu_oracle_solve_c1():
    """The oracle's Jacobi-PCG solve of the 512-triangle N=3 workload (manufactured
    sin(pi x) sin(pi y), Dirichlet) to 1e-10, matrix-free: wall time in ms,
    iterations, relative residual."""
    from dg_inputs import config_mesh, manufactured
    from oracle.sipdg import Sipdg
    from oracle.solvers import cg
    m, N = config_mesh("c1_poisson_512tri_N3")
    ora = Sipdg(m.VX, m.VY, m.EToV, m.bc, N)
    uex, fex = manufactured("sin_pi_x_sin_pi_y")
    b = ora.rhs(fex(ora.x, ora.y), uex(ora.x, ora.y))
    dinv = 1.0 / ora.diagonal()
    t0 = time.perf_counter()
    _, it, rr = cg(ora.apply, b, tol=1e-10, maxit=5000, prec=lambda r: dinv * r)
    return (time.perf_counter() - t0) * 1e3, int(it), float(rr)


def oracle_child():
    """--oracle-child: the oracle apply sample and the c1 solve in this process
    (started with the BLAS thread pools limited to one thread by the parent)."""
    N = 8
    ora, times, cores = cpu_oracle_sample(N, 1024, reps=2)
    ms, it, rr = cpu_oracle_solve_c1()
    print(json.dumps({"apply_gdofs": 1024 * ora.Np / float(np.min(times)) / 1e9, "cores": cores,
                      "solve_c1_ms": ms}), flush=True)


def cpu_oracle_one_core():
    """The oracle timed in a child process on one core (BLAS threads set to 1)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child"], capture_output=True,
                           text=True, env=env, timeout=600)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as ex:  # reported, not fatal: the baseline is context
        return {"error": str(ex)[:200]}


def run_reference(args, world, rank):
    if rank != 0:
        return
    N = 8
    n_elems = 3072
    ora, _, _ = cpu_oracle_sample(N, 64, reps=1)
    from dg_inputs import config_mesh, uniform_field
    m, _ = config_mesh(MESH_NAME)
    u = uniform_field((m.K, ora.Np), seed=1)
    elems = np.linspace(0, m.K - 1, n_elems).astype(np.int64)
    for _ in range(args.warmup):
        ora.apply(u, elems=elems[:256])
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        ora.apply(u, elems=elems)
    wall = time.perf_counter() - t0
    cores = busy_cores(time.process_time() - c0, wall)
    dt = wall / args.steps
    val = n_elems * ora.Np / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GDOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512 jittered grid, 524288 triangles, N=8, Poisson apply (oracle sample)",
                   "sample_elements": n_elems},
        "cpu_baseline": {"value": val, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 oracle Poisson apply on {n_elems} of 524288 elements per step"},
        "e2e": {"value": val, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    from dg_inputs import config_mesh, manufactured, uniform_field

    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    L = P.lib()
    N = 8
    m, _ = config_mesh(MESH_NAME)
    mesh = P.Mesh.from_inputs(m, N)
    K, Np = mesh.K, mesh.Np
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    u64 = torch.from_numpy(uniform_field((K, Np), seed=1)).to(dev)
    u32 = u64.float()
    out64 = torch.empty_like(u64)
    out32 = torch.empty_like(u32)
    xn, yn = mesh.nodes()
    uex, fex = manufactured("sin_2pi_x_cos_3pi_y")
    xh, yh = xn.cpu().numpy(), yn.cpu().numpy()
    b = mesh.rhs(torch.from_numpy(fex(xh, yh)).to(dev), torch.from_numpy(uex(xh, yh)).to(dev))
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts_mixed = P._binding.default_opts(precond=P.PREC_PMG, degrees=PMG_DEGREES, tol=1e-10, max_iter=200,
                                         mixed=1, cheb_degree=CHEB, coarse_tol=1e-2, coarse_max_iter=COARSE_PASSES,
                                         coarse_amg=1)
    opts_mixed_host = P._binding.default_opts(precond=P.PREC_PMG, degrees=PMG_DEGREES, tol=1e-10, max_iter=200,
                                              mixed=1, cheb_degree=CHEB, coarse_tol=1e-2, coarse_max_iter=COARSE_PASSES,
                                              coarse_amg=1, graph=0)
    opts_fp64 = P._binding.default_opts(precond=P.PREC_PMG, degrees=PMG_DEGREES, tol=1e-10, max_iter=200,
                                        mixed=0, cheb_degree=CHEB, coarse_tol=1e-2, coarse_max_iter=COARSE_PASSES,
                                        coarse_amg=1)

    def flush():
        flush_buf.fill_(1.0)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        return e0, e1, r

    def step(record):
        ev = {}
        ev["poisson_f64"] = timed(lambda: mesh.apply(u64, out=out64))
        ev["poisson_f32"] = timed(lambda: mesh.apply(u32, out=out32))
        ev["helmholtz_f64"] = timed(lambda: mesh.apply(u64, lam=1.0, out=out64))
        ev["helmholtz_f32"] = timed(lambda: mesh.apply(u32, lam=1.0, out=out32))
        x_m = torch.zeros_like(b)
        ev["solve_mixed"] = timed(lambda: mesh.solve(b, x_m, opts=opts_mixed))
        x_d = torch.zeros_like(b)
        ev["solve_fp64"] = timed(lambda: mesh.solve(b, x_d, opts=opts_fp64))
        x_h = torch.zeros_like(b)
        ev["solve_mixed_host_loop"] = timed(lambda: mesh.solve(b, x_h, opts=opts_mixed_host))
        if record is not None:
            torch.cuda.synchronize()
            record["x_last"] = {"mixed": x_m, "fp64": x_d}
            for k, (e0, e1, r) in ev.items():
                record.setdefault(k, []).append(e0.elapsed_time(e1))
                if k.startswith("solve"):
                    record.setdefault(k + "_iters", []).append(r[1]["iters"][0])
                    record.setdefault(k + "_relres", []).append(r[1]["relres"][0])
                    record.setdefault(k + "_coarse", []).append(r[1]["coarse_iters"])

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    rec = {}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    n0 = L.dg_launch_count()
    with Clocks(local) as clk:
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            step(rec)
        s1.record(stream)
        torch.cuda.synchronize()
    launches = int(L.dg_launch_count() - n0)
    total_ms = s0.elapsed_time(s1)
    if world > 1:
        total_ms, ax_ms_max = ranks_max([total_ms, float(np.mean(rec["poisson_f64"]))], dev)
    else:
        ax_ms_max = float(np.mean(rec["poisson_f64"]))
    clocks = clk.summary()

    # end to end through the public API from pinned host buffers: dg_apply_host copies
    # u in and A u out inside the call (chunked copies overlapped with the apply)
    uh = torch.from_numpy(uniform_field((K, Np), seed=1)).pin_memory()
    oh = torch.empty_like(uh).pin_memory()
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush()
        e0.record(stream)
        mesh.apply_host(uh, out=oh)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))

    # true residual ||b - A x|| / ||b|| of the last step's solutions, with the
    # apply kernel that runs every operation on the FP64 pipe (no slicing; an
    # operator path independent of the one inside the solves)
    def true_relres(xx):
        return float((b - mesh.apply(xx, fp64_pipe=True)).norm() / b.norm())

    relres_true = {k: true_relres(v) for k, v in rec["x_last"].items()}
    del rec["x_last"]
    batched = batched_solves(P, m, b, opts_mixed, opts_fp64, stream) if not args.no_extras else {}
    ins = ins_measure(P, 2, 3) if (not args.no_extras and world == 1) else None

    pk = peaks()
    bytes64, flops = algo_per_element(N, 8)
    bytes32, _ = algo_per_element(N, 4)
    ax = {}
    for k in ("poisson_f64", "poisson_f32", "helmholtz_f64", "helmholtz_f32"):
        ms = float(np.mean(rec[k]))
        bpe = bytes64 if k.endswith("f64") else bytes32
        fl = flops + (2 * Np * Np if k.startswith("helmholtz") else 0)
        ax[k] = {"ms": ms, "gdofs": K * Np / (ms * 1e-3) / 1e9,
                 "hbm_frac": K * bpe / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                 "gflops": K * fl / (ms * 1e-3) / 1e9}
    value = job_gdofs(world, K, Np, ax_ms_max)
    fp64_ms = ax["poisson_f64"]["ms"]
    achieved = K * flops / (fp64_ms * 1e-3) / 1e9
    # BF16 MMA flops the tensor-core FP64 apply issues per launch at N=8 (Poisson):
    # 36 slice products x 2 flops x padded (rows x depth) of its two products (the
    # tcgen05 kernel pads the depth to 32-column chunks, the mma.sync one to 16)
    k64 = mesh.kernel(N, P.DG_F64, 0)
    tc_flops = 36 * 2 * ((96 * 64 + 48 * 192) if k64 == P.KERNEL_TC64 else (96 * 48 + 48 * 176)) * K
    algo_gbs = K * bytes64 / (fp64_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512 jittered grid (jitter 0.1h, seed 0), 524288 triangles, N=8 (Np=45), "
                               "Dirichlet; Poisson apply FP64 (value), FP32, Helmholtz, pMG-FCG solves",
                   "K": K, "N": N, "Np": Np, "batch": 1, "pmg_degrees": PMG_DEGREES,
                   "fp64_kernel": KERNEL_NAMES.get(mesh.kernel(N, P.DG_F64, 0), "?"),
                   "fp32_kernel": KERNEL_NAMES.get(mesh.kernel(N, P.DG_F32, 0), "?"),
                   "l2": "256 MB buffer written before every timed launch",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "ax": ax,
        "pcg_solve_ms": {"mixed": float(np.mean(rec["solve_mixed"])), "fp64": float(np.mean(rec["solve_fp64"])),
                         "mixed_host_loop": float(np.mean(rec["solve_mixed_host_loop"])),
                         "graph": "whole solve as one CUDA graph with device-side loops (host loop beside it)",
                         "iters_mixed": int(rec["solve_mixed_iters"][-1]),
                         "iters_fp64": int(rec["solve_fp64_iters"][-1]),
                         "coarse_iters_mixed": int(rec["solve_mixed_coarse"][-1]),
                         "coarse_iters_fp64": int(rec["solve_fp64_coarse"][-1]),
                         "relres_mixed": float(rec["solve_mixed_relres"][-1]),
                         "relres_fp64": float(rec["solve_fp64_relres"][-1]),
                         "relres_true_mixed": relres_true["mixed"],
                         "relres_true_fp64": relres_true["fp64"],
                         "relres_true_how": "||b - A x|| / ||b|| with the FP64-pipe tile kernel (DG_F64_DFMA)",
                         "batched": batched},
        # the dominant kernel against the metric's own roof: the method's algorithmic
        # bytes per apply (read u, write A u, 4 geometry words, 3 neighbour ids per
        # element) over the measured HBM copy bandwidth
        "roofline": {"bound": "hbm", "achieved": algo_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": algo_gbs / pk["hbm_gbs"],
                     # DRAM bytes read + written per apply in one ncu capture of the current
                     # kernels on this workload; None while the kernels differ from that capture
                     "traffic": TENSOR_APPLY_TRAFFIC,
                     "algorithmic_bytes": K * bytes64,
                     "kernel": "FP64 Poisson apply, N=8 (default kernel sequence; see config.fp64_kernel)",
                     "peak_src": pk["hbm_src"] + " HBM copy bandwidth (MEASURED_PEAKS.json)",
                     "fp64_equiv_tflops": achieved / 1e3,
                     "fp64_pipe_peak_tflops": pk["fp64_gflops"] / 1e3,
                     # the FP64 emulation's own work (BF16 slice products on padded tiles), kept
                     # apart from frac: it is work the method does not need
                     "emulation_bf16_tflops": tc_flops / (fp64_ms * 1e-3) / 1e12,
                     "emulation_bf16_frac": tc_flops / (fp64_ms * 1e-3) / 1e12 / pk["bf16_tflops"]},
        "ins_step": ins,
        "e2e": {"value": K * Np / (float(np.mean(e2e_ms)) * 1e-3) / 1e9, "unit": "GDOF/s",
                "h2d_bytes_per_step": int(uh.numel() * 8), "d2h_bytes_per_step": int(oh.numel() * 8)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, times, cores = cpu_oracle_sample(N, 2048, reps=3)
        cv = 2048 * Np / float(np.min(times)) / 1e9
        solve_ms, solve_it, solve_rr = cpu_oracle_solve_c1()
        one = cpu_oracle_one_core()
        line["cpu_baseline"] = {"value": cv, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                                "sample": "FP64 oracle Poisson apply on 2048 of the 524288 elements (numpy)",
                                "nproc": os.cpu_count(),
                                "value_1core": one.get("apply_gdofs"),
                                "solve_c1_ms": solve_ms, "solve_c1_iters": solve_it, "solve_c1_relres": solve_rr,
                                "solve_c1_ms_1core": one.get("solve_c1_ms"),
                                "solve_c1": "oracle Jacobi-PCG, 512 triangles, N=3, to 1e-10 (matrix-free)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_solves(P, m, b, opts_mixed, opts_fp64, stream, batches=(4, 16)):
    """The N=8 pressure solve with B right-hand sides in one batched solve
    (mixed and plain FP64), once to capture the graph and once timed, on a
    mesh of its own (destroyed after each B, which frees its workspaces); the
    right-hand sides are b scaled by 1, 1/2, 1/3, ... (every one converges
    on its own). Per B: ms of the solve, ms per right-hand side, iterations,
    largest recurrence and true relative residual (FP64-pipe apply)."""
    import torch
    out = {}
    for B in batches:
        mesh = P.Mesh.from_inputs(m, 8)
        bb = torch.stack([b / (i + 1) for i in range(B)])

        def true_relres(xx):
            r = bb - mesh.apply(xx, fp64_pipe=True)
            return float((r.norm(dim=(1, 2)) / bb.norm(dim=(1, 2))).max())

        for key, opts in (("mixed", opts_mixed), ("fp64", opts_fp64)):
            x = torch.zeros_like(bb)
            mesh.solve(bb, x, opts=opts)
            x.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = mesh.solve(bb, x, opts=opts)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[f"B{B}_{key}"] = {"ms": ms, "ms_per_rhs": ms / B, "iters": max(info["iters"]),
                                  "relres": max(info["relres"]), "relres_true": true_relres(x)}
            del x
        del bb
        mesh.close()
        torch.cuda.empty_cache()
    return out


def ins_measure(P, warmup, steps):
    """ms per dg_ins_step on the 64x64 Kovasznay workload (8,192 triangles,
    N=8, Re=40, dt=0.01, 32 LSERK substeps), velocity and pressure solves by
    mixed-precision pMG-FCG (8->4->1, Chebyshev degree 3, one AMG-preconditioned
    coarse iteration) to 1e-10; and the velocity's distance from the closed
    form after the timed steps."""
    import torch
    from dg_inputs import config_mesh
    from dg_inputs.fields import kovasznay
    from dg_inputs.mesh import ins_pressure_tags
    m, N = config_mesh("c3_ins_8192tri_N8")
    mp = ins_pressure_tags(m, dirichlet_sides=(1,))
    mu_l, mp_l = P.Mesh.from_inputs(m, N), P.Mesh.from_inputs(mp, N)
    nu, fu, fv, fp = kovasznay(40.0)
    x, y = mu_l.nodes()
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    U0 = torch.from_numpy(np.stack([fu(xh, yh), fv(xh, yh)])).cuda()
    P0 = torch.from_numpy(fp(xh, yh)).cuda()
    o = dict(precond=P.PREC_PMG, degrees=[N, N // 2, 1], cheb_degree=3, coarse_amg=1, coarse_max_iter=1,
             tol=1e-10, max_iter=500, mixed=1)
    st = P.InsStepper(mu_l, mp_l, nu, 0.01, 32, U0.clone(), P0.clone(), U0.clone(), P0.clone(),
                      vel_opts=P._binding.default_opts(**o), pr_opts=P._binding.default_opts(**o))
    st.step(warmup)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("ins_steps")
    out = st.step(steps)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    err = float((st.U - U0).abs().max())
    return {"workload": "64x64 Kovasznay, 8192 triangles, N=8, dt=0.01, 32 substeps", "steps": steps,
            "ms_per_step": out["ms"] / steps, "vel_iters": out["vel_iters"], "pr_iters": out["pr_iters"],
            "max_err_u": err}


def run_apply_only(args):
    """Only the N=8 Poisson applies (FP64 then FP32), for profiler captures."""
    import torch
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    from dg_inputs import config_mesh, uniform_field
    build.build()
    m, _ = config_mesh(MESH_NAME)
    N = args.degree
    mesh = P.Mesh.from_inputs(m, N)
    kn = {"tile": P.KERNEL_TILE, "gemm": P.KERNEL_GEMM, "tensor": P.KERNEL_TENSOR, "ept": P.KERNEL_EPT,
          "tensor_pipe": P.KERNEL_TENSOR_PIPE, "tc05": P.KERNEL_TC05, "tc64": P.KERNEL_TC64}
    if args.kernel64:
        mesh.set_kernel(N, P.DG_F64, 0, kn[args.kernel64])
    if args.kernel32:
        mesh.set_kernel(N, P.DG_F32, 0, kn[args.kernel32])
    u64 = torch.from_numpy(uniform_field((mesh.K, mesh.Np), seed=1)).cuda()
    u32 = u64.float()
    o64, o32 = torch.empty_like(u64), torch.empty_like(u32)
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ms = {"f64": [], "f32": []}
    for it in range(args.warmup + args.steps):
        for key, u, o in (("f64", u64, o64), ("f32", u32, o32)):
            flush_buf.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mesh.apply(u, out=o)
            e1.record()
            if it == 0 and key == "f64":
                mesh.apply(u, out=o, fp64_pipe=True)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ms[key].append(e0.elapsed_time(e1))
    print(json.dumps({"apply_only": True, "N": N, "K": mesh.K, "ms_f64": float(np.mean(ms["f64"])),
                      "ms_f32": float(np.mean(ms["f32"]))}), flush=True)


def run_sweep(args):
    """Throughput sweep of the applies: N = 1..8, Poisson and Helmholtz
    (lambda = 1), FP64 and FP32, batches 1/4/16, every available kernel
    (tile, FP32 GEMM, tensor-core FP64, element per thread). One JSON line per
    case; `default` marks the kernel the library picks without tuning."""
    import torch
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    from dg_inputs import config_mesh, uniform_field
    build.build()
    m, _ = config_mesh(MESH_NAME)
    pk = peaks()
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    degrees = [int(d) for d in args.sweep_degrees.split(",")]
    batches = [int(b) for b in args.sweep_batches.split(",")]
    names = {P.KERNEL_TILE: "tile", P.KERNEL_GEMM: "gemm", P.KERNEL_TENSOR: "tensor", P.KERNEL_EPT: "ept",
             P.KERNEL_TENSOR_PIPE: "tensor_pipe", P.KERNEL_TC05: "tc05", P.KERNEL_TC64: "tc64"}
    for N in degrees:
        mesh = P.Mesh.from_inputs(m, N)
        K, Np = mesh.K, mesh.Np
        for B in batches:
            u64 = torch.from_numpy(uniform_field((B, K, Np), seed=1)).cuda()
            u32 = u64.float()
            o64, o32 = torch.empty_like(u64), torch.empty_like(u32)
            for lam in (0.0, 1.0):
                for key, prec, u, o in (("f64", P.DG_F64, u64, o64), ("f32", P.DG_F32, u32, o32)):
                    default = mesh.kernel(N, prec, lam != 0.0)
                    for k in mesh.kernels_available(N, prec):
                        mesh.set_kernel(N, prec, lam != 0.0, k)
                        ms = []
                        for it in range(args.warmup + args.steps):
                            flush_buf.fill_(1.0)
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            e0.record()
                            mesh.apply(u, lam=lam, out=o)
                            e1.record()
                            torch.cuda.synchronize()
                            if it >= args.warmup:
                                ms.append(e0.elapsed_time(e1))
                        t = float(np.median(ms)) * 1e-3
                        word = 4 if key == "f32" else 8
                        bpe, fpe = algo_per_element(N, word)
                        fpe += 2 * Np * Np if lam else 0
                        geo = 4 * word + 12
                        nbytes = K * (B * (bpe - geo) + geo)
                        pipe_peak = pk["fp32_gflops"] if key == "f32" else pk["fp64_gflops"]
                        print(json.dumps({
                            "sweep": True, "N": N, "Np": Np, "K": K, "B": B,
                            "op": "helmholtz" if lam else "poisson", "prec": key, "kernel": names[k],
                            "default": k == default, "ms": t * 1e3, "gdofs": B * K * Np / t / 1e9,
                            "hbm_gbs": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / pk["hbm_gbs"],
                            "gflops": B * K * fpe / t / 1e9,
                            "pipe_frac": B * K * fpe / t / 1e9 / pipe_peak,
                            "t_hbm_ms": nbytes / (pk["hbm_gbs"] * 1e9) * 1e3,
                            "t_pipe_ms": B * K * fpe / (pipe_peak * 1e9) * 1e3}), flush=True)
                    mesh.set_kernel(N, prec, lam != 0.0, P.KERNEL_AUTO)
            del u64, u32, o64, o32
        del mesh
        torch.cuda.empty_cache()


def run_tet(args):
    """Tetrahedral apply throughput: 6 n^3 jittered tetrahedra (n = 32:
    196,608 elements), N = 1..5, Poisson and Helmholtz, FP64 and FP32, B = 1
    and 4, L2 flushed between launches; one JSON line per case. Algorithmic
    bytes per element: u read and Au written once (2 B Np words), the geometry
    (40 words), the connectivity (4 ints) and the neighbour node map (4 Nfp
    ints)."""
    import torch
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    from dg_inputs import uniform_field
    from dg_inputs.tetmesh import jittered_tet_grid
    build.build()
    pk = peaks()
    m = jittered_tet_grid(args.tet_n, jitter=0.1, seed=1, bc_sides=(1, 2, 2, 1, 1, 2))
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for N in [int(d) for d in args.tet_degrees.split(",")]:
        mesh = P.TetMesh.from_inputs(m, N)
        K, Np, Nfp = mesh.K, mesh.Np, (N + 1) * (N + 2) // 2
        for B in [int(b) for b in args.tet_batches.split(",")]:
            u64 = torch.from_numpy(uniform_field((B, K, Np), seed=1)).cuda()
            for key, u, pipe in (("f64", u64, False), ("f64", u64, True), ("f32", u64.float(), False)):
                o = torch.empty_like(u)
                word = u.element_size()
                for lam in (0.0, 1.0):
                    ms = []
                    for it in range(args.warmup + args.steps):
                        flush_buf.fill_(1.0)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        mesh.apply(u, lam=lam, out=o, fp64_pipe=pipe)
                        e1.record()
                        torch.cuda.synchronize()
                        if it >= args.warmup:
                            ms.append(e0.elapsed_time(e1))
                    t = float(np.median(ms)) * 1e-3
                    nbytes = K * (2 * B * Np * word + 40 * word + 4 * 4 + 4 * Nfp * 4)
                    print(json.dumps({
                        "tet": True, "N": N, "Np": Np, "K": K, "B": B, "op": "helmholtz" if lam else "poisson",
                        "prec": key, "kernel": ("fp64_pipe" if pipe or (key == "f64" and N <= 2)
                                                else ("tc64" if key == "f64" else "cuda_cores")),
                        "default": not pipe,
                        "ms": t * 1e3, "gdofs": B * K * Np / t / 1e9,
                        "hbm_gbs": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / pk["hbm_gbs"]}), flush=True)
            del u64
        del mesh
        torch.cuda.empty_cache()


def run_solve_only(args):
    """One mixed-precision pMG-FCG solve on the N=8 workload inside an NVTX
    range "timed_solve" (after a set-up solve), for per-kernel launch lists."""
    import torch
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    from dg_inputs import config_mesh, manufactured
    build.build()
    m, _ = config_mesh(MESH_NAME)
    mesh = P.Mesh.from_inputs(m, 8)
    xn, yn = mesh.nodes()
    uex, fex = manufactured("sin_2pi_x_cos_3pi_y")
    xh, yh = xn.cpu().numpy(), yn.cpu().numpy()
    dev = xn.device
    b = mesh.rhs(torch.from_numpy(fex(xh, yh)).to(dev), torch.from_numpy(uex(xh, yh)).to(dev))
    opts = P._binding.default_opts(precond=P.PREC_PMG, degrees=PMG_DEGREES, tol=1e-10, max_iter=200,
                                   mixed=0 if args.fp64 else 1, cheb_degree=CHEB, coarse_max_iter=COARSE_PASSES,
                                   coarse_amg=1, graph=args.graph)
    mesh.solve(b, torch.zeros_like(b), opts=opts)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_solve")
    _, info = mesh.solve(b, torch.zeros_like(b), opts=opts)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"solve_only": True, "mixed": not args.fp64, "graph": args.graph, "ms": info["ms"],
                      "iters": info["iters"][0], "coarse_iters": info["coarse_iters"]}), flush=True)


def run_amg_compare(args):
    """Section 3's preconditioner comparison on the 32768-triangle N=6 workload
    (128x128 jittered grid): p-multigrid 6->3->1 with algebraic multigrid on the
    degree-1 level (FP32 levels and FP64), against algebraic multigrid alone on
    the probed degree-6 matrix. One JSON line per preconditioner: outer
    iterations, solve time (set-up excluded: a first solve builds the
    hierarchy), wall time of that first solve, device bytes of the
    preconditioner per element."""
    import time
    import torch
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    from dg_inputs import config_mesh, manufactured
    build.build()
    m, N = config_mesh("c2_pmg_32768tri_N6")
    mesh = P.Mesh.from_inputs(m, N)
    xn, yn = mesh.nodes()
    uex, fex = manufactured("sin_2pi_x_cos_3pi_y")
    xh, yh = xn.cpu().numpy(), yn.cpu().numpy()
    dev = xn.device
    b = mesh.rhs(torch.from_numpy(fex(xh, yh)).to(dev), torch.from_numpy(uex(xh, yh)).to(dev))
    cases = (("pmg_amg_mixed", dict(precond=P.PREC_PMG, degrees=[6, 3, 1], coarse_amg=1, mixed=1)),
             ("pmg_amg_fp64", dict(precond=P.PREC_PMG, degrees=[6, 3, 1], coarse_amg=1, mixed=0)),
             ("amg", dict(precond=P.PREC_AMG)))
    for name, kw in cases:
        opts = P._binding.default_opts(tol=1e-10, max_iter=1000, **kw)
        t0 = time.time()
        mesh.solve(b, torch.zeros_like(b), opts=opts)
        torch.cuda.synchronize()
        first = time.time() - t0
        _, info = mesh.solve(b, torch.zeros_like(b), opts=opts)
        print(json.dumps({"amg_compare": True, "precond": name, "K": mesh.K, "N": N, "iters": info["iters"][0],
                          "relres": info["relres"][0], "ms": info["ms"], "first_solve_s": first,
                          "precond_bytes_per_element": info["precond_bytes"] / mesh.K}), flush=True)


def run_ins(args):
    """The split INS step on the 64x64 Kovasznay workload alone (see ins_measure)."""
    import paper_1801_00246_gb300 as P
    from paper_1801_00246_gb300 import build
    build.build()
    print(json.dumps(dict(ins=True, **ins_measure(P, args.warmup, args.steps))), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched solves and the INS step measured after the timed region")
    ap.add_argument("--apply-only", action="store_true", help="only the Poisson applies (profiling)")
    ap.add_argument("--degree", type=int, default=8, help="degree for --apply-only")
    ap.add_argument("--kernel64", default="", help="--apply-only: FP64 kernel (tile, tensor, tensor_pipe, ept, tc64)")
    ap.add_argument("--kernel32", default="", help="--apply-only: FP32 kernel (tile, gemm, tensor, tensor_pipe, ept, tc05)")
    ap.add_argument("--sweep", action="store_true", help="apply throughput for N=1..10, FP64/FP32, B=1/4/16")
    ap.add_argument("--solve-only", action="store_true", help="one N=8 pMG-FCG solve in an NVTX range (profiling)")
    ap.add_argument("--graph", type=int, default=1, help="--solve-only: 1 = CUDA-graph solve, 0 = host loop")
    ap.add_argument("--fp64", action="store_true", help="--solve-only: FP64 multigrid levels")
    ap.add_argument("--ins", action="store_true", help="time dg_ins_step on the 8192-triangle Kovasznay case")
    ap.add_argument("--oracle-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--amg-compare", action="store_true",
                    help="pMG-AMG against AMG alone on the 32768-triangle N=6 workload")
    ap.add_argument("--tet", action="store_true", help="tetrahedral apply throughput, N = 1..5")
    ap.add_argument("--tet-n", type=int, default=32, help="--tet: cubes per side (6 n^3 tetrahedra)")
    ap.add_argument("--tet-degrees", default="1,2,3,4,5")
    ap.add_argument("--tet-batches", default="1,4")
    ap.add_argument("--sweep-degrees", default="1,2,3,4,5,6,7,8,9,10")
    ap.add_argument("--sweep-batches", default="1,4,16")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.apply_only:
        run_apply_only(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.tet:
        run_tet(args)
        return
    if args.solve_only:
        run_solve_only(args)
        return
    if args.ins:
        run_ins(args)
        return
    if args.amg_compare:
        run_amg_compare(args)
        return
    if args.oracle_child:
        oracle_child()
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
