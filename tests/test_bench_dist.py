"""The benchmark's multi-rank path on CPU: two gloo ranks (one process per
GPU on a real node) reduce their timings with a max, the whole-job value
counts every replica's nodes, and only rank 0 runs the oracle arm."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx = bench.ranks_max([1.0 + rank, 10.0 - rank, 3.0], "cpu")

    class A:
        gpus, steps, warmup = world, 1, 3

    out = bench.run_reference(A, world, rank) if rank != 0 else "rank0"
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, out))


def test_two_gloo_ranks_reduce_with_max_and_rank0_reports():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict((r, (mx, out)) for r, mx, out in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r][0] == [2.0, 10.0, 3.0]  # element-wise max over ranks
    assert res[1][1] is None                   # rank 1 runs nothing for the oracle arm


def test_job_value_counts_every_replica():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    K, Np = 524288, 45
    one = bench.job_gdofs(1, K, Np, 3.0)
    assert bench.job_gdofs(4, K, Np, 3.0) == pytest.approx(4 * one)
    assert one == pytest.approx(K * Np / 3e-3 / 1e9)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys the benchmark contract names."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"] and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_clock_summary_reads_nvidia_smi_samples(tmp_path):
    """The clocks record of the JSON line: median SM clock over the loaded
    samples (idle samples below half the peak are left out), the maximum clock,
    and every throttle reason seen Active; malformed lines are skipped."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    path = tmp_path / "clocks.csv"
    na = "Not Active"
    lines = ["0, 345, 2070, 120.5, 0x0, %s, %s, %s, %s" % (na, na, na, na),
             "0, 2070, 2070, 900.1, 0x0, %s, %s, %s, %s" % (na, na, na, na),
             "0, 1980, 2070, 1390.0, 0x4, %s, %s, %s, Active" % (na, na, na),
             "0, 2055, 2070, 1200.0, 0x0, %s, %s, %s, %s" % (na, na, na, na),
             "garbage line",
             "0, [N/A], 2070, 0, 0x0, %s, %s, %s, %s" % (na, na, na, na)]
    path.write_text("\n".join(lines) + "\n")
    c = bench.Clocks(0)
    c.path = str(path)
    c.proc = object()  # as if the sampler had run
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    path.write_text("")
    assert bench.Clocks.summary(c)["reasons"] == ["no samples"]
    c.proc = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]
