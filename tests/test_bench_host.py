"""Host-side logic of bench.py: the multi-rank aggregation (replicas, weak
scaling; world_size 2 over gloo on CPU), the reference arm's JSON line, and
the launch count and NTT work it derives from the library's plan."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]  # rank 1 is the slower replica
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    q.put((rank, ms, bench.aggregate_rate(1 << 30, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 180.0                              # max over ranks
        assert rate == pytest.approx(2 * (1 << 30) / 0.180 / 1e9)  # both ranks' bits / slowest time


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "small_n2^24_m64_s2^18_k2^17", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Gbit/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_launch_count_and_ntt_work_follow_the_plan_string():
    """gpu_launches and the NTT roofline's work are derived from the plan the
    library describes: the gather form (two bucket stages, window passes or
    plain passes), the launch groups, and whether seed windows are
    transformed per run."""
    import importlib
    bench = importlib.import_module("bench")
    ntt = ("ntt: N=1048576 (512 x 2048) P=2 pieces per sub-block, 16 sub-blocks per launch group, prime "
           "7*2^26+1, %s; sms=152; gather=%s")
    shared_buckets = ntt % ("shared seed spectrum", "buckets (2^16-bit chunks, 40548-word sub-block regions)")
    assert bench.launches_per_step(True, 1024, shared_buckets, 1 << 30) == 2 + 3 * 64
    windows = ntt % ("shared seed spectrum", "windows (8 input windows)")
    assert bench.launches_per_step(True, 4096, windows, 1 << 32) == 8 + 3 * 256
    plain_big = ntt % ("shared seed spectrum", "plain")
    assert bench.launches_per_step(True, 4096, plain_big, 1 << 32) == 4 * 256   # a gather per group
    plain_small = ntt % ("shared seed spectrum", "plain")
    assert bench.launches_per_step(True, 64, plain_small, 1 << 24) == 1 + 3 * 4
    direct = "lop3 tile: rows=1024 ... w_pad=32768 sms=152; gather=plain"
    assert bench.launches_per_step(False, 128, direct, 1 << 30) == 2 + 1       # two input windows + hash
    assert bench.launches_per_step(False, 128, direct, 1 << 27) == 1 + 1
    m, s, k = 1024, 1 << 20, 1 << 19
    per_run = ntt % ("seed windows transformed per run (one seed per sub-block)", "plain")
    resident = ntt % ("seed spectra resident (one seed per sub-block)", "plain")
    w_shared = bench.ntt_roofline(1 << 30, m, s, k, 10.0, shared_buckets)["work_per_launch"]
    w_per_run = bench.ntt_roofline(1 << 30, m, s, k, 10.0, per_run)["work_per_launch"]
    w_resident = bench.ntt_roofline(1 << 30, m, s, k, 10.0, resident)["work_per_launch"]
    assert "m x 3 transforms" in w_shared and "m x 3 transforms" in w_resident
    assert "m x 5 transforms" in w_per_run
    bfly = m * 3 * (1 << 19) * 20
    r = bench.ntt_roofline(1 << 30, m, s, k, 10.0, shared_buckets)
    assert abs(r["achieved"] - bfly / 1e-2 / 1e12) < 1e-9 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
