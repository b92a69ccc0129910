"""Serving: continuous batching under a device-memory budget.

Every job's output must be the same when it is served alone, when it is
served in a mix of overlapping jobs, and as extract_run / the oracle give it.
Budget admission, refusal, timeouts and concurrent submitters are exercised
on the host side (no GPU fault is involved)."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2308_02856_gb300 import build as pkg_build
from paper_2308_02856_gb300 import extract as X
from paper_2308_02856_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg_build.build()
    X.load()


def _dev(words):
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _jobs(count, seed, n_lo, n_hi, s_set):
    shapes = synth.job_shapes(count, seed, n_lo, n_hi, s_set=s_set)
    jobs, ins = [], []
    for j in shapes:
        j = dict(j)
        j["seed"] = synth.uniform_bits(j["s"] + j["k"] - 1, j["seed_seed"])
        jobs.append(j)
        ins.append(_dev(synth.bernoulli_bits(j["n"], j["p"], j["in_seed"])))
    return jobs, ins


def _out(j, fill=-1):
    return torch.full(((j["m"] * j["k"] + 31) // 32,), fill, dtype=torch.int32, device="cuda")


def test_each_result_is_the_same_alone_and_in_the_mix():
    jobs, ins = _jobs(40, 51, 2 ** 12, 2 ** 23, (1 << 10, 1 << 12, 1 << 14, 1 << 16))
    # every job served alone
    alone = []
    with X.Server(8 << 30, max_slots=4) as srv:
        for j, d in zip(jobs, ins):
            o = _out(j)
            srv.wait(srv.submit(j, d, o))
            alone.append(_host(o))
    # all jobs served in a mix: Poisson arrivals, many in flight at once
    arrivals = synth.poisson_arrivals(len(jobs), 2000.0, 52)
    mixed = [_out(j, fill=7) for j in jobs]
    with X.Server(8 << 30, max_slots=16, wave_us=500) as srv:
        t0 = time.perf_counter()
        tickets = []
        for j, d, o, ta in zip(jobs, ins, mixed, arrivals):
            while time.perf_counter() - t0 < ta:
                pass
            tickets.append(srv.submit(j, d, o))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["waves"] > 1
    for i, (j, d) in enumerate(zip(jobs, ins)):
        got = _host(mixed[i])
        assert np.array_equal(got, alone[i]), "job %d differs in the mix" % i
        with X.Extractor(j["n"], j["m"], j["s"], j["k"], j["seed"], j["key"]) as ex:
            assert np.array_equal(got, _host(ex.run(d))), "job %d differs from extract_run" % i
    # and the small ones against the oracle
    small = sorted(range(len(jobs)), key=lambda i: jobs[i]["n"] * jobs[i]["k"])[:6]
    for i in small:
        j = jobs[i]
        w = ins[i].cpu().numpy().view(np.uint32)
        want = oracle.extract(j["n"], j["m"], j["s"], j["k"], w, j["seed"], j["key"])
        assert np.array_equal(_host(mixed[i]), want), "job %d vs oracle" % i


def test_budget_limits_admission_and_refuses_oversize_jobs():
    jobs, ins = _jobs(12, 61, 2 ** 18, 2 ** 20, (1 << 12, 1 << 14))
    need = max(j["n"] * 4 + j["n"] // 8 * 2 + j["m"] * j["k"] // 8 + (1 << 20) for j in jobs)
    budget = int(need * 2.5)  # about two jobs at a time
    outs = [_out(j) for j in jobs]
    with X.Server(budget, max_slots=64) as srv:
        tickets = [srv.submit(j, d, o) for j, d, o in zip(jobs, ins, outs)]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
        assert st["bytes_peak"] <= budget
        assert st["completed"] == len(jobs)
        # a job that can never fit is refused at once
        big = dict(jobs[0])
        big["n"], big["m"] = budget * 2, 1  # order alone is 8x the budget
        big["s"], big["k"] = jobs[0]["s"], jobs[0]["k"]
        with pytest.raises(X.ExtractError) as e:
            srv.submit(big, ins[0], outs[0])
        assert e.value.code == X.EXTRACT_EBUDGET
        assert srv.stats()["rejected"] == 1
    for j, d, o in zip(jobs, ins, outs):
        with X.Extractor(j["n"], j["m"], j["s"], j["k"], j["seed"], j["key"]) as ex:
            assert np.array_equal(_host(o), _host(ex.run(d)))


def test_wait_times_out_then_completes():
    n, m, s, k = 1 << 26, 64, 1 << 20, 1 << 18   # ~0.1 s of hashing
    j = {"n": n, "m": m, "s": s, "k": k, "key": 5, "seed": synth.uniform_bits(s + k - 1, 9)}
    d = _dev(synth.bernoulli_bits(n, 0.7, 8))
    o = _out(j)
    with X.Server(16 << 30, max_slots=4) as srv:
        t = srv.submit(j, d, o)
        with pytest.raises(X.ExtractError) as e:
            srv.wait(t, timeout_ms=0)
        assert e.value.code == X.EXTRACT_ETIMEDOUT
        lat = srv.wait(t)
        assert lat > 0
    with X.Extractor(n, m, s, k, j["seed"], 5) as ex:
        assert np.array_equal(_host(o), _host(ex.run(d)))


def test_concurrent_submitters_and_bad_jobs():
    jobs, ins = _jobs(24, 71, 2 ** 14, 2 ** 21, (1 << 12, 1 << 14, 1 << 16))
    outs = [_out(j) for j in jobs]
    errors = []
    with X.Server(8 << 30, max_slots=12, wave_us=300) as srv:
        def worker(idx):
            try:
                ts = [srv.submit(jobs[i], ins[i], outs[i]) for i in idx]
                for t in ts:
                    srv.wait(t)
            except Exception as ex:  # surfaced below
                errors.append(ex)
        th = [threading.Thread(target=worker, args=(list(range(w, len(jobs), 4)),)) for w in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        bad = dict(jobs[0])
        bad["k"] = bad["s"] + 1
        with pytest.raises(X.ExtractError) as e:
            srv.submit(bad, ins[0], outs[0])
        assert e.value.code == X.EXTRACT_EINVAL
    assert not errors
    for j, d, o in zip(jobs, ins, outs):
        with X.Extractor(j["n"], j["m"], j["s"], j["k"], j["seed"], j["key"]) as ex:
            assert np.array_equal(_host(o), _host(ex.run(d)))


def test_server_ntt_lane_and_waves_give_the_same_bits():
    """Large-s jobs take the NTT lane, small ones the direct waves; all run
    at once and every output equals extract_run's."""
    shapes = synth.job_shapes(16, 81, 2 ** 18, 2 ** 22, s_set=(1 << 12, 1 << 18, 1 << 20))
    jobs, ins = [], []
    for j in shapes:
        j = dict(j)
        j["seed"] = synth.uniform_bits(j["s"] + j["k"] - 1, j["seed_seed"])
        jobs.append(j)
        ins.append(_dev(synth.bernoulli_bits(j["n"], j["p"], j["in_seed"])))
    assert any(j["s"] >= (1 << 18) for j in jobs) and any(j["s"] < (1 << 18) for j in jobs)
    outs = [_out(j) for j in jobs]
    with X.Server(16 << 30, max_slots=16, wave_us=500) as srv:
        tickets = [srv.submit(j, d, o) for j, d, o in zip(jobs, ins, outs)]
        for t in tickets:
            srv.wait(t)
        assert srv.stats()["completed"] == len(jobs)
    for j, d, o in zip(jobs, ins, outs):
        with X.Extractor(j["n"], j["m"], j["s"], j["k"], j["seed"], j["key"], X.EXTRACT_METHOD_DIRECT) as ex:
            assert np.array_equal(_host(o), _host(ex.run(d)))
