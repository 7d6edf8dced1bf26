"""GPU tests of the continuous-batching request loop: results match the oracle per step,
each request's result is the same alone and in a mix (bit for bit), admission respects the
HBM budget, and the host-side failure paths (bad request, oversized request, cancellation,
bounded wait) return their status without touching a kernel."""
import time

import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def _mix():
    reqs = W.serve_stream(24, 1000.0, seed=77, max_qubits=16, steps=5)
    reqs += [dict(W.hea_instance(14, 2, 40, 5), steps=4,
                  lr=0.05, name="big14", arrival_s=0.0)]
    return reqs


def test_results_match_oracle_per_step():
    srv = svqe.Server(steps_per_tick=2)
    reqs = W.serve_stream(10, 1000.0, seed=78, max_qubits=14, steps=3)
    ids = [srv.submit(r, r["steps"], r["lr"]) for r in reqs]
    for r, rid in zip(reqs, ids):
        th, es, info = srv.wait(rid, 60000)
        assert info.status == 0
        theta = np.array(r["theta"], dtype=np.float64)
        for t in range(r["steps"]):
            e0, g0 = oracle.energy_grad(r, theta)
            assert_energy(es[t], e0, r["ham"], f"{r['name']} step {t}")
            theta = theta - r["lr"] * g0
        assert_grad((np.asarray(r["theta"]) - th) / r["lr"],
                    (np.asarray(r["theta"]) - theta) / r["lr"], r["ham"])
    srv.close()


def test_same_result_alone_and_in_the_mix():
    reqs = _mix()
    mixed = svqe.Server(steps_per_tick=2)
    ids = [mixed.submit(r, r["steps"], r["lr"]) for r in reqs]
    out_mix = [mixed.wait(i, 120000) for i in ids]
    mixed.close()
    for k in (0, 3, 11, len(reqs) - 1):
        alone = svqe.Server(serial=True)
        th, es, _ = alone.wait(alone.submit(reqs[k], reqs[k]["steps"], reqs[k]["lr"]), 120000)
        alone.close()
        assert np.array_equal(th, out_mix[k][0]), reqs[k]["name"]
        assert np.array_equal(es, out_mix[k][1]), reqs[k]["name"]


def test_admission_respects_the_budget():
    reqs = [dict(W.hea_instance(12, 4, 300, s), steps=6, lr=0.01) for s in range(12)]
    srv0 = svqe.Server()
    probe = srv0.submit(reqs[0], 6, 0.01)
    _, _, info = srv0.wait(probe, 60000)
    srv0.close()
    budget = int(info.footprint_bytes * 2.5)  # room for two requests at a time
    srv = svqe.Server(hbm_budget_bytes=budget)
    ids = [srv.submit(r, r["steps"], r["lr"]) for r in reqs]
    infos = [srv.wait(i, 120000)[2] for i in ids]
    st = srv.stats()
    assert st.peak_bytes_in_use <= budget
    assert st.completed == len(reqs)
    # at most two were resident at any time
    events = sorted([(i.admit_s, 1) for i in infos] + [(i.done_s, -1) for i in infos])
    live, peak = 0, 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak <= 2
    srv.close()


def test_failure_paths_are_host_side_statuses():
    srv = svqe.Server(hbm_budget_bytes=64 << 20, max_active_large=1)
    bad = W.hea_instance(5, 1, 10, 1)
    bad["circuit"]["wires"][0][0] = 9
    with pytest.raises(svqe.SvError) as e:
        srv.submit(bad, 2, 0.1)
    assert e.value.status == svqe.SV_EINVAL
    huge = W.hea_instance(24, 1, 10, 1)  # 2 x 256 MiB of state > 64 MiB budget
    with pytest.raises(svqe.SvError) as e:
        srv.submit(huge, 1, 0.1)
    assert e.value.status == svqe.SV_ENOMEM
    # one large request at a time: the second waits in the queue, so a 1 ms wait times out
    a = srv.submit(W.hea_instance(16, 4, 50, 2), 30, 0.01)
    b = srv.submit(W.hea_instance(16, 4, 50, 3), 30, 0.01)
    with pytest.raises(svqe.SvError) as e:
        srv.wait(b, 1)
    assert e.value.status == svqe.SV_ETIMEOUT
    srv.cancel(b)
    with pytest.raises(svqe.SvError):
        srv.wait(b, 1000)
    th, es, info = srv.wait(a, 120000)
    assert info.status == 0
    assert srv.stats().cancelled == 1
    srv.close()


def test_idle_contexts_are_reused_and_evicted_within_the_budget():
    """Large requests leave their buffers idle for the next request of the same width; a
    request of another width that needs the room evicts them.  Results are bit for bit those
    of a fresh server, and the budget holds throughout."""
    reqs = [dict(W.hea_instance(15, 2, 40, s), steps=3, lr=0.02) for s in (1, 2)]
    reqs += [dict(W.hea_instance(16, 2, 40, 3), steps=3, lr=0.02)]
    reqs += [dict(W.hea_instance(15, 2, 40, 4), steps=3, lr=0.02)]
    fresh = []
    for r in reqs:
        one = svqe.Server(serial=True)
        th, es, info = one.wait(one.submit(r, r["steps"], r["lr"]), 120000)
        one.close()
        fresh.append((th, es, info.footprint_bytes))
    fp15 = max(f[2] for f, r in zip(fresh, reqs) if r["circuit"]["n"] == 15)
    fp16 = fresh[2][2]
    budget = fp16 + fp15 // 2  # one request at a time; an idle 15-qubit set must go for n = 16
    srv = svqe.Server(hbm_budget_bytes=budget, serial=True)
    for r, (th0, es0, _) in zip(reqs, fresh):
        th, es, info = srv.wait(srv.submit(r, r["steps"], r["lr"]), 120000)
        assert info.status == 0
        assert np.array_equal(th, th0) and np.array_equal(es, es0), r["name"]
    theta = np.array(reqs[3]["theta"], dtype=np.float64)
    e0, _ = oracle.energy_grad(reqs[3], theta)
    assert_energy(fresh[3][1][0], e0, reqs[3]["ham"], "reused context, step 0")
    st = srv.stats()
    assert st.completed == len(reqs) and st.peak_bytes_in_use <= budget
    srv.close()


def test_heavy_requests_respect_their_quota():
    """With heavy_qubits = 14 and max_active_heavy = 1, the 14-qubit requests run one at a
    time while 13-qubit and batched requests run beside them; every result is bit for bit the
    serial server's."""
    reqs = [dict(W.hea_instance(14, 2, 40, s), steps=3, lr=0.02) for s in (11, 12, 13)]
    reqs += [dict(W.hea_instance(13, 2, 40, s), steps=3, lr=0.02) for s in (21, 22)]
    reqs += [dict(W.hea_instance(8, 2, 40, s), steps=3, lr=0.02) for s in (31, 32)]
    srv = svqe.Server(max_active_large=4, max_active_heavy=1, heavy_qubits=14)
    ids = [srv.submit(r, r["steps"], r["lr"]) for r in reqs]
    out = [srv.wait(i, 120000) for i in ids]
    srv.close()
    heavy = sorted((o[2].admit_s, o[2].done_s) for o in out if o[2].n_qubits == 14)
    for (a0, d0), (a1, d1) in zip(heavy, heavy[1:]):
        assert a1 >= d0  # admitted only after the previous heavy request finished
    for r, (th, es, info) in zip(reqs, out):
        assert info.status == 0
        one = svqe.Server(serial=True)
        th0, es0, _ = one.wait(one.submit(r, r["steps"], r["lr"]), 120000)
        one.close()
        assert np.array_equal(th, th0) and np.array_equal(es, es0), r["name"]


def test_bench_stream_sampled_against_the_oracle():
    """The serving benchmark's own seeded stream (60 requests, n = 4-24, 20 steps each),
    submitted at once to a default server.  Sampled requests of 4-13 qubits are replayed
    step by step with the oracle's gradient (energy before every update, final theta); the
    24-qubit request matches the serial server bit for bit and its first energy matches the
    oracle."""
    reqs = W.serve_stream(60, 1.0, seed=1005)
    srv = svqe.Server(hbm_budget_bytes=64 << 30, steps_per_tick=2)
    ids = [srv.submit(r, r["steps"], r["lr"]) for r in reqs]
    out = [srv.wait(i, 600000) for i in ids]
    srv.close()
    ns = [r["circuit"]["n"] for r in reqs]
    sample = []
    for n in (4, 5, 7, 10, 13):
        sample.append(ns.index(n))
    for k in sample:
        r, (th, es, info) = reqs[k], out[k]
        assert info.status == 0
        theta = np.array(r["theta"], dtype=np.float64)
        for t in range(r["steps"]):
            e0, g0 = oracle.energy_grad(r, theta)
            assert_energy(es[t], e0, r["ham"], f"{r['name']} step {t}")
            theta = theta - r["lr"] * g0
        assert_grad((np.asarray(r["theta"]) - th) / r["lr"],
                    (np.asarray(r["theta"]) - theta) / r["lr"], r["ham"], r["name"])
    big = max(range(len(reqs)), key=lambda i: ns[i])
    one = svqe.Server(serial=True)
    th0, es0, _ = one.wait(one.submit(reqs[big], reqs[big]["steps"], reqs[big]["lr"]), 600000)
    one.close()
    assert np.array_equal(out[big][0], th0) and np.array_equal(out[big][1], es0)
    assert_energy(out[big][1][0], oracle.energy(reqs[big]), reqs[big]["ham"], reqs[big]["name"])
