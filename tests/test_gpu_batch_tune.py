"""The batched kernel's layout autotuner (sv_batch_set_autotune): every layout it may choose --
the fixed rule's team and the team with twice its warps, commuting-layer segments on or off,
diagonal segments on or off -- gives the oracle's energies and gradients, and a tuned batch
gives them too, with the layout it chose reported per qubit count."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu

FIXED_WARPS = {n: 1 if n <= 9 else 2 if n == 10 else 4 if n == 11 else 8 for n in range(1, 13)}


@pytest.fixture
def tuner():
    svqe.batch_set_autotune(True)
    yield
    svqe.batch_set_autotune(False)
    for n in range(1, 13):
        svqe.batch_set_layout(n, 0, 0, 0)


def _check(insts, b, e, g, which):
    for i in which:
        e0, g0 = oracle.energy_grad(insts[i])
        assert_energy(e[i], e0, insts[i]["ham"], insts[i]["name"])
        assert_grad(g[b.offsets[i]:b.offsets[i + 1]], g0, insts[i]["ham"], insts[i]["name"])


@pytest.mark.parametrize("n", [4, 6, 9, 10, 11])
def test_every_candidate_layout_matches_the_oracle(tuner, n):
    insts = [W.hea_instance(n, 2 + s % 3, 60 + 20 * s, 300 + n, stream=s) for s in range(6)]
    warps = [FIXED_WARPS[n]] + ([2 * FIXED_WARPS[n]] if FIXED_WARPS[n] < 8 else [])
    for w in warps:
        for ml in (2, svqe.SEG_OFF):
            for md in (3, svqe.SEG_OFF):
                svqe.batch_set_layout(n, w, ml, md)
                b = svqe.Batch(insts)
                assert b.layout(n) == (w, ml, md)
                e, g = b.run(b.theta_of(insts))
                _check(insts, b, e, g, (0, 5))
                b.close()


def test_tuned_mixed_batch_matches_the_oracle(tuner):
    insts = W.hea_batch(180)
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    sample = []
    for n in range(4, 13):
        idx = [i for i, it in enumerate(insts) if it["circuit"]["n"] == n]
        w, ml, md = b.layout(n)
        if not idx:
            assert (w, ml, md) == (0, 0, 0)
            continue
        assert w in (FIXED_WARPS[n], 2 * FIXED_WARPS[n]) and ml in (2, svqe.SEG_OFF)
        assert md in (3, svqe.SEG_OFF)
        sample.append(idx[0])
    _check(insts, b, e, g, sample)
    # the cache answers the next tuned batch with the same layouts
    b2 = svqe.Batch(insts[:40])
    for n in range(4, 13):
        if b2.layout(n)[0]:
            assert b2.layout(n) == b.layout(n)
    b.close()
    b2.close()
