"""Seeded random circuits of every gate type, in random order, against the oracle: runs of
RZ/CZ (diagonal segments, CZ included), runs of CNOT/X (permutation segments, X included),
RY/RX layers cut short by a repeated qubit, H, SingleExcitation and DoubleExcitation, fixed
angles and shared parameters.  On the batched kernel (1-12 qubits, every team class) and on
the single-state path with fused passes and whole-state segments (14-16 qubits)."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def random_instance(n, seed, n_blocks=10, n_terms=40):
    rng = np.random.default_rng([seed, n])
    cb = W.CircuitBuilder(n)
    params = []

    def param():
        if params and rng.random() < 0.15:  # a shared parameter
            return int(rng.choice(params))
        if rng.random() < 0.1:  # a fixed angle
            return None
        p = cb.n_params
        params.append(p)
        return "new"

    for _ in range(n_blocks):
        kind = rng.integers(0, 6)
        if kind == 0:  # diagonal run
            for _ in range(int(rng.integers(1, 2 * n + 2))):
                if n >= 2 and rng.random() < 0.3:
                    a, b = rng.choice(n, 2, replace=False)
                    cb.add(W.CZ, (int(a), int(b)))
                else:
                    cb.add(W.RZ, (int(rng.integers(n)),), param=param(),
                           angle=float(rng.uniform(-3, 3)))
        elif kind == 1:  # permutation run
            for _ in range(int(rng.integers(1, n + 3))):
                if n >= 2 and rng.random() < 0.7:
                    a, b = rng.choice(n, 2, replace=False)
                    cb.add(W.CNOT, (int(a), int(b)))
                else:
                    cb.add(W.X, (int(rng.integers(n)),))
        elif kind == 2:  # a layer, possibly cut short by a repeated qubit
            g = W.RY if rng.random() < 0.6 else W.RX
            for q in rng.choice(n, int(rng.integers(1, n + 1)), replace=True):
                cb.add(g, (int(q),), param=param(), angle=float(rng.uniform(-3, 3)))
        elif kind == 3:
            cb.add(W.H, (int(rng.integers(n)),))
        elif kind == 4 and n >= 2:
            a, b = rng.choice(n, 2, replace=False)
            cb.add(W.SINGLE_EXC, (int(a), int(b)), param=param(), angle=float(rng.uniform(-3, 3)))
        elif kind == 5 and n >= 4:
            w = rng.choice(n, 4, replace=False)
            cb.add(W.DOUBLE_EXC, tuple(int(v) for v in w), param=param(),
                   angle=float(rng.uniform(-3, 3)))
    circ = cb.build()
    ham = W.random_pauli_sum(rng, n, n_terms, 0.5, min(4, n), 1.0)
    return {"name": f"random_n{n}_s{seed}", "circuit": circ, "ham": ham,
            "ref": int(rng.integers(0, 1 << n)),
            "theta": rng.uniform(-np.pi, np.pi, circ["n_params"])}


def _check(e, g, inst):
    e0, g0 = oracle.energy_grad(inst)
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])


def test_batched_kernel_random_circuits():
    insts = [random_instance(n, s) for n in range(1, 13) for s in range(6)]
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    for i, inst in enumerate(insts):
        _check(e[i], g[b.offsets[i]:b.offsets[i + 1]], inst)
    b.close()


@pytest.mark.parametrize("n,seed", [(14, 1), (14, 4), (15, 2), (15, 5), (16, 3), (16, 6)])
def test_single_state_path_random_circuits(n, seed):
    inst = random_instance(n, seed, n_blocks=8)
    ctx = svqe.Context(n)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    _check(e, g, inst)
    H.close()
    ctx.close()
