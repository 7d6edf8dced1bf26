"""Degenerate inputs of the method, on the single-state path and in the batched kernel, against
the oracle: a circuit with no gates (E = <ref|H|ref>, no gradient), a circuit with fixed
angles only (no parameters), one parameter shared by several gates, a Hamiltonian that is
only the identity (E = c, gradient 0) and one with no terms at all (E = 0), and a batch of a
single instance."""
import numpy as np
import pytest

import oracle
from paper_2601_09951_gb300 import svqe
from paper_2601_09951_gb300 import workloads as W
from tests.parity import assert_energy, assert_grad

pytestmark = pytest.mark.gpu


def _ham(terms):
    return {"x": np.array([t[0] for t in terms], np.uint64),
            "z": np.array([t[1] for t in terms], np.uint64),
            "coeff": np.array([t[2] for t in terms], np.float64)}


def _cases():
    base = W.hea_instance(5, 2, 40, 71)
    cb = W.CircuitBuilder(5)
    empty = dict(base, name="no gates", circuit=cb.build(), theta=np.zeros(0))
    cb = W.CircuitBuilder(5)
    for q in range(5):
        cb.add(W.RY, [q], angle=0.3 + 0.1 * q)
    for q in range(4):
        cb.add(W.CNOT, [q, q + 1])
    cb.add(W.DOUBLE_EXC, [0, 1, 2, 3], angle=-0.7)
    fixed = dict(base, name="fixed angles only", circuit=cb.build(), theta=np.zeros(0))
    cb = W.CircuitBuilder(5)
    p = cb.add(W.RY, [0], param="new")
    cb.add(W.RY, [3], param=p)
    cb.add(W.CNOT, [0, 2])
    cb.add(W.RZ, [2], param=p)
    cb.add(W.SINGLE_EXC, [1, 4], param="new")
    shared = dict(base, name="shared parameter", circuit=cb.build(), theta=np.array([0.9, -0.4]))
    ident = dict(base, name="identity only", ham=_ham([(0, 0, -2.5)]))
    none = dict(base, name="no terms", ham=_ham([]))
    return [empty, fixed, shared, ident, none]


def _check(e, g, inst):
    e0, g0 = oracle.energy_grad(inst)
    g = np.asarray(g)[:len(g0)]
    assert len(g) == len(g0) == inst["circuit"]["n_params"]
    if len(inst["ham"]["coeff"]) == 0:  # no terms: H = 0 exactly
        assert e == 0.0 and e0 == 0.0 and np.all(g == 0.0)
        return
    assert_energy(e, e0, inst["ham"], inst["name"])
    assert_grad(g, g0, inst["ham"], inst["name"])
    if inst["name"] == "identity only":  # E = c <psi|psi>, dE/dtheta = 0
        assert abs(e - (-2.5)) <= 1e-13 and np.all(np.abs(g) <= 1e-13)


@pytest.mark.parametrize("k", range(5))
def test_single_state_path(k):
    inst = _cases()[k]
    ctx = svqe.Context(5)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    e, g = ctx.adjoint_grad(inst["circuit"], inst["theta"], H)
    _check(e, g, inst)
    H.close()
    ctx.close()


def test_batched_kernel_with_every_degenerate_instance():
    insts = _cases() + [W.hea_instance(7, 2, 60, 72)]
    b = svqe.Batch(insts)
    e, g = b.run(b.theta_of(insts))
    for i, inst in enumerate(insts):
        _check(e[i], g[b.offsets[i]:b.offsets[i + 1]], inst)
    b.close()


@pytest.mark.parametrize("k", range(5))
def test_batch_of_one_instance(k):
    inst = _cases()[k]
    b = svqe.Batch([inst])
    e, g = b.run(b.theta_of([inst]))
    _check(e[0], g[b.offsets[0]:b.offsets[1]], inst)
    b.close()
