"""Tolerances of the parity tests (floating point, complex128 arithmetic).

Energies:   |dE| <= 1e-10 * max(|E|, ||c||_1)
Gradients:  |dg| <= 1e-9  * max(|g|, ||c||_1)
States:     max |d psi_k| <= 1e-12 for unit-norm states (a few ulps per gate over hundreds of
            gates, far below the energy tolerance).
|E| <= ||c||_1 and |dE/dtheta| <= ||c||_1 for these generators, so the bounds are relative to
the largest value the quantity can take.
"""
import numpy as np

E_TOL = 1e-10
G_TOL = 1e-9
PSI_TOL = 1e-12


def l1(ham):
    return float(np.abs(np.asarray(ham["coeff"])).sum())


def assert_energy(got, want, ham, what=""):
    bound = E_TOL * max(abs(want), l1(ham), 1e-300)
    assert abs(got - want) <= bound, f"{what} energy {got!r} vs {want!r} (bound {bound:.3g})"


def assert_grad(got, want, ham, what=""):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (got.shape, want.shape)
    bound = G_TOL * np.maximum(np.abs(want), max(l1(ham), 1e-300))
    bad = np.abs(got - want) > bound
    assert not bad.any(), (f"{what} gradient mismatch at {np.flatnonzero(bad)[:8]}: "
                           f"{got[bad][:4]} vs {want[bad][:4]}")
