"""The oracle's stored full-size values (tests/golden/*_oracle.txt, written by
make_fullsize_golden.py from oracle/ only) still belong to the instances the generators make:
each file's SHA-256 fingerprint matches the regenerated instance, and each holds a finite
energy within |E| <= ||c||_1 and the gradient entries the GPU tests compare (CPU only)."""
import os
import sys

import numpy as np
import pytest

from paper_2601_09951_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_fullsize_golden as MG  # noqa: E402

CASES = [("uccsd20_oracle.txt", lambda: W.uccsd_instance(), 400)]
CASES += [(f"hea_single_n{n}_oracle.txt", (lambda n=n: W.hea_single(n)), k)
          for n, k in ((24, 3), (26, 1), (28, 1), (30, 0), (31, 0))]


@pytest.mark.parametrize("fname,make,n_grad", CASES, ids=[c[0] for c in CASES])
def test_stored_values_match_their_instance(fname, make, n_grad):
    path = os.path.join(GOLDEN, fname)
    assert os.path.exists(path), f"{fname} is missing: run make_fullsize_golden.py"
    g = MG.read_golden(path)
    inst = make()
    assert g["sha"] == MG.fingerprint(inst)
    c1 = float(np.abs(inst["ham"]["coeff"]).sum())
    assert g["energy"] is not None and np.isfinite(g["energy"]) and abs(g["energy"]) <= c1
    assert len(g["grad"]) == n_grad
    for p, v in g["grad"].items():
        assert 0 <= p < inst["circuit"]["n_params"] and np.isfinite(v) and abs(v) <= c1
