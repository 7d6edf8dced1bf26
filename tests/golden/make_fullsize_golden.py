"""Write the oracle's values for the full-size single-state workloads to tests/golden/.

Calls only ``oracle/`` (plain C, parameter shift) and the seeded input generators; nothing here
touches the CUDA library.  The GPU parity tests compare against these files because the oracle
needs minutes to hours per value at these sizes (one energy of the 20-qubit UCCSD-shaped
circuit is about 13 s on one core; one of the 31-qubit hardware-efficient circuit is about two
hours), far more than a GPU test run should spend on the host.

Each file records a SHA-256 fingerprint of the instance arrays it was computed on; the tests
regenerate the instance and refuse to compare when the fingerprint differs.

    python tests/golden/make_fullsize_golden.py uccsd20 --threads 4
    python tests/golden/make_fullsize_golden.py hea 24 --params 0,250,479 --threads 3
    python tests/golden/make_fullsize_golden.py hea 31

Targets:
  uccsd20   the 20-qubit UCCSD-shaped circuit (400 Givens gates, 2000 terms): the energy and
            all 400 parameter-shift gradient entries (four-term rule, 1,601 evaluations).
  hea N     the 10-layer hardware-efficient circuit on N qubits with 100 random strings: the
            energy and the listed gradient entries (two-term rule).
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2601_09951_gb300 import workloads as W  # noqa: E402


def fingerprint(inst):
    """SHA-256 over the arrays that define the instance (gates, Hamiltonian, reference, theta)."""
    h = hashlib.sha256()
    c, ham = inst["circuit"], inst["ham"]
    for a in (np.asarray(c["types"], np.int32), np.asarray(c["wires"], np.int32),
              np.asarray(c["params"], np.int32), np.asarray(c["fixed"], np.float64),
              np.asarray(ham["x"], np.uint64), np.asarray(ham["z"], np.uint64),
              np.asarray(ham["coeff"], np.float64), np.asarray(inst["theta"], np.float64),
              np.asarray([c["n"], c["n_params"], inst["ref"]], np.int64)):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def read_golden(path):
    """{"sha": str, "energy": float, "grad": {p: float}} from a file this script wrote."""
    out = {"sha": None, "energy": None, "grad": {}}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            if k == "sha256":
                out["sha"] = v[0]
            elif k == "E":
                out["energy"] = float(v[0])
            elif k == "g":
                out["grad"][int(v[0])] = float(v[1])
    return out


def write_golden(path, inst, what, e, grad, seconds, threads):
    with open(path + ".tmp", "w") as f:
        f.write(f"# {what}\n")
        f.write("# Written by tests/golden/make_fullsize_golden.py from oracle/ only: energy\n")
        f.write("# <psi|H|psi> (Sec. 3.1, Eq. 2) of U(theta)|ref> (Sec. 3.3, Eq. 4) and\n")
        f.write("# parameter-shift gradient entries (Algorithm 1's gradient step, Sec. 4.3).\n")
        f.write(f"# instance {inst['name']}: {len(inst['circuit']['types'])} gates, "
                f"{inst['circuit']['n_params']} parameters, {len(inst['ham']['coeff'])} terms\n")
        f.write(f"# oracle time {seconds:.0f} s on {threads} host thread(s)\n")
        f.write(f"sha256 {fingerprint(inst)}\n")
        f.write(f"E {e!r}\n")
        for p in sorted(grad):
            f.write(f"g {p} {grad[p]!r}\n")
    os.replace(path + ".tmp", path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("target", choices=["uccsd20", "hea"])
    ap.add_argument("n", nargs="?", type=int)
    ap.add_argument("--params", default="")
    ap.add_argument("--threads", type=int, default=1)
    a = ap.parse_args()
    oracle.set_threads(a.threads)
    t0 = time.time()
    if a.target == "uccsd20":
        inst = W.uccsd_instance()
        e, g = oracle.energy_grad(inst)
        grad = {p: float(g[p]) for p in range(len(g))}
        path = os.path.join(HERE, "uccsd20_oracle.txt")
        what = ("20-qubit UCCSD-shaped circuit (HF with 10 electrons, 400 Givens gates, "
                "2000 terms): energy and all 400 gradient entries")
    else:
        inst = W.hea_single(a.n)
        which = [int(p) for p in a.params.split(",") if p]
        if which:
            e, gd = oracle.energy_grad_subset(inst, which)
        else:
            e, gd = oracle.energy(inst), {}
        grad = {int(p): float(v) for p, v in gd.items()}
        path = os.path.join(HERE, f"hea_single_n{a.n}_oracle.txt")
        what = (f"{a.n}-qubit hardware-efficient circuit, 10 layers of RY, RZ and a CNOT ring, "
                f"100 random strings of weight <= 6: energy and {len(grad)} gradient entries")
    write_golden(path, inst, what, float(e), grad, time.time() - t0, a.threads)
    print(path, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
