"""Plain CPU oracle for the VQE hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import this package.  The product path (the CUDA library and its binding) never does, and
this package imports nothing from it.  The arithmetic lives in ``svqe_oracle.c`` (plain C,
IEEE binary64, gate by gate and term by term); this module only marshals numpy arrays.

What it computes (paper sections): the state |psi(theta)> = U(theta)|HF> (Sec. 3.3, Eq. 4-5),
the energy E = <psi|H|psi> (Sec. 3.1, Eq. 2) of a Pauli-sum H (Sec. 3.2, Eq. 3), and the
parameter-shift gradient used in Algorithm 1 (Sec. 4.3).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i32, u64, dbl = ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        P = ctypes.c_void_p
        L.orc_apply_gate.argtypes = [i32, P, i32, P, dbl]
        L.orc_apply_gate.restype = i32
        L.orc_init_basis.argtypes = [i32, P, u64]
        L.orc_init_basis.restype = None
        L.orc_apply_circuit.argtypes = [i32, P, i32, P, P, P, P, P, i32, dbl]
        L.orc_apply_circuit.restype = i32
        L.orc_expval.argtypes = [i32, P, i32, P, P, P, P, P]
        L.orc_expval.restype = None
        L.orc_energy.argtypes = [i32, u64, i32, P, P, P, P, P, i32, P, P, P, P]
        L.orc_energy.restype = i32
        L.orc_energy_grad.argtypes = [i32, u64, i32, P, P, P, P, P, i32, i32, P, P, P, P, P]
        L.orc_energy_grad.restype = i32
        L.orc_energy_grad_subset.argtypes = [i32, u64, i32, P, P, P, P, P, i32, i32, P, P, P,
                                             P, i32, P, P]
        L.orc_energy_grad_subset.restype = i32
        L.orc_state.argtypes = [i32, u64, i32, P, P, P, P, P, P]
        L.orc_state.restype = i32
        L.orc_set_threads.argtypes = [i32]
        L.orc_set_threads.restype = None
        L.orc_get_threads.argtypes = []
        L.orc_get_threads.restype = i32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _circ(circuit):
    """Contiguous copies of a circuit's gate arrays, in the oracle's own argument order."""
    types = np.ascontiguousarray(circuit["types"], dtype=np.int32)
    wires = np.ascontiguousarray(circuit["wires"], dtype=np.int32).reshape(-1, 4)
    params = np.ascontiguousarray(circuit["params"], dtype=np.int32)
    fixed = np.ascontiguousarray(circuit["fixed"], dtype=np.float64)
    return types, wires, params, fixed


def _ham(ham):
    return (np.ascontiguousarray(ham["x"], dtype=np.uint64),
            np.ascontiguousarray(ham["z"], dtype=np.uint64),
            np.ascontiguousarray(ham["coeff"], dtype=np.float64))


def set_threads(k: int) -> None:
    """Number of OpenMP threads the parameter-shift gradient may use."""
    lib().orc_set_threads(int(k))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def apply_gate(psi, n, gtype, wires, angle=0.0):
    """Apply one gate to a copy of ``psi`` (complex128, 2^n) and return it."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    w = np.full(4, -1, dtype=np.int32)
    w[:len(wires)] = wires
    rc = lib().orc_apply_gate(int(n), _p(out), int(gtype), _p(w), float(angle))
    if rc != 0:
        raise ValueError("malformed gate")
    return out


def apply_circuit(psi, circuit, theta):
    """Apply a whole circuit (gates in list order) to a copy of ``psi``."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    types, wires, params, fixed = _circ(circuit)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    rc = lib().orc_apply_circuit(int(circuit["n"]), _p(out), len(types), _p(types), _p(wires),
                                 _p(params), _p(fixed), _p(th) if th.size else None, -1, 0.0)
    if rc != 0:
        raise ValueError("malformed circuit")
    return out


def basis_state(n, b):
    out = np.empty(1 << n, dtype=np.complex128)
    lib().orc_init_basis(int(n), _p(out), int(b))
    return out


def state(circuit, theta, ref):
    """U(theta)|ref> as a complex128 vector of 2^n amplitudes."""
    n = int(circuit["n"])
    out = np.empty(1 << n, dtype=np.complex128)
    types, wires, params, fixed = _circ(circuit)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    rc = lib().orc_state(n, int(ref), len(types), _p(types), _p(wires), _p(params), _p(fixed),
                         _p(th) if th.size else None, _p(out))
    if rc != 0:
        raise ValueError("malformed circuit")
    return out


def expval(psi, n, ham):
    """(Re, Im) of sum_t c_t <psi|P_t|psi>."""
    x, z, c = _ham(ham)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_expval(int(n), _p(psi), len(c), _p(x), _p(z), _p(c), ctypes.byref(re),
                     ctypes.byref(im))
    return re.value, im.value


def energy(inst, theta=None):
    """E(theta) for an instance dict (circuit, ham, ref)."""
    circ, ham = inst["circuit"], inst["ham"]
    theta = inst["theta"] if theta is None else theta
    types, wires, params, fixed = _circ(circ)
    x, z, c = _ham(ham)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    e = ctypes.c_double()
    rc = lib().orc_energy(int(circ["n"]), int(inst["ref"]), len(types), _p(types), _p(wires),
                          _p(params), _p(fixed), _p(th) if th.size else None, len(c), _p(x),
                          _p(z), _p(c), ctypes.byref(e))
    if rc != 0:
        raise ValueError(f"oracle energy failed ({rc})")
    return e.value


def energy_grad(inst, theta=None):
    """(E, dE/dtheta) by the parameter-shift rule."""
    circ, ham = inst["circuit"], inst["ham"]
    theta = inst["theta"] if theta is None else theta
    types, wires, params, fixed = _circ(circ)
    x, z, c = _ham(ham)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    n_params = int(circ["n_params"])
    g = np.zeros(max(n_params, 1), dtype=np.float64)
    e = ctypes.c_double()
    rc = lib().orc_energy_grad(int(circ["n"]), int(inst["ref"]), len(types), _p(types),
                               _p(wires), _p(params), _p(fixed), _p(th) if th.size else None,
                               n_params, len(c), _p(x), _p(z), _p(c), ctypes.byref(e), _p(g))
    if rc != 0:
        raise ValueError(f"oracle gradient failed ({rc})")
    return e.value, g[:n_params]


def energy_grad_subset(inst, which, theta=None):
    """(E, {p: dE/dtheta_p}) for the parameters in `which` only (same shift rules)."""
    circ, ham = inst["circuit"], inst["ham"]
    theta = inst["theta"] if theta is None else theta
    types, wires, params, fixed = _circ(circ)
    x, z, c = _ham(ham)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    n_params = int(circ["n_params"])
    w = np.ascontiguousarray(list(which), dtype=np.int32)
    g = np.zeros(max(n_params, 1), dtype=np.float64)
    e = ctypes.c_double()
    rc = lib().orc_energy_grad_subset(int(circ["n"]), int(inst["ref"]), len(types), _p(types),
                                      _p(wires), _p(params), _p(fixed),
                                      _p(th) if th.size else None, n_params, len(c), _p(x),
                                      _p(z), _p(c), _p(w), len(w), ctypes.byref(e), _p(g))
    if rc != 0:
        raise ValueError(f"oracle gradient failed ({rc})")
    return e.value, {int(p): float(g[p]) for p in w}


def gd_trajectory(inst, lr, n_steps, theta0=None):
    """Plain gradient descent theta <- theta - lr * g (the update of the bond-length loop in
    Algorithm 1, with a fixed step instead of Adam).  Returns (E_t, g_t, theta_t) before each
    update and the final theta."""
    theta = np.array(inst["theta"] if theta0 is None else theta0, dtype=np.float64)
    es, gs, ths = [], [], []
    for _ in range(n_steps):
        e, g = energy_grad(inst, theta)
        es.append(e)
        gs.append(g.copy())
        ths.append(theta.copy())
        theta = theta - lr * g
    return np.array(es), np.array(gs), np.array(ths), theta


def adam_trajectory(inst, lr, n_steps, theta0=None, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam, the optimizer of the paper's loop (Sec. 3.4; Algorithm 1's update), on the
    parameter-shift gradient: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), t = 1, 2, ...
    Returns (E_t, theta_t) before each update and the final theta."""
    theta = np.array(inst["theta"] if theta0 is None else theta0, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    es, ths = [], []
    for t in range(1, n_steps + 1):
        e, g = energy_grad(inst, theta)
        es.append(e)
        ths.append(theta.copy())
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        theta = theta - lr * mh / (np.sqrt(vh) + eps)
    return np.array(es), np.array(ths), theta
