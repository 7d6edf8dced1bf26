"""ctypes binding of libsvqe.so (the C ABI in include/svqe.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.
There is no CPU fallback; if the library is missing or fails to load, every call raises.
Build it with ``paper_2601_09951_gb300.build.build()`` (or ``__graft_entry__.build()``).
"""
import ctypes
import os

import numpy as np

from . import build as _build

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_ETIMEOUT, SV_EUNSUPPORTED, SV_EBUSY = range(7)
BATCH_MAX_QUBITS = 12

GATE_DTYPE = np.dtype([("type", "<i4"), ("wires", "<i4", (4,)), ("param", "<i4"),
                       ("fixed_angle", "<f8")], align=True)
assert GATE_DTYPE.itemsize == 32


class SvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_STATUS = {0: "SV_OK", 1: "SV_EINVAL", 2: "SV_ENOMEM", 3: "SV_ECUDA", 4: "SV_ETIMEOUT",
           5: "SV_EUNSUPPORTED", 6: "SV_EBUSY"}


class _Circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32),
                ("n_params", ctypes.c_int32), ("gates", ctypes.c_void_p)]


class _PauliSum(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_terms", ctypes.c_int32),
                ("x_mask", ctypes.c_void_p), ("z_mask", ctypes.c_void_p),
                ("coeff", ctypes.c_void_p)]


class _Instance(ctypes.Structure):
    _fields_ = [("circuit", _Circuit), ("ham", _PauliSum), ("ref", ctypes.c_uint64)]


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """The loaded library.  Raises if it has not been built: the product path has no
    fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(paper_2601_09951_gb300.build.build())")
    L = ctypes.CDLL(path)
    P, i32, i64, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_double)
    sigs = {
        "sv_status_str": ([i32], ctypes.c_char_p),
        "sv_last_error": ([], ctypes.c_char_p),
        "sv_abi_version": ([], i32),
        "sv_state_bytes": ([i32], u64),
        "sv_ctx_device_bytes": ([i32], u64),
        "sv_create": ([P, i32, P], i32),
        "sv_destroy": ([P], i32),
        "sv_set_checkpoint_bytes": ([P, u64], i32),
        "sv_set_autotune": ([P, i32], i32),
        "sv_tile_bits": ([P, P], i32),
        "sv_ham_upload": ([P, P, P], i32),
        "sv_ham_free": ([P], i32),
        "sv_ham_info": ([P, P, P], i32),
        "sv_ham_lower": ([P, i32, P, P, P, P, P, P, P], i32),
        "sv_circuit_plan": ([P, i32, P, P], i32),
        "sv_batch_segments": ([P, i32, P, P, P, P], i32),
        "sv_init_reference": ([P, u64], i32),
        "sv_apply_circuit": ([P, P, P], i32),
        "sv_expval_paulisum": ([P, P, P], i32),
        "sv_adjoint_grad": ([P, P, P, P, P, P], i32),
        "sv_adjoint_grad_dev": ([P, P, P, P, P, P], i32),
        "vqe_step": ([P, P, P, P, dbl, i32, P], i32),
        "sv_get_state": ([P, P], i32),
        "sv_set_state": ([P, P], i32),
        "sv_state_device_ptr": ([P, P], i32),
        "sv_batch_create": ([P, i32, P, P], i32),
        "sv_batch_free": ([P], i32),
        "sv_batch_info": ([P, P, P], i32),
        "sv_batch_cost": ([P, P, P], i32),
        "sv_batch_run": ([P, P, P, P], i32),
        "sv_batch_run_dev": ([P, P, P, P], i32),
        "sv_batch_vqe_dev": ([P, P, dbl, i32, P], i32),
        "sv_batch_adam_dev": ([P, P, dbl, i32, P, i32], i32),
        "sv_adjoint_grad_noalloc": ([P, u64, i32, P, i32, P, i64, P, P, P, P], i32),
        "sv_fp64_probe": ([i32, i32, i32, i32, P, P, P], i32),
        "sv_batch_set_autotune": ([i32], i32),
        "sv_batch_layout": ([P, i32, P, P, P], i32),
        "sv_batch_set_layout": ([i32, i32, i32, i32], i32),
        "sv_server_create": ([P, P], i32),
        "sv_server_submit": ([P, P, P, i32, dbl, P], i32),
        "sv_server_wait": ([P, u64, i32, P, P, P], i32),
        "sv_server_cancel": ([P, u64], i32),
        "sv_server_get_stats": ([P, P], i32),
        "sv_server_destroy": ([P], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


_LEGACY_STREAM = 1  # cudaStreamLegacy: torch reports its default stream as handle 0


def _stream_arg(stream):
    """None: the library creates its own stream; an int handle (0 = torch's default stream,
    passed on as cudaStreamLegacy) otherwise."""
    if stream is None:
        return None
    return ctypes.c_void_p(int(stream) if int(stream) != 0 else _LEGACY_STREAM)


def _check(status):
    if status != SV_OK:
        msg = lib().sv_last_error()
        raise SvError(status, msg.decode() if msg else "")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def state_bytes(n):
    return int(lib().sv_state_bytes(int(n)))


def ctx_device_bytes(n):
    return int(lib().sv_ctx_device_bytes(int(n)))


class Circuit:
    """Gate records of a circuit dict (see workloads) in the ABI layout."""

    def __init__(self, circuit):
        c = circuit
        G = len(c["types"])
        self.gates = np.zeros(G, dtype=GATE_DTYPE)
        self.gates["type"] = np.asarray(c["types"], dtype=np.int32)
        self.gates["wires"] = np.asarray(c["wires"], dtype=np.int32).reshape(G, 4)
        self.gates["param"] = np.asarray(c["params"], dtype=np.int32)
        self.gates["fixed_angle"] = np.asarray(c["fixed"], dtype=np.float64)
        self.n = int(c["n"])
        self.n_params = int(c["n_params"])
        self.struct = _Circuit(self.n, G, self.n_params,
                               self.gates.ctypes.data if G else None)

    def ref(self):
        return ctypes.byref(self.struct)


class PauliSum:
    def __init__(self, ham, n):
        self.x = np.ascontiguousarray(ham["x"], dtype=np.uint64)
        self.z = np.ascontiguousarray(ham["z"], dtype=np.uint64)
        self.c = np.ascontiguousarray(ham["coeff"], dtype=np.float64)
        self.n = int(n)
        self.struct = _PauliSum(self.n, len(self.c), self.x.ctypes.data, self.z.ctypes.data,
                                self.c.ctypes.data)

    def ref(self):
        return ctypes.byref(self.struct)


def ham_lower(ham, n, kmax):
    """Host-only view of the X-mask grouping: (x, zu, cls, toff, table[complex])."""
    ps = PauliSum(ham, n)
    ng, nt = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(lib().sv_ham_lower(ps.ref(), int(kmax), ctypes.byref(ng), ctypes.byref(nt),
                              None, None, None, None, None))
    x = np.zeros(ng.value, np.uint64)
    zu = np.zeros(ng.value, np.uint64)
    cls = np.zeros(ng.value, np.int32)
    toff = np.zeros(ng.value, np.int64)
    table = np.zeros(max(nt.value, 1), np.complex128)
    _check(lib().sv_ham_lower(ps.ref(), int(kmax), ctypes.byref(ng), ctypes.byref(nt),
                              _ptr(x), _ptr(zu), _ptr(cls), _ptr(toff), _ptr(table)))
    return x, zu, cls, toff, table[:nt.value]


def circuit_plan(circuit, tile_bits=0):
    """Host-only fused-pass plan: (number of passes, pass index of every gate)."""
    C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
    npass = ctypes.c_int32()
    pog = np.zeros(max(len(C.gates), 1), np.int32)
    _check(lib().sv_circuit_plan(C.ref(), int(tile_bits), ctypes.byref(npass), _ptr(pog)))
    return npass.value, pog[:len(C.gates)]


def batch_segments(circuit):
    """Host-only segmentation of a circuit for the batched kernel: (segments as an (S, 5) int32
    array of kind, split, first gate, gate count, checkpoint slot; checkpoint slots; checkpoint
    scratch of one instance in amplitudes)."""
    C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
    ns, nc = ctypes.c_int32(), ctypes.c_int32()
    amps = ctypes.c_int64()
    _check(lib().sv_batch_segments(C.ref(), 0, None, ctypes.byref(ns), ctypes.byref(nc),
                                   ctypes.byref(amps)))
    segs = np.zeros((max(ns.value, 1), 5), np.int32)
    _check(lib().sv_batch_segments(C.ref(), ns.value, _ptr(segs), ctypes.byref(ns),
                                   ctypes.byref(nc), None))
    return segs[:ns.value], nc.value, amps.value


GROUP_DTYPE = np.dtype([("x_mask", "<u8"), ("z_union", "<u8"), ("z_bits", "<i4"),
                        ("cls", "<i4"), ("table_offset", "<i8")])
assert GROUP_DTYPE.itemsize == 32
NOALLOC_MAX_QUBITS = 14
NOALLOC_MAX_GATES = 256


def group_records(ham, n, kmax=14):
    """(sv_group records, complex128 tables) of a Hamiltonian, from the host-only lowering,
    for callers that place them in device memory of their own."""
    x, zu, cls, toff, table = ham_lower(ham, n, kmax)
    rec = np.zeros(len(x), dtype=GROUP_DTYPE)
    rec["x_mask"], rec["z_union"], rec["cls"], rec["table_offset"] = x, zu, cls, toff
    rec["z_bits"] = [bin(int(v)).count("1") for v in zu]
    return rec, np.ascontiguousarray(table, dtype=np.complex128)


def adjoint_grad_noalloc(circuit, ref, ham_n_qubits, groups_ptr, n_groups, tables_ptr,
                         n_table, theta_ptr, energy_ptr, grad_ptr, stream):
    """sv_adjoint_grad_noalloc: every pointer is a device address the caller owns; the
    library allocates no device memory.  `stream` is the integer handle of the CUDA stream the
    inputs were written on (for torch: torch.cuda.current_stream().cuda_stream); unlike the
    context calls there is no library-owned stream here, and 0 means torch's default stream.
    Stream-ordered (synchronise before reading)."""
    C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
    _check(lib().sv_adjoint_grad_noalloc(
        C.ref(), int(ref), int(ham_n_qubits), ctypes.c_void_p(groups_ptr), int(n_groups),
        ctypes.c_void_p(tables_ptr), int(n_table), ctypes.c_void_p(theta_ptr),
        ctypes.c_void_p(energy_ptr), ctypes.c_void_p(grad_ptr), _stream_arg(int(stream))))


def batch_set_autotune(enable):
    """sv_batch_set_autotune: process-wide switch of the batched kernel's layout tuner."""
    _check(lib().sv_batch_set_autotune(1 if enable else 0))


def batch_set_layout(n_qubits, team_warps, min_layer, min_diag_rz):
    """sv_batch_set_layout: pin (or with team_warps = 0 forget) the tuner's layout for one
    qubit count."""
    _check(lib().sv_batch_set_layout(int(n_qubits), int(team_warps), int(min_layer),
                                     int(min_diag_rz)))


SEG_OFF = 1 << 20  # a segment width no run reaches: that segment kind is not used


def fp64_probe(blocks, threads, chains, iters, out_ptr, stream):
    """sv_fp64_probe: enqueue the FP64 FMA-rate probe on `stream` (integer handle, 0 = torch's
    default stream); returns the number of FMAs the launch executes."""
    d = ctypes.c_double()
    _check(lib().sv_fp64_probe(int(blocks), int(threads), int(chains), int(iters),
                               ctypes.c_void_p(out_ptr), _stream_arg(int(stream)),
                               ctypes.byref(d)))
    return d.value


class Ham:
    """A device-resident grouped Pauli sum (sv_ham)."""

    def __init__(self, ctx, ham):
        self._h = ctypes.c_void_p()
        ps = PauliSum(ham, ctx.n)
        _check(lib().sv_ham_upload(ctx.handle, ps.ref(), ctypes.byref(self._h)))
        self.n = ctx.n

    @property
    def handle(self):
        return self._h

    def info(self):
        g, b = ctypes.c_int32(), ctypes.c_uint64()
        _check(lib().sv_ham_info(self._h, ctypes.byref(g), ctypes.byref(b)))
        return g.value, b.value

    def close(self):
        if self._h:
            lib().sv_ham_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One n-qubit state (sv_ctx): psi and lambda buffers on the device plus a stream."""

    def __init__(self, n, stream=None):
        self._c = ctypes.c_void_p()
        self.n = int(n)
        _check(lib().sv_create(ctypes.byref(self._c), self.n, _stream_arg(stream)))

    @property
    def handle(self):
        return self._c

    def init_reference(self, b):
        _check(lib().sv_init_reference(self._c, int(b)))

    def apply_circuit(self, circuit, theta):
        C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        _check(lib().sv_apply_circuit(self._c, C.ref(), _ptr(th) if th.size else None))

    def expval(self, ham):
        e = ctypes.c_double()
        _check(lib().sv_expval_paulisum(self._c, ham.handle, ctypes.byref(e)))
        return e.value

    def adjoint_grad(self, circuit, theta, ham):
        C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        g = np.zeros(max(C.n_params, 1), dtype=np.float64)
        e = ctypes.c_double()
        _check(lib().sv_adjoint_grad(self._c, C.ref(), _ptr(th) if th.size else None,
                                     ham.handle, ctypes.byref(e), _ptr(g)))
        return e.value, g[:C.n_params]

    def adjoint_grad_dev(self, circuit, theta_ptr, ham, energy_ptr, grad_ptr):
        C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
        _check(lib().sv_adjoint_grad_dev(self._c, C.ref(), ctypes.c_void_p(theta_ptr),
                                         ham.handle, ctypes.c_void_p(energy_ptr),
                                         ctypes.c_void_p(grad_ptr)))

    def vqe_step(self, circuit, ham, theta, lr, n_steps):
        C = circuit if isinstance(circuit, Circuit) else Circuit(circuit)
        th = np.array(theta, dtype=np.float64, copy=True)
        es = np.zeros(max(n_steps, 1), dtype=np.float64)
        _check(lib().vqe_step(self._c, C.ref(), ham.handle, _ptr(th) if th.size else None,
                              float(lr), int(n_steps), _ptr(es)))
        return th, es[:n_steps]

    def get_state(self):
        out = np.empty(1 << self.n, dtype=np.complex128)
        _check(lib().sv_get_state(self._c, _ptr(out)))
        return out

    def set_checkpoint_bytes(self, nbytes):
        """Device memory for psi checkpoints of commuting layers (sv_set_checkpoint_bytes)."""
        _check(lib().sv_set_checkpoint_bytes(self._c, int(nbytes)))

    def set_autotune(self, enable=True):
        """Autotune the fused-pass tile size per circuit structure (sv_set_autotune)."""
        _check(lib().sv_set_autotune(self._c, 1 if enable else 0))

    def tile_bits(self):
        """Tile size (bits) of the last staged circuit's fused passes."""
        t = ctypes.c_int32()
        _check(lib().sv_tile_bits(self._c, ctypes.byref(t)))
        return t.value

    def set_state(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        if a.size != 1 << self.n:
            raise ValueError("state has the wrong size")
        _check(lib().sv_set_state(self._c, _ptr(a)))

    def state_ptr(self):
        p = ctypes.c_void_p()
        _check(lib().sv_state_device_ptr(self._c, ctypes.byref(p)))
        return p.value

    def close(self):
        if self._c:
            lib().sv_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many small instances (n <= 12) compiled for the persistent batched kernel."""

    def __init__(self, instances, stream=None):
        self._b = ctypes.c_void_p()
        self._keep = []
        arr = (_Instance * len(instances))()
        offs = [0]
        for i, inst in enumerate(instances):
            C = Circuit(inst["circuit"])
            H = PauliSum(inst["ham"], C.n)
            self._keep += [C, H]
            arr[i].circuit = C.struct
            arr[i].ham = H.struct
            arr[i].ref = int(inst["ref"])
            offs.append(offs[-1] + C.n_params)
        self.offsets = np.array(offs, dtype=np.int64)
        _check(lib().sv_batch_create(arr, len(instances), _stream_arg(stream),
                                     ctypes.byref(self._b)))
        self._keep = None
        ni, npar = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().sv_batch_info(self._b, ctypes.byref(ni), ctypes.byref(npar)))
        self.n_instances, self.n_params = ni.value, npar.value

    def layout(self, n_qubits):
        """(warps per instance team, min commuting-layer width, min diagonal RZ count) the batch
        was compiled with for n_qubits-qubit instances (zeros if it holds none)."""
        w, ml, md = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sv_batch_layout(self._b, int(n_qubits), ctypes.byref(w), ctypes.byref(ml),
                                     ctypes.byref(md)))
        return w.value, ml.value, md.value

    def cost(self):
        """(FP64 flops, HBM bytes) of one run, from the compiled segments."""
        f, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().sv_batch_cost(self._b, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def theta_of(self, instances):
        return np.concatenate([np.asarray(i["theta"], np.float64) for i in instances]) \
            if self.n_params else np.zeros(0)

    def run(self, theta, energy_out=None, grad_out=None):
        """Host buffers in and out (copies included).  Returns (energy[n], grad[P])."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        e = energy_out if energy_out is not None else np.empty(self.n_instances, np.float64)
        g = grad_out if grad_out is not None else np.empty(max(self.n_params, 1), np.float64)
        _check(lib().sv_batch_run(self._b, _ptr(th), _ptr(e), _ptr(g)))
        return e, g[:self.n_params]

    def run_ptr(self, theta_ptr, energy_ptr, grad_ptr, energy_host_ptr=None):
        """Host pointers (e.g. pinned tensors): the same call as run(), without numpy."""
        _check(lib().sv_batch_run(self._b, ctypes.c_void_p(theta_ptr),
                                  ctypes.c_void_p(energy_ptr), ctypes.c_void_p(grad_ptr)))

    def run_dev(self, theta_ptr, energy_ptr, grad_ptr):
        _check(lib().sv_batch_run_dev(self._b, ctypes.c_void_p(theta_ptr),
                                      ctypes.c_void_p(energy_ptr), ctypes.c_void_p(grad_ptr)))

    def vqe_dev(self, theta_ptr, lr, n_steps, etraj_ptr=None):
        _check(lib().sv_batch_vqe_dev(self._b, ctypes.c_void_p(theta_ptr), float(lr),
                                      int(n_steps),
                                      ctypes.c_void_p(etraj_ptr) if etraj_ptr else None))

    def adam_dev(self, theta_ptr, lr, n_steps, etraj_ptr=None, reset=True):
        _check(lib().sv_batch_adam_dev(self._b, ctypes.c_void_p(theta_ptr), float(lr),
                                       int(n_steps),
                                       ctypes.c_void_p(etraj_ptr) if etraj_ptr else None,
                                       1 if reset else 0))

    def close(self):
        if self._b:
            lib().sv_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_active_small", ctypes.c_int32),
                ("steps_per_tick", ctypes.c_int32), ("max_active_large", ctypes.c_int32),
                ("serial", ctypes.c_int32), ("max_active_heavy", ctypes.c_int32),
                ("heavy_qubits", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("n_qubits", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("n_steps", ctypes.c_int32), ("footprint_bytes", ctypes.c_uint64),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64),
                ("peak_bytes_in_use", ctypes.c_uint64), ("queued", ctypes.c_int32),
                ("running", ctypes.c_int32)]


class Server:
    """The continuous-batching request loop (sv_server_*)."""

    def __init__(self, hbm_budget_bytes=0, max_active_small=0, steps_per_tick=0,
                 max_active_large=0, serial=False, max_active_heavy=0, heavy_qubits=0):
        self._s = ctypes.c_void_p()
        cfg = _ServerConfig(int(hbm_budget_bytes), int(max_active_small), int(steps_per_tick),
                            int(max_active_large), 1 if serial else 0, int(max_active_heavy),
                            int(heavy_qubits))
        _check(lib().sv_server_create(ctypes.byref(cfg), ctypes.byref(self._s)))
        self._meta = {}

    def submit(self, inst, n_steps, lr, theta0=None):
        C = Circuit(inst["circuit"])
        H = PauliSum(inst["ham"], C.n)
        one = _Instance()
        one.circuit = C.struct
        one.ham = H.struct
        one.ref = int(inst["ref"])
        th = np.ascontiguousarray(inst["theta"] if theta0 is None else theta0, dtype=np.float64)
        rid = ctypes.c_uint64()
        _check(lib().sv_server_submit(self._s, ctypes.byref(one), _ptr(th) if th.size else None,
                                      int(n_steps), float(lr), ctypes.byref(rid)))
        self._meta[rid.value] = (C.n_params, int(n_steps))
        return rid.value

    def wait(self, rid, timeout_ms=-1):
        """(theta_final, energies[n_steps], RequestInfo); raises SvError on failure/timeout."""
        P, T = self._meta[rid]
        th = np.zeros(max(P, 1))
        es = np.zeros(max(T, 1))
        info = RequestInfo()
        _check(lib().sv_server_wait(self._s, int(rid), int(timeout_ms), _ptr(th), _ptr(es),
                                    ctypes.byref(info)))
        del self._meta[rid]
        return th[:P], es[:T], info

    def cancel(self, rid):
        _check(lib().sv_server_cancel(self._s, int(rid)))

    def stats(self):
        st = ServerStats()
        _check(lib().sv_server_get_stats(self._s, ctypes.byref(st)))
        return st

    def close(self):
        if self._s:
            lib().sv_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
