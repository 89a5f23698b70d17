"""Python binding of the C ABI in include/qsim.h (argument marshalling only).

Every step of the evolution, every observable and every reduction runs in the
CUDA kernels of libqsim.so; this module only converts arguments, owns the
borrowed state tensors (allocated by PyTorch on the GPU) and raises on error.
There is no CPU path: if the library cannot be loaded or built, import fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from . import build as _build

QS_OK = 0
STATUS = {0: "QS_OK", 1: "QS_ERR_ARG", 2: "QS_ERR_OOM", 3: "QS_ERR_CUDA", 4: "QS_ERR_NONFINITE",
          5: "QS_ERR_TIMEOUT", 6: "QS_ERR_STATE"}
QS_PERIODIC, QS_OPEN = 0, 1
QS_GAUGE_HIGGS, QS_UNITARY_GAUGE = 0, 1
QS_C64, QS_C128 = 0, 1
QS_NOALLOC_MAX_BATCH = 16     # include/qsim.h
QS_NORM, QS_PLAQUETTE, QS_WILSON, QS_X, QS_ENERGY, QS_ENERGY_S, QS_GAUSS, QS_THOOFT = range(8)
QS_OPT_METHOD, QS_OPT_RENORM_EVERY, QS_OPT_PROFILE, QS_OPT_GRAPH, QS_OPT_XPASS, QS_OPT_TMA_BUFFERS, QS_OPT_ADJOINT, \
    QS_OPT_TMA_STORE, QS_OPT_XMERGE, QS_OPT_PDL, QS_OPT_SHARED_BUFFERS, QS_OPT_PLAN, QS_OPT_SCAN_BUFFERS, \
    QS_OPT_SHARED_KERNEL, QS_OPT_C128_DF = range(15)


class QsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class qs_couplings(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("h", ctypes.c_double), ("g", ctypes.c_double),
                ("lambda_", ctypes.c_double)]


_LIB = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_LL = ctypes.c_longlong
_U64 = ctypes.c_uint64
_CP = ctypes.POINTER(qs_couplings)
_DP = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "qs_create": ([_I, _I, _I, _I, _I, _I, ctypes.POINTER(_P)], _I),
    "qs_destroy": ([_P], None),
    "qs_last_error": ([_P], ctypes.c_char_p),
    "qs_num_qubits": ([_P], _I),
    "qs_state_bytes": ([_P], _SZ),
    "qs_bind_state": ([_P, _I, _P, _SZ], _I),
    "qs_set_stream": ([_P, _P], _I),
    "qs_set_option": ([_P, _I, _LL], _I),
    "qs_init_plus": ([_P], _I),
    "qs_init_toric": ([_P, _I], _I),
    "qs_evolve_path": ([_P, _CP, _D, _I, _I], _I),
    "qs_upload_state": ([_P, _P, _SZ], _I),
    "qs_download_state": ([_P, _P, _SZ], _I),
    "qs_trotter_step": ([_P, _CP, _D, _D, _I], _I),
    "qs_evolve": ([_P, _CP, _DP, _D, _I, _I], _I),
    "qs_expect": ([_P, _I, _I, _CP, _D, _DP], _I),
    "qs_expect_pauli": ([_P, _I, _U64, _DP], _I),
    "qs_fidelity": ([_P, _P, _DP], _I),
    "qs_sync": ([_P], _I),
    "qs_selftest_wait": ([_P, _D], _I),
    "qs_num_links": ([_P], _I),
    "qs_dos": ([_P, _DP], _I),
    "qs_autotune": ([_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                     ctypes.POINTER(_I), _DP], _I),
    "qs_save": ([_P, ctypes.c_char_p], _I),
    "qs_load": ([_P, ctypes.c_char_p], _I),
    "qs_scan": ([_P, _CP, _I, _DP, _D, _I, _I, _DP], _I),
    "qs_adjoint_grad": ([_P, _CP, _DP, _D, _I, _I, _I, _P, _DP, _DP], _I),
    "qs_profile_read": ([_P, _DP, ctypes.POINTER(_LL)], _I),
    "qs_profile_read_kinds": ([_P, _DP, ctypes.POINTER(_LL)], _I),
    "qs_launch_count": ([_P], _LL),
    "qs_expect_z_noalloc": ([_P, _I, _I, _I, _U64, _P, _P], _I),
    "qs_autotune_plan": ([_P, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _DP], _I),
    "qs_plan": ([_P, ctypes.POINTER(_I), _I], _I),
    "qs_scan_mixed": ([_P, _CP, _I, _P, _CP, _I, _DP, _D, _I, _I, _DP, _DP], _I),
}


def library() -> ctypes.CDLL:
    """Load libqsim.so (building it with nvcc first if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _LIB = lib
    return _LIB


def library_path() -> str:
    return _build.LIB


def _check(sim, status: int):
    if status != QS_OK:
        msg = library().qs_last_error(sim)
        raise QsError(status, msg.decode() if msg else "")


def _couplings(cs, batch: int):
    arr = (qs_couplings * batch)()
    if isinstance(cs, (tuple, list)) and len(cs) and not isinstance(cs[0], (tuple, list, dict, qs_couplings)):
        cs = [cs]
    cs = list(cs)
    if len(cs) == 1 and batch > 1:
        cs = cs * batch
    if len(cs) != batch:
        raise ValueError(f"need {batch} coupling records, got {len(cs)}")
    for i, c in enumerate(cs):
        if isinstance(c, qs_couplings):
            arr[i] = c
        elif isinstance(c, dict):
            arr[i] = qs_couplings(c.get("J", 1.0), c.get("h", 1.0), c["g"], c["lambda"])
        else:   # (g, lambda[, J, h])
            g, lam = c[0], c[1]
            J = c[2] if len(c) > 2 else 1.0
            h = c[3] if len(c) > 3 else 1.0
            arr[i] = qs_couplings(J, h, g, lam)
    return arr


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------
def qs_create(Lx, Ly, boundary=QS_PERIODIC, form=QS_GAUGE_HIGGS, dtype=QS_C64, batch=1):
    h = _P()
    st = library().qs_create(Lx, Ly, boundary, form, dtype, batch, ctypes.byref(h))
    _check(None, st)
    return h


def qs_destroy(sim):
    library().qs_destroy(sim)


def qs_last_error(sim=None) -> str:
    msg = library().qs_last_error(sim)
    return msg.decode() if msg else ""


def qs_num_qubits(sim) -> int:
    return library().qs_num_qubits(sim)


def qs_state_bytes(sim) -> int:
    return library().qs_state_bytes(sim)


def qs_bind_state(sim, slot: int, dev_ptr: int, nbytes: int):
    _check(sim, library().qs_bind_state(sim, slot, dev_ptr, nbytes))


def qs_set_stream(sim, stream_handle: int):
    _check(sim, library().qs_set_stream(sim, stream_handle))


def qs_set_option(sim, key: int, value: int):
    _check(sim, library().qs_set_option(sim, key, int(value)))


def qs_init_plus(sim):
    _check(sim, library().qs_init_plus(sim))


def qs_init_toric(sim, which: int):
    _check(sim, library().qs_init_toric(sim, which))


def qs_evolve_path(sim, per_step, dt: float, order: int, batch: int = 1):
    """per_step: sequence of n_steps coupling records (batch 1) or of n_steps lists of
    `batch` records; step k evolves under H1 with those couplings.  A float64 numpy array
    of shape (n_steps * batch, 4) with columns (g, lambda, J, h), step-major, is passed
    without a per-record Python loop."""
    if hasattr(per_step, "shape") and hasattr(per_step, "dtype"):
        import numpy as np
        a = np.asarray(per_step, dtype=np.float64)
        if a.ndim != 2 or a.shape[1] != 4 or a.shape[0] % batch:
            raise ValueError("per-step coupling array must have shape (n_steps * batch, 4)")
        rec = np.ascontiguousarray(a[:, [2, 3, 0, 1]])          # qs_couplings layout {J, h, g, lambda}
        arr = rec.ctypes.data_as(ctypes.POINTER(qs_couplings))
        _check(sim, library().qs_evolve_path(sim, arr, dt, a.shape[0] // batch, order))
        return
    flat = []
    for rec in per_step:
        if batch == 1:
            flat.append(rec)
        else:
            assert len(rec) == batch
            flat.extend(rec)
    n_steps = len(flat) // batch
    arr = _couplings(flat, len(flat))
    _check(sim, library().qs_evolve_path(sim, arr, dt, n_steps, order))


def qs_upload_state(sim, host_ptr: int, nbytes: int):
    _check(sim, library().qs_upload_state(sim, host_ptr, nbytes))


def qs_download_state(sim, host_ptr: int, nbytes: int):
    _check(sim, library().qs_download_state(sim, host_ptr, nbytes))


def qs_trotter_step(sim, couplings, s: float, dt: float, order: int, batch: int = 1):
    arr = _couplings(couplings, batch)
    _check(sim, library().qs_trotter_step(sim, arr, s, dt, order))


def qs_evolve(sim, couplings, s: Sequence[float], dt: float, order: int, batch: int = 1):
    arr = _couplings(couplings, batch)
    sv = np.ascontiguousarray(s, dtype=np.float64)
    _check(sim, library().qs_evolve(sim, arr, sv.ctypes.data_as(_DP), dt, int(sv.size), order))


def qs_expect(sim, kind: int, index: int = 0, couplings=None, s: float = 1.0, batch: int = 1):
    out = np.zeros(batch, dtype=np.float64)
    arr = _couplings(couplings, batch) if couplings is not None else None
    _check(sim, library().qs_expect(sim, kind, index, arr, s, out.ctypes.data_as(_DP)))
    return out


def qs_expect_pauli(sim, ptype: int, mask: int, batch: int = 1):
    out = np.zeros(batch, dtype=np.float64)
    _check(sim, library().qs_expect_pauli(sim, ptype, mask, out.ctypes.data_as(_DP)))
    return out


def qs_fidelity(sim, ref_dev_ptr: int, batch: int = 1):
    out = np.zeros(batch, dtype=np.float64)
    _check(sim, library().qs_fidelity(sim, ref_dev_ptr, out.ctypes.data_as(_DP)))
    return out


def qs_adjoint_grad(sim, couplings, s: Sequence[float], dt: float, order: int, target: int = 0,
                    ref_dev_ptr: int | None = None, batch: int = 1):
    """Returns (value[batch], dV/ds[batch, n_steps]) (see include/qsim.h)."""
    arr = _couplings(couplings, batch)
    sv = np.ascontiguousarray(s, dtype=np.float64)
    grad = np.zeros((batch, sv.size), dtype=np.float64)
    val = np.zeros(batch, dtype=np.float64)
    _check(sim, library().qs_adjoint_grad(sim, arr, sv.ctypes.data_as(_DP), dt, int(sv.size), order, target,
                                          ref_dev_ptr, grad.ctypes.data_as(_DP), val.ctypes.data_as(_DP)))
    return val, grad


QS_SCAN_NOBS = 8


def qs_scan(sim, points, s: Sequence[float], dt: float, order: int = 2):
    """Independent runs for every coupling record; returns out[n_points, QS_SCAN_NOBS]."""
    pts = _couplings(points, len(points))
    sv = np.ascontiguousarray(s, dtype=np.float64)
    out = np.zeros((len(points), QS_SCAN_NOBS), dtype=np.float64)
    _check(sim, library().qs_scan(sim, pts, len(points), sv.ctypes.data_as(_DP), dt, int(sv.size), order,
                                  out.ctypes.data_as(_DP)))
    return out


def qs_scan_mixed(sim12, points12, sim, points17, s: Sequence[float], dt: float, order: int = 2):
    """Both lattices' points in one launch; returns (out12[n12, 8], out17[n17, 8])."""
    n12, n17 = len(points12), len(points17)
    p12 = _couplings(points12, n12) if n12 else None
    p17 = _couplings(points17, n17) if n17 else None
    sv = np.ascontiguousarray(s, dtype=np.float64)
    o12 = np.zeros((max(n12, 1), QS_SCAN_NOBS), dtype=np.float64)
    o17 = np.zeros((max(n17, 1), QS_SCAN_NOBS), dtype=np.float64)
    _check(sim, library().qs_scan_mixed(sim12, p12, n12, sim, p17, n17, sv.ctypes.data_as(_DP), dt, int(sv.size),
                                        order, o12.ctypes.data_as(_DP), o17.ctypes.data_as(_DP)))
    return o12[:n12], o17[:n17]


def qs_num_links(sim) -> int:
    return library().qs_num_links(sim)


def qs_dos(sim, batch: int = 1):
    """Density of states of Z~ = -sum_l sigma^z_l: out[b, k] = weight of Z~ = 2k - n_links."""
    nl = qs_num_links(sim)
    out = np.zeros((batch, nl + 1), dtype=np.float64)
    _check(sim, library().qs_dos(sim, out.ctypes.data_as(_DP)))
    return out


def qs_autotune(sim, n_steps: int = 20):
    """Returns (xpass kernel, tile buffers, store mode, shared-pass tile buffers,
    shared-pass kernel, ms per step) of the fastest configuration."""
    xp, nb, so, ns, sk, ms = _I(), _I(), _I(), _I(), _I(), ctypes.c_double()
    _check(sim, library().qs_autotune(sim, n_steps, ctypes.byref(xp), ctypes.byref(nb), ctypes.byref(so),
                                      ctypes.byref(ns), ctypes.byref(sk), ctypes.byref(ms)))
    return xp.value, nb.value, so.value, ns.value, sk.value, ms.value


def qs_autotune_plan(sim, n_steps: int = 20):
    """Returns (qubits fused per pass, ms per step) of the fastest pass plan."""
    buf = (_I * 16)()
    np_, ms = _I(), ctypes.c_double()
    _check(sim, library().qs_autotune_plan(sim, n_steps, buf, 16, ctypes.byref(np_), ctypes.byref(ms)))
    return [buf[i] for i in range(np_.value)], ms.value


def qs_plan(sim):
    """Qubits fused by each tiled X pass (the first pass 12); [] below one tile."""
    buf = (_I * 64)()
    n = library().qs_plan(sim, buf, 64)
    if n < 0:
        raise QsError(1, "qs_plan failed")
    return [buf[i] for i in range(n)]


def plan_code(qubits_per_pass) -> int:
    """QS_OPT_PLAN value of a plan given as qubits per pass (first pass 12)."""
    code = 0
    for j, k in enumerate(qubits_per_pass[1:]):
        code |= int(k) << (4 * j)
    return code


def qs_selftest_wait(sim, limit_ms: float):
    _check(sim, library().qs_selftest_wait(sim, float(limit_ms)))


def qs_save(sim, path: str):
    _check(sim, library().qs_save(sim, os.fsencode(path)))


def qs_load(sim, path: str):
    _check(sim, library().qs_load(sim, os.fsencode(path)))


def qs_sync(sim):
    _check(sim, library().qs_sync(sim))


def qs_profile_read(sim):
    ms = ctypes.c_double()
    cnt = _LL()
    _check(sim, library().qs_profile_read(sim, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def qs_profile_read_kinds(sim):
    """((ms, launches) of passes of one factor group, (ms, launches) of shared passes)."""
    ms = (ctypes.c_double * 2)()
    cnt = (_LL * 2)()
    _check(sim, library().qs_profile_read_kinds(sim, ms, cnt))
    return (ms[0], cnt[0]), (ms[1], cnt[1])


def qs_launch_count(sim) -> int:
    return library().qs_launch_count(sim)


def qs_expect_z_noalloc(state_dev_ptr: int, n_qubits: int, dtype: int, batch: int, zmask: int,
                        out_dev_ptr: int, stream_handle: int = 0):
    """Norm and <Z_mask> per batch element into caller-owned device memory
    out[2b], out[2b+1], with no allocation (see include/qsim.h)."""
    _check(None, library().qs_expect_z_noalloc(state_dev_ptr, n_qubits, dtype, batch, zmask,
                                               out_dev_ptr, stream_handle))


# ---------------------------------------------------------------------------
# convenience object: owns a torch state buffer on the GPU and a qs_sim handle
# ---------------------------------------------------------------------------
class Simulator:
    """Lattice simulator with PyTorch-allocated device state(s).

    form: "gh" (gauge-Higgs, Eq. (1)) or "ug" (unitary gauge, Eq. (4));
    dtype: "c64" or "c128"; boundary: "periodic" or "open".
    """

    def __init__(self, Lx: int, Ly: int, form: str = "gh", dtype: str = "c64",
                 boundary: str = "periodic", batch: int = 1, device: str = "cuda:0",
                 method: str = "fused", renorm_every: int = 0, aux: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the qsim engine needs a CUDA GPU; there is no CPU path")
        self.torch = torch
        self.batch = batch
        self.form = form
        self.dtype_name = dtype
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        self.h = qs_create(Lx, Ly, QS_PERIODIC if boundary == "periodic" else QS_OPEN,
                           QS_GAUGE_HIGGS if form == "gh" else QS_UNITARY_GAUGE,
                           QS_C64 if dtype == "c64" else QS_C128, batch)
        self.n = qs_num_qubits(self.h)
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        self.state = torch.empty((batch, 1 << self.n), dtype=tdt, device=self.device)
        qs_bind_state(self.h, 0, self.state.data_ptr(), self.state.numel() * self.state.element_size())
        self.aux = None
        if aux:
            self.aux = torch.empty_like(self.state)
            qs_bind_state(self.h, 1, self.aux.data_ptr(), self.aux.numel() * self.aux.element_size())
        self.set_stream(torch.cuda.current_stream(self.device))
        self.set_option(QS_OPT_METHOD, 0 if method == "fused" else 1)
        self.set_option(QS_OPT_RENORM_EVERY, renorm_every)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            qs_destroy(h)
            self.h = None

    # --- plumbing ---
    def set_stream(self, stream):
        self.stream = stream
        qs_set_stream(self.h, stream.cuda_stream)

    def set_option(self, key, value):
        qs_set_option(self.h, key, value)

    @property
    def state_bytes(self) -> int:
        return qs_state_bytes(self.h)

    # --- evolution ---
    def init_plus(self):
        qs_init_plus(self.h)

    def init_toric(self, which=0):
        qs_init_toric(self.h, which)

    def evolve_path(self, per_step, dt, order=2):
        qs_evolve_path(self.h, per_step, dt, order, self.batch)

    def trotter_step(self, couplings, s, dt, order=2):
        qs_trotter_step(self.h, couplings, s, dt, order, self.batch)

    def evolve(self, couplings, s, dt, order=2):
        qs_evolve(self.h, couplings, s, dt, order, self.batch)

    # --- observables ---
    def expect(self, kind, index=0, couplings=None, s=1.0):
        return qs_expect(self.h, kind, index, couplings, s, self.batch)

    def energy(self, couplings, s=None):
        if s is None:
            return self.expect(QS_ENERGY, 0, couplings, 1.0)
        return self.expect(QS_ENERGY_S, 0, couplings, s)

    def expect_pauli(self, ptype, mask):
        return qs_expect_pauli(self.h, ptype, mask, self.batch)

    def fidelity(self, ref_state):
        assert ref_state.shape == self.state.shape and ref_state.dtype == self.state.dtype
        return qs_fidelity(self.h, ref_state.data_ptr(), self.batch)

    def upload(self, host_tensor):
        assert host_tensor.is_contiguous() and host_tensor.numel() == self.state.numel()
        qs_upload_state(self.h, host_tensor.data_ptr(), self.state_bytes)

    def download(self, host_tensor=None):
        if host_tensor is None:
            host_tensor = self.torch.empty(self.state.shape, dtype=self.state.dtype, pin_memory=True)
        qs_download_state(self.h, host_tensor.data_ptr(), self.state_bytes)
        return host_tensor

    def sync(self):
        qs_sync(self.h)

    def autotune(self, n_steps: int = 20, cache: bool = True):
        """Pick the fastest pass plan (qubits fused per X pass) and then the fastest
        X-pass configuration for this lattice, dtype and batch on this GPU, remembering
        both in a JSON cache (QSIM_CACHE, default ~/.cache/qsim_gb300/autotune.json).
        Overwrites the state."""
        import json
        key = "|".join(str(x) for x in (self.torch.cuda.get_device_name(self.device), self.n, self.dtype_name,
                                        self.form, self.batch))
        path = os.environ.get("QSIM_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "qsim_gb300",
                                                         "autotune.json"))
        table = {}
        if cache and os.path.exists(path):
            try:
                table = json.load(open(path))
            except (OSError, ValueError):
                table = {}
        if cache and key in table and "shared_kernel" in table[key] and "plan" in table[key]:
            e = table[key]
            if self.n > 12:
                self.set_option(QS_OPT_PLAN, plan_code(e["plan"]))
            self.set_option(QS_OPT_XPASS, e["xpass"])
            self.set_option(QS_OPT_TMA_BUFFERS, e["buffers"])
            self.set_option(QS_OPT_TMA_STORE, e["store"])
            self.set_option(QS_OPT_SHARED_BUFFERS, e["shared_buffers"])
            self.set_option(QS_OPT_SHARED_KERNEL, e["shared_kernel"])
            return e
        plan, plan_ms = (qs_autotune_plan(self.h, n_steps) if self.n > 12 else (qs_plan(self.h), None))
        xp, nb, so, ns, sk, ms = qs_autotune(self.h, n_steps)
        entry = {"plan": plan, "plan_ms_per_step": plan_ms, "xpass": xp, "buffers": nb, "store": so,
                 "shared_buffers": ns, "shared_kernel": sk, "ms_per_step": ms}
        if cache:
            table[key] = entry
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                json.dump(table, open(path, "w"), indent=1)
            except OSError:
                pass
        return entry

    def plan(self):
        return qs_plan(self.h)

    def dos(self):
        return qs_dos(self.h, self.batch)

    def save(self, path):
        qs_save(self.h, path)

    def load(self, path):
        qs_load(self.h, path)

    def scan(self, points, s, dt, order=2):
        return qs_scan(self.h, points, s, dt, order)

    def adjoint_grad(self, couplings, s, dt, order=2, target="energy", ref_state=None):
        """Forward evolution from the current state, value and dV/ds_k by the adjoint
        sweep.  Needs aux=True at construction (the adjoint work state)."""
        if self.aux is None:
            raise ValueError("construct the Simulator with aux=True for the adjoint")
        ref = None
        if target == "fidelity":
            assert ref_state is not None and ref_state.shape == self.state.shape
            ref = ref_state.data_ptr()
        return qs_adjoint_grad(self.h, couplings, s, dt, order, 0 if target == "energy" else 1, ref,
                               self.batch)

    def profile_read(self):
        return qs_profile_read(self.h)

    def profile_read_kinds(self):
        return qs_profile_read_kinds(self.h)

    def launch_count(self):
        return qs_launch_count(self.h)
