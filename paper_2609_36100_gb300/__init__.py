"""Python binding of the GB300 pseudospectral ImEx-ARK phase-field library.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libpf.so`` behind the C ABI of ``include/pf.h``.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library is missing or no
GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build  # noqa: F401

PF_OK = 0
PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENONFINITE, PF_ESTEPFAIL, PF_ETIMEOUT, PF_EUNSUPPORTED = range(-1, -8, -1)
PF_EULER, PF_ARK2, PF_ARK3, PF_ARK4 = 1, 2, 3, 4
PF_FP64, PF_FP32BULK = 0, 1
METHODS = {"euler": PF_EULER, "ark2": PF_ARK2, "ark3": PF_ARK3, "ark4": PF_ARK4}
PRECISIONS = {"fp64": PF_FP64, "fp32bulk": PF_FP32BULK, "fp32": PF_FP32BULK}


class PFGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class PFParams(C.Structure):
    _fields_ = [
        ("A_m", C.c_double), ("A_v", C.c_double), ("A0_m", C.c_double), ("A0_v", C.c_double),
        ("B_m0", C.c_double), ("B_v", C.c_double), ("dBm_dT", C.c_double),
        ("M0", C.c_double), ("Q_act", C.c_double), ("T", C.c_double), ("T0", C.c_double), ("L", C.c_double),
        ("kappa", (C.c_double * 6) * 3), ("omega_bar", C.c_double), ("omega_pair", C.c_double * 3),
        ("pair_eps", C.c_double),
        ("C11", C.c_double), ("C12", C.c_double), ("C44", C.c_double),
        ("eps_star", (C.c_double * 6) * 3),
        ("method", C.c_int), ("precision", C.c_int),
        ("rtol", C.c_double), ("atol", C.c_double),
        ("h0", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double),
        ("max_rejects", C.c_int),
        ("safety", C.c_double), ("k1", C.c_double), ("k2", C.c_double),
        ("eta_max", C.c_double), ("eta_min", C.c_double), ("eta_reject_min", C.c_double),
        ("el_inhom", C.c_int), ("C11_v", C.c_double), ("C12_v", C.c_double), ("C44_v", C.c_double),
        ("el_tol", C.c_double), ("el_max_iter", C.c_int), ("el_warm", C.c_int),
        ("barrier", C.c_int),
    ]


class PFStats(C.Structure):
    _fields_ = [("steps_accepted", C.c_longlong), ("steps_rejected", C.c_longlong), ("rhs_evals", C.c_longlong),
                ("t", C.c_double), ("h", C.c_double), ("last_wrms", C.c_double), ("wall_s", C.c_double),
                ("point_stages", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every entry point of include/pf.h: name -> (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "pf_create": (C.c_int, [C.POINTER(PFGrid), C.POINTER(PFParams), _P, C.POINTER(_P)]),
    "pf_destroy": (None, [_P]),
    "pf_set_state": (C.c_int, [_P, _P, C.c_int]),
    "pf_get_state": (C.c_int, [_P, _P, C.c_int]),
    "pf_set_state_hat": (C.c_int, [_P, _P, C.c_int]),
    "pf_get_state_hat": (C.c_int, [_P, _P, C.c_int]),
    "pf_rhs_explicit": (C.c_int, [_P, _P, _P]),
    "pf_solve_implicit": (C.c_int, [_P, C.c_double, _P, _P]),
    "pf_step": (C.c_int, [_P, C.c_double, C.POINTER(C.c_double)]),
    "pf_advance": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.POINTER(PFStats)]),
    "pf_advance_attempts": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(PFStats)]),
    "pf_batch_advance": (C.c_int, [C.POINTER(_P), C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(PFStats)]),
    "pf_batch_mode": (C.c_int, [C.c_int]),
    "pf_batch_last": (C.c_int, [C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "pf_free_energy": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "pf_get_time": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pf_set_time": (C.c_int, [_P, C.c_double, C.c_double]),
    "pf_get_stats": (C.c_int, [_P, C.POINTER(PFStats)]),
    "pf_get_controller": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "pf_elastic_iterations": (C.c_int, [_P]),
    "pf_set_controller": (C.c_int, [_P, C.c_double, C.c_int]),
    "pf_batch_round_cap": (C.c_longlong, [C.c_longlong]),
    "pf_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "pf_get_attempts": (C.c_int, [_P, C.POINTER(C.c_double), C.c_int]),
    "pf_method_tableau": (C.c_int, [C.c_int] + [C.POINTER(C.c_double)] * 6),
    "pf_last_error": (C.c_char_p, [_P]),
    "pf_profile_enable": (C.c_int, [_P, C.c_int]),
    "pf_profile_read": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "pf_kernel_name": (C.c_char_p, [C.c_int]),
    "pf_state_to_real_noalloc": (C.c_int, [C.POINTER(PFGrid), _P, _P, _P]),
    "pf_get_tuning": (C.c_int, [_P, C.POINTER(C.c_int), C.c_int]),
    "pf_set_tuning": (C.c_int, [_P, C.POINTER(C.c_int), C.c_int]),
    "pf_autotune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pf_fno_create": (C.c_int, [C.c_int] * 8 + [_P, C.POINTER(_P)]),
    "pf_fno_destroy": (None, [_P]),
    "pf_fno_num_params": (C.c_longlong, [_P]),
    "pf_fno_set_params": (C.c_int, [_P, _P, C.c_longlong]),
    "pf_fno_get_params": (C.c_int, [_P, _P, C.c_longlong]),
    "pf_fno_get_grads": (C.c_int, [_P, _P, C.c_longlong]),
    "pf_fno_set_norm": (C.c_int, [_P, _P, _P, _P]),
    "pf_fno_forward": (C.c_int, [_P, _P, _P]),
    "pf_fno_backward": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
    "pf_fno_adam": (C.c_int, [_P, C.c_float, C.c_float, C.c_float, C.c_float]),
    "pf_fno_train_step": (C.c_int, [_P, _P, _P, C.c_float, C.POINTER(C.c_double)]),
    "pf_fno_last_error": (C.c_char_p, [_P]),
    "pf_fno_fit_norm": (C.c_int, [_P, _P, C.c_int, C.c_int]),
    "pf_fno_train_pair": (C.c_int, [_P, _P, _P, C.c_float, C.POINTER(C.c_double)]),
    "pf_surrogate_step": (C.c_int, [_P, _P, C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)]),
}
NKERNELS = 11
TUNE_LEN = 43
_DPTR_ARGS = {"pf_method_tableau"}

_lib = None


def lib(path: str | None = None):
    """Load libpf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    so = path or LIB
    if not os.path.exists(so):
        raise RuntimeError("libpf.so not built (%s): run paper_2609_36100_gb300.build.build()" % so)
    L = C.CDLL(so)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = L
    return L


class PFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pf error %d: %s" % (code, msg))
        self.code = code


def _check(rc, ctx=None):
    if rc != PF_OK:
        msg = lib().pf_last_error(ctx)
        raise PFError(rc, msg.decode() if msg else "")
    return rc


def make_params(p: dict, method="ark4", precision="fp64") -> PFParams:
    """Pack a parameter dict (synth.load_params layout) into the C struct."""
    q = PFParams()
    for k in ("A_m", "A_v", "A0_m", "A0_v", "B_m0", "B_v", "dBm_dT", "M0", "Q_act", "T", "T0", "L", "omega_bar",
              "C11", "C12", "C44", "pair_eps", "rtol", "atol", "h0", "h_min", "h_max", "safety", "k1", "k2", "eta_max",
              "eta_min", "eta_reject_min"):
        setattr(q, k, float(p[k]))
    for v in range(3):
        for i in range(6):
            q.kappa[v][i] = float(p["kappa"][v][i])
            q.eps_star[v][i] = float(p["eps_star"][v][i])
        q.omega_pair[v] = float(p["omega_pair"][v])
    q.max_rejects = int(p["max_rejects"])
    q.el_inhom = int(p.get("el_inhom", 0))
    q.C11_v = float(p.get("C11_v", p["C11"]))
    q.C12_v = float(p.get("C12_v", p["C12"]))
    q.C44_v = float(p.get("C44_v", p["C44"]))
    q.el_tol = float(p.get("el_tol", 1e-6))
    q.el_max_iter = int(p.get("el_max_iter", 20))
    q.el_warm = int(p.get("el_warm", 1))
    q.barrier = int(p.get("barrier", 0))
    q.method = METHODS[method] if isinstance(method, str) else int(method)
    q.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return q


def method_tableau(method="ark4"):
    """Butcher arrays compiled into the library (host query, no GPU)."""
    m = METHODS[method] if isinstance(method, str) else int(method)
    bufs = [(C.c_double * 64)() for _ in range(6)]
    s = lib().pf_method_tableau(m, *[C.cast(b, C.POINTER(C.c_double)) for b in bufs])
    if s < 0:
        raise PFError(s, "unknown method")
    AE = np.array(bufs[0][: s * s]).reshape(s, s)
    AI = np.array(bufs[1][: s * s]).reshape(s, s)
    return AE, AI, np.array(bufs[2][:s]), np.array(bufs[3][:s]), np.array(bufs[4][:s]), np.array(bufs[5][:s])


def _torch():
    import torch
    return torch


class Simulation:
    """One periodic phase-field simulation on the current CUDA device.

    shape = (nz, ny, nx); the state is 4 fields (X, phi_1..3)."""

    def __init__(self, shape, p: dict, method="ark4", precision="fp64", dx=None, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        d = float(p["dx"] if dx is None else dx)
        self.grid = PFGrid(nx, ny, nz, d, d, d)
        self.params = make_params(p, method, precision)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = C.c_void_p()
        rc = lib().pf_create(C.byref(self.grid), C.byref(self.params), C.c_void_p(self.stream.cuda_stream),
                             C.byref(ctx))
        _check(rc, None)
        self.ctx = ctx
        self.nxh = nx // 2 + 1

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            lib().pf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state ----------------------------------------------------------------
    def set_state(self, fields):
        """Real-space fields [4][nz][ny][nx] (numpy host array or CUDA tensor)."""
        torch = _torch()
        if isinstance(fields, torch.Tensor):
            t = fields.to(torch.float64).contiguous()
            _check(lib().pf_set_state(self.ctx, C.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0), self.ctx)
        else:
            a = np.ascontiguousarray(fields, dtype=np.float64)
            assert a.shape == (4,) + self.shape
            _check(lib().pf_set_state(self.ctx, a.ctypes.data_as(C.c_void_p), 0), self.ctx)

    def get_state(self, out=None):
        """Real-space fields as a numpy array (or into a CUDA float64 tensor)."""
        if out is not None:
            assert out.dtype == _torch().float64 and out.is_contiguous() and out.numel() == 4 * int(np.prod(self.shape))
            _check(lib().pf_get_state(self.ctx, C.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0), self.ctx)
            return out
        a = np.empty((4,) + self.shape, dtype=np.float64)
        _check(lib().pf_get_state(self.ctx, a.ctypes.data_as(C.c_void_p), 0), self.ctx)
        return a

    def k_shape(self):
        return (4,) + self.shape[:2] + (self.nxh,)

    def state_hat(self):
        """k-space state y^ as a CUDA complex128 tensor [4][nz][ny][nx/2+1]."""
        torch = _torch()
        t = torch.empty(self.k_shape(), dtype=torch.complex128, device="cuda")
        _check(lib().pf_get_state_hat(self.ctx, C.c_void_p(t.data_ptr()), 1), self.ctx)
        return t

    def set_state_hat(self, y_hat):
        torch = _torch()
        if isinstance(y_hat, torch.Tensor) and y_hat.is_cuda:
            t = y_hat.to(torch.complex128).contiguous()
            _check(lib().pf_set_state_hat(self.ctx, C.c_void_p(t.data_ptr()), 1), self.ctx)
        else:
            a = np.ascontiguousarray(y_hat, dtype=np.complex128)
            _check(lib().pf_set_state_hat(self.ctx, a.ctypes.data_as(C.c_void_p), 0), self.ctx)

    # -- operators --------------------------------------------------------------
    def rhs_explicit(self, y_hat):
        torch = _torch()
        y = y_hat.to(torch.complex128).contiguous()
        out = torch.empty_like(y)
        _check(lib().pf_rhs_explicit(self.ctx, C.c_void_p(y.data_ptr()), C.c_void_p(out.data_ptr())), self.ctx)
        return out

    def solve_implicit(self, gamma, r_hat):
        torch = _torch()
        r = r_hat.to(torch.complex128).contiguous()
        out = torch.empty_like(r)
        _check(lib().pf_solve_implicit(self.ctx, float(gamma), C.c_void_p(r.data_ptr()), C.c_void_p(out.data_ptr())),
               self.ctx)
        return out

    # -- integration --------------------------------------------------------------
    def step(self, dt, want_lte=True):
        e = C.c_double(0.0)
        _check(lib().pf_step(self.ctx, float(dt), C.byref(e) if want_lte else None), self.ctx)
        return e.value

    def advance(self, t_final, rtol=None, atol=None):
        st = PFStats()
        rtol = self.params.rtol if rtol is None else rtol
        atol = self.params.atol if atol is None else atol
        _check(lib().pf_advance(self.ctx, float(t_final), float(rtol), float(atol), C.byref(st)), self.ctx)
        return st.as_dict()

    def advance_attempts(self, n, t_final=1e30, rtol=None, atol=None):
        """Up to n controller-driven step attempts toward t_final."""
        st = PFStats()
        rtol = self.params.rtol if rtol is None else rtol
        atol = self.params.atol if atol is None else atol
        _check(lib().pf_advance_attempts(self.ctx, float(t_final), float(rtol), float(atol), int(n), C.byref(st)),
               self.ctx)
        return st.as_dict()

    def attempts(self):
        n = lib().pf_get_attempts(self.ctx, None, 0)
        buf = (C.c_double * (4 * max(n, 1)))()
        lib().pf_get_attempts(self.ctx, C.cast(buf, C.POINTER(C.c_double)), n)
        a = np.array(buf[: 4 * n]).reshape(n, 4)
        return [(float(t), float(h), float(e), bool(ok)) for t, h, e, ok in a]

    def free_energy(self):
        F = C.c_double()
        _check(lib().pf_free_energy(self.ctx, C.byref(F)), self.ctx)
        return F.value

    def time(self):
        t, h = C.c_double(), C.c_double()
        _check(lib().pf_get_time(self.ctx, C.byref(t), C.byref(h)), self.ctx)
        return t.value, h.value

    def set_time(self, t, h):
        _check(lib().pf_set_time(self.ctx, float(t), float(h)), self.ctx)

    def elastic_iterations(self):
        """Hu-Chen solves of the last right-hand-side evaluation (1 without phase contrast)."""
        n = lib().pf_elastic_iterations(self.ctx)
        _check(n if n < 0 else PF_OK, self.ctx)
        return n

    def controller(self):
        """(e_prev, after_reject) of the PI controller (checkpoint/resume)."""
        e, r = C.c_double(), C.c_int()
        _check(lib().pf_get_controller(self.ctx, C.byref(e), C.byref(r)), self.ctx)
        return e.value, bool(r.value)

    def set_controller(self, e_prev, after_reject):
        _check(lib().pf_set_controller(self.ctx, float(e_prev), 1 if after_reject else 0), self.ctx)

    def checkpoint(self):
        """(k-space state as a host array, t, h, e_prev, after_reject)."""
        a = np.empty(self.k_shape(), dtype=np.complex128)
        _check(lib().pf_get_state_hat(self.ctx, a.ctypes.data_as(C.c_void_p), 0), self.ctx)
        t, h = self.time()
        e, r = self.controller()
        return a, t, h, e, r

    def restore(self, ck):
        y, t, h, e, r = ck
        self.set_state_hat(y)
        self.set_time(t, h)
        self.set_controller(e, r)

    def profile(self, on=True):
        _check(lib().pf_profile_enable(self.ctx, 1 if on else 0), self.ctx)

    def profile_read(self):
        """{kernel name: (ms, algorithmic bytes, launches)} since the last read."""
        ms = (C.c_double * NKERNELS)()
        by = (C.c_double * NKERNELS)()
        n = (C.c_longlong * NKERNELS)()
        _check(lib().pf_profile_read(self.ctx, ms, by, n), self.ctx)
        return {lib().pf_kernel_name(k).decode(): (ms[k], by[k], n[k]) for k in range(NKERNELS) if n[k]}

    def tuning(self):
        buf = (C.c_int * TUNE_LEN)()
        _check(lib().pf_get_tuning(self.ctx, buf, TUNE_LEN), self.ctx)
        return list(buf)

    def set_tuning(self, cfg):
        buf = (C.c_int * TUNE_LEN)(*[int(v) for v in cfg])
        _check(lib().pf_set_tuning(self.ctx, buf, TUNE_LEN), self.ctx)

    def autotune(self, reps=3, cache=None):
        """Pick the fastest launch schedule for this grid/precision by timing
        step attempts; with `cache` (a JSON path) reuse/record the choice
        keyed by grid, precision, method and device name."""
        import json
        import os
        torch = _torch()
        key = "%s|%d|%d|%s" % ("x".join(map(str, self.shape)), self.params.precision, self.params.method,
                               torch.cuda.get_device_name())
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                self.set_tuning(table[key]["cfg"])
                return table[key]
        b, a = C.c_double(), C.c_double()
        _check(lib().pf_autotune(self.ctx, int(reps), C.byref(b), C.byref(a)), self.ctx)
        rec = {"cfg": self.tuning(), "ms_before": b.value, "ms_after": a.value}
        if cache:
            table[key] = rec
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        return rec

    def stats(self):
        st = PFStats()
        _check(lib().pf_get_stats(self.ctx, C.byref(st)), self.ctx)
        return st.as_dict()


def batch_advance(sims, t_final, rtol=1e-4, atol=1e-8, polled=False):
    """Advance several simulations (same method and precision) to t_final;
    `polled` forces the host-polled round driver instead of the device-looped
    graph."""
    n = len(sims)
    arr = (C.c_void_p * n)(*[s.ctx.value for s in sims])
    st = (PFStats * n)()
    prev = lib().pf_batch_mode(1 if polled else 0)
    try:
        rc = lib().pf_batch_advance(arr, n, float(t_final), float(rtol), float(atol), st)
    finally:
        lib().pf_batch_mode(prev)
    _check(rc, sims[0].ctx if rc != PF_OK else None)
    return [s.as_dict() for s in st]


def fma_peak(precision="fp64"):
    """Measured dense FMA throughput of the current device (TFLOP/s)."""
    v = C.c_double()
    _check(lib().pf_fma_peak(PRECISIONS[precision] if isinstance(precision, str) else int(precision), C.byref(v)))
    return v.value


def batch_round_cap(cap=0):
    """Set the round cap of batch_advance (cap > 0) and return the previous
    one; cap <= 0 only queries."""
    return int(lib().pf_batch_round_cap(int(cap)))


def batch_last():
    """(rounds, device_looped) of the last batch_advance call."""
    r, lp = C.c_longlong(), C.c_int()
    lib().pf_batch_last(C.byref(r), C.byref(lp))
    return r.value, bool(lp.value)


class FNO:
    """Fourier-neural-operator surrogate on the current CUDA device (forward,
    backward and Adam in the library's kernels).  Arrays are CUDA float32
    tensors [4][nz][ny][nx]."""

    def __init__(self, shape, C=32, modes=12, H=128, L=4, bf16=True, stream=None):
        torch = _torch()
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ptr = _ctypes_void_p()
        rc = lib().pf_fno_create(nx, ny, nz, C_int(C), C_int(modes), C_int(H), C_int(L), 1 if bf16 else 0,
                                 _ctypes_void_p(self.stream.cuda_stream), _byref(ptr))
        if rc != PF_OK:
            raise PFError(rc, lib().pf_fno_last_error(None).decode())
        self.f = ptr
        self.n = int(lib().pf_fno_num_params(self.f))

    def _chk(self, rc):
        if rc != PF_OK:
            raise PFError(rc, lib().pf_fno_last_error(self.f).decode())

    def close(self):
        if getattr(self, "f", None):
            lib().pf_fno_destroy(self.f)
            self.f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.n
        self._chk(lib().pf_fno_set_params(self.f, a.ctypes.data_as(_ctypes_void_p), self.n))

    def params(self):
        a = np.empty(self.n, dtype=np.float32)
        self._chk(lib().pf_fno_get_params(self.f, a.ctypes.data_as(_ctypes_void_p), self.n))
        return a

    def grads(self):
        a = np.empty(self.n, dtype=np.float32)
        self._chk(lib().pf_fno_get_grads(self.f, a.ctypes.data_as(_ctypes_void_p), self.n))
        return a

    def set_norm(self, in_mean, in_std, out_std):
        arrs = [np.ascontiguousarray(v, dtype=np.float32) for v in (in_mean, in_std, out_std)]
        self._chk(lib().pf_fno_set_norm(self.f, *[a.ctypes.data_as(_ctypes_void_p) for a in arrs]))
        self._norm = arrs

    def forward(self, x):
        torch = _torch()
        out = torch.empty_like(x)
        self._chk(lib().pf_fno_forward(self.f, _ctypes_void_p(x.data_ptr()), _ctypes_void_p(out.data_ptr())))
        return out

    def backward(self, target):
        l = C_double()
        self._chk(lib().pf_fno_backward(self.f, _ctypes_void_p(target.data_ptr()), _byref(l)))
        return l.value

    def train_step(self, x, target, lr):
        l = C_double()
        self._chk(lib().pf_fno_train_step(self.f, _ctypes_void_p(x.data_ptr()), _ctypes_void_p(target.data_ptr()),
                                          float(lr), _byref(l)))
        return l.value

    def fit_norm(self, snaps):
        """Normalisation from a CUDA float32 tensor [n_traj][n_snap][4][nz][ny][nx]."""
        assert snaps.is_cuda and snaps.dtype == _torch().float32 and snaps.is_contiguous()
        self._chk(lib().pf_fno_fit_norm(self.f, _ctypes_void_p(snaps.data_ptr()), int(snaps.shape[0]),
                                        int(snaps.shape[1])))

    def train_pair(self, s0, s1, lr):
        l = C_double()
        self._chk(lib().pf_fno_train_pair(self.f, _ctypes_void_p(s0.data_ptr()), _ctypes_void_p(s1.data_ptr()),
                                          float(lr), _byref(l)))
        return l.value

    def surrogate_step(self, sim, tau, h, rtol=1e-4, atol=1e-8):
        """(accepted, WRMS distance of the proposal to the verified integration)."""
        acc = C_int()
        dist = C_double()
        self._chk(lib().pf_surrogate_step(sim.ctx, self.f, float(tau), float(h), float(rtol), float(atol),
                                          _byref(acc), _byref(dist)))
        return bool(acc.value), dist.value


_ctypes_void_p = C.c_void_p
_byref = C.byref
C_int = C.c_int
C_double = C.c_double
