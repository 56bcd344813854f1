"""Thin ctypes binding of libbicadmm.so (include/bicadmm.h).  Argument marshalling only:
every step of the solver runs in the library's CUDA kernels.

The functions mirror the C ABI names without the ``bicadmm_`` prefix.  Device buffers
may be passed as torch CUDA tensors (their data pointers are handed over); host buffers
as numpy arrays or CPU tensors.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build_lib import LIB

LOSS_SQUARED, LOSS_LOGISTIC, LOSS_SOFTMAX, LOSS_SQHINGE = 0, 1, 2, 3
PREC_FP64, PREC_FP32, PREC_BF16, PREC_TF32 = 0, 1, 2, 3
DTYPE_F64, DTYPE_F32, DTYPE_BF16 = 0, 1, 2
FIELD_X, FIELD_U, FIELD_Z, FIELD_S, FIELD_OMEGA, FIELD_NU, FIELD_SCALARS, FIELD_P = range(8)

STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_STATE",
          -5: "ERR_NUMERIC", -6: "ERR_TIMEOUT", -7: "ERR_UNSUPPORTED"}


class Params(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("K", ctypes.c_int64),
                ("N_shards", ctypes.c_int32), ("M_blocks", ctypes.c_int32),
                ("kappa", ctypes.c_int64),
                ("gamma", ctypes.c_double), ("rho_c", ctypes.c_double),
                ("rho_b", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("inner_iters", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("tol_rel", ctypes.c_double),
                ("pass_rows", ctypes.c_int32), ("pass_stages", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("p_r", ctypes.c_double), ("d_r", ctypes.c_double), ("b_r", ctypes.c_double),
                ("i_r", ctypes.c_double),
                ("p_rel", ctypes.c_double), ("d_rel", ctypes.c_double),
                ("b_rel", ctypes.c_double), ("i_rel", ctypes.c_double),
                ("t", ctypes.c_double), ("v", ctypes.c_double), ("tau", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("objective", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("iters_per_round", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("polish", ctypes.c_int32), ("pad", ctypes.c_int32)]


class BicadmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


_lib = None

# (name, restype, argtypes) for every symbol declared in include/bicadmm.h
_VP = ctypes.c_void_p
SIGNATURES = [
    ("bicadmm_default_params", ctypes.c_int, [ctypes.POINTER(Params)]),
    ("bicadmm_create", ctypes.c_int, [ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)]),
    ("bicadmm_setup", ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                     _VP, ctypes.c_int32, ctypes.c_int32]),
    ("bicadmm_step", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(Info)]),
    ("bicadmm_solve", ctypes.c_int, [_VP, ctypes.POINTER(Info)]),
    ("bicadmm_get_x", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                     ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_get_state", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int64]),
    ("bicadmm_set_profiling", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("bicadmm_set_graph", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("bicadmm_get_pass_time", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_get_kernel_times", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("bicadmm_get_trace", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_inject_pass_stall", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64]),
    ("bicadmm_create_path", ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int64), _VP, ctypes.POINTER(_VP)]),
    ("bicadmm_path_info", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(Info)]),
    ("bicadmm_path_get_x", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_consensus_step_noalloc", ctypes.c_int,
     [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
      ctypes.c_double, _VP]),
    ("bicadmm_batch_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int32, _VP, ctypes.c_int32,
                                            ctypes.POINTER(_VP)]),
    ("bicadmm_batch_step", ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_batch_tiling", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
    ("bicadmm_batch_kernel_times", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_batch_destroy", ctypes.c_int, [_VP]),
    ("bicadmm_batch_last_error", ctypes.c_char_p, [_VP]),
    ("bicadmm_estimate_bytes", ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_server_create", ctypes.c_int, [ctypes.POINTER(ServerParams), ctypes.POINTER(_VP)]),
    ("bicadmm_server_clock", ctypes.c_double, [_VP]),
    ("bicadmm_server_submit", ctypes.c_int, [_VP, ctypes.POINTER(Params), _VP, ctypes.c_int32,
                                             ctypes.c_int64, ctypes.c_int32, _VP, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_server_run", ctypes.c_int, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_server_set_open", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("bicadmm_server_timing", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    ("bicadmm_server_result", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(Info), ctypes.POINTER(ctypes.c_double)]),
    ("bicadmm_server_stats", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    ("bicadmm_server_destroy", ctypes.c_int, [_VP]),
    ("bicadmm_server_last_error", ctypes.c_char_p, [_VP]),
    ("bicadmm_destroy", ctypes.c_int, [_VP]),
    ("bicadmm_last_error", ctypes.c_char_p, [_VP]),
]


def lib():
    """Load libbicadmm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libbicadmm.so is not built (%s); run "
                               "`python -m paper_2405_16267_b300.build_lib`" % LIB)
        L = ctypes.CDLL(LIB)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, handle=None):
    if code != 0:
        msg = lib().bicadmm_last_error(handle)
        raise BicadmmError(code, msg.decode() if msg else "")


def default_params(**kw) -> Params:
    p = Params()
    _check(lib().bicadmm_default_params(ctypes.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def create(params: Params, stream=None):
    """stream: a torch.cuda.Stream, an int handle, or None for the default stream."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = _VP()
    _check(lib().bicadmm_create(ctypes.byref(params), _VP(stream or 0), ctypes.byref(h)))
    return h


def _buffer(arr):
    """(pointer, dtype code, on_device, keepalive) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(arr, torch.Tensor):
            codes = {torch.float64: DTYPE_F64, torch.float32: DTYPE_F32, torch.bfloat16: DTYPE_BF16}
            if arr.dtype not in codes:
                raise TypeError("A and b must be float64, float32 or bfloat16")
            if not arr.is_contiguous():
                arr = arr.contiguous()
            return arr.data_ptr(), codes[arr.dtype], int(arr.is_cuda), arr
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(arr)
    if a.dtype not in (np.float64, np.float32):
        a = a.astype(np.float64)
    code = DTYPE_F64 if a.dtype == np.float64 else DTYPE_F32
    return a.ctypes.data, code, 0, a


def setup(h, A, b):
    """A: (m, n) row-major; b: (m,).  numpy arrays / CPU tensors (host) or CUDA tensors."""
    pa, ca, da, ka = _buffer(A)
    pb, cb, db, kb = _buffer(b)
    n = ka.shape[1]
    _check(lib().bicadmm_setup(h, pa, ca, n, da, pb, cb, db), h)
    return None


def step(h, n_iters, info=True):
    if info:
        inf = Info()
        _check(lib().bicadmm_step(h, int(n_iters), ctypes.byref(inf)), h)
        return inf
    _check(lib().bicadmm_step(h, int(n_iters), None), h)
    return None


def solve(h) -> Info:
    inf = Info()
    _check(lib().bicadmm_solve(h, ctypes.byref(inf)), h)
    return inf


def get_x(h, n, polished=False, with_support=False, kappa=None):
    x = np.zeros(n)
    sup = None
    sp = None
    if with_support:
        sup = np.zeros(int(kappa), dtype=np.int64)
        sp = sup.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(lib().bicadmm_get_x(h, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n,
                               int(bool(polished)), sp), h)
    return (x, sup) if with_support else x


def get_state(h, field, length):
    out = np.zeros(int(length))
    _check(lib().bicadmm_get_state(h, int(field), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   int(length)), h)
    return out


TRACE_FIELDS = ("iter", "p_r", "d_r", "b_r", "i_r", "p_rel", "d_rel", "b_rel", "i_rel", "t", "v",
                "tau", "znorm", "zt_steps", "zt_lists")


def get_trace(h, max_records=4096):
    """Residual records of the last iterations as a dict of numpy arrays (oldest first)."""
    out = np.zeros((int(max_records), len(TRACE_FIELDS)))
    cnt = ctypes.c_int64()
    _check(lib().bicadmm_get_trace(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   int(max_records), ctypes.byref(cnt)), h)
    out = out[:cnt.value]
    return {k: out[:, i] for i, k in enumerate(TRACE_FIELDS)}


KERNEL_KINDS = ("pass", "xupd", "dual", "rhs")


def set_profiling(h, on=True):
    """on: False/0 off, True/1 the A pass only, 2 every kernel of the iteration."""
    _check(lib().bicadmm_set_profiling(h, int(on)), h)


def set_graph(h, iters_per_graph):
    """Replay iters_per_graph outer iterations per CUDA graph launch (0 = eager launches)."""
    _check(lib().bicadmm_set_graph(h, int(iters_per_graph)), h)


def get_kernel_times(h, reset=True):
    """{kind: (total ms, launches)} for the kernels timed since profiling was switched on."""
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    _check(lib().bicadmm_get_kernel_times(h, ms, cnt, int(bool(reset))), h)
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def get_pass_time(h):
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(lib().bicadmm_get_pass_time(h, ctypes.byref(ms), ctypes.byref(cnt)), h)
    return ms.value, cnt.value


def inject_pass_stall(h, panel, wait_limit_cycles=2_000_000):
    """Test hook: the next K = 1 A pass never loads `panel`, so its CTA times out after
    wait_limit_cycles (see include/bicadmm.h); panel < 0 disarms it."""
    _check(lib().bicadmm_inject_pass_stall(h, int(panel), int(wait_limit_cycles)), h)


def check_noalloc_args(w, z, s, tvt):
    """Reject, before any launch, tensors the kernels would index out of bounds: every
    argument a contiguous float64 CUDA tensor on one device, len(z) == len(s) == len(w) = n,
    len(tvt) >= 4.  Returns n."""
    import torch
    names = ("w", "z", "s", "tvt")
    for name, t in zip(names, (w, z, s, tvt)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != torch.float64:
            raise ValueError("%s must be float64, got %s" % (name, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    n = w.numel()
    if z.numel() != n or s.numel() != n:
        raise ValueError("w, z and s must have the same length (%d, %d, %d)"
                         % (n, z.numel(), s.numel()))
    if tvt.numel() < 4:
        raise ValueError("tvt must hold at least 4 doubles")
    for name, t in zip(names, (w, z, s, tvt)):
        if not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
    if len({t.device for t in (w, z, s, tvt)}) != 1:
        raise ValueError("w, z, s and tvt must be on one device")
    if w.device.index != torch.cuda.current_device():
        raise ValueError("the tensors must be on the current CUDA device (the library "
                         "launches there)")
    return n


def consensus_step_noalloc(w, z, s, tvt, kappa, N_shards, rho_c, rho_b, stream=None):
    """Allocation-free consensus update on caller device tensors (float64, contiguous):
    w, z, s of length n and tvt of length 4 (see include/bicadmm.h)."""
    n = check_noalloc_args(w, z, s, tvt)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(lib().bicadmm_consensus_step_noalloc(w.data_ptr(), z.data_ptr(), s.data_ptr(),
                                                tvt.data_ptr(), n, int(kappa), int(N_shards),
                                                float(rho_c), float(rho_b), _VP(stream or 0)))


BATCH_GRAPH, BATCH_AUTOTUNE, BATCH_PROFILE = 1, 2, 4


def _bcheck(code, b=None):
    if code != 0:
        msg = lib().bicadmm_batch_last_error(b)
        raise BicadmmError(code, msg.decode() if msg else "")


def batch_create(handles, stream=None, flags=0):
    """Batch over set-up handles (raw handles or Solver objects)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    hs = [getattr(h, "h", h) for h in handles]
    arr = (_VP * len(hs))(*[h.value if hasattr(h, "value") else h for h in hs])
    b = _VP()
    _bcheck(lib().bicadmm_batch_create(arr, len(hs), _VP(stream or 0), int(flags), ctypes.byref(b)))
    return b


def batch_step(b, n_iters):
    cnt = ctypes.c_int64()
    _bcheck(lib().bicadmm_batch_step(b, int(n_iters), ctypes.byref(cnt)), b)
    return cnt.value


def batch_tiling(b):
    r = ctypes.c_int32()
    st = ctypes.c_int32()
    _bcheck(lib().bicadmm_batch_tiling(b, ctypes.byref(r), ctypes.byref(st)), b)
    return r.value, st.value


def batch_kernel_times(b):
    """{kind: (ms, launches)} since the last call (needs BATCH_PROFILE)."""
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    _bcheck(lib().bicadmm_batch_kernel_times(b, ms, cnt), b)
    return {k: (ms[i], cnt[i]) for i, k in enumerate(("pass", "xupd", "dual", "consensus"))}


def batch_destroy(b):
    if b:
        _bcheck(lib().bicadmm_batch_destroy(b))


def estimate_bytes(params):
    dev = ctypes.c_int64()
    extra = ctypes.c_int64()
    _check(lib().bicadmm_estimate_bytes(ctypes.byref(params), ctypes.byref(dev), ctypes.byref(extra)))
    return dev.value, extra.value


def _scheck(code, s=None):
    if code != 0:
        msg = lib().bicadmm_server_last_error(s)
        raise BicadmmError(code, msg.decode() if msg else "")


class Server:
    """Serving loop with continuous batching (include/bicadmm.h, bicadmm_server_*)."""

    def __init__(self, hbm_budget_bytes, max_active=64, iters_per_round=10,
                 precision=PREC_FP32, use_graph=True, polish=True):
        sp = ServerParams(int(hbm_budget_bytes), int(max_active), int(iters_per_round),
                          int(precision), int(bool(use_graph)), int(bool(polish)), 0)
        self.s = _VP()
        _scheck(lib().bicadmm_server_create(ctypes.byref(sp), ctypes.byref(self.s)))
        self._keep = {}
        self._n = {}

    def clock(self):
        return lib().bicadmm_server_clock(self.s)

    def submit(self, A, b, arrival, **params):
        """A, b: numpy arrays (host) or torch tensors (host or device); kept alive here
        until the request's result is taken."""
        pa, ca, da, ka = _buffer(A)
        pb, cb, db, kb = _buffer(b)
        m, n = ka.shape
        p = default_params(m=m, n=n, **params)
        rid = ctypes.c_int64()
        _scheck(lib().bicadmm_server_submit(self.s, ctypes.byref(p), pa, ca, n, da, pb, cb, db,
                                            float(arrival), ctypes.byref(rid)), self.s)
        self._keep[rid.value] = (ka, kb)
        self._n[rid.value] = (n, p.kappa)
        return rid.value

    def run(self, until=1e30):
        done = ctypes.c_int64()
        _scheck(lib().bicadmm_server_run(self.s, float(until), ctypes.byref(done)), self.s)
        return done.value

    def result(self, rid):
        n, kappa = self._n[rid]
        x = np.zeros(n)
        sup = np.zeros(kappa, dtype=np.int64)
        inf = Info()
        t = (ctypes.c_double * 3)()
        code = lib().bicadmm_server_result(self.s, int(rid), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          n, sup.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          ctypes.byref(inf), t)
        if code != -4:  # finished (or failed): the server no longer reads its A and b
            self._keep.pop(rid, None)
        return dict(status=code, x=x, support=sup, info=inf, arrival=t[0], admitted=t[1], done=t[2])

    def set_open(self, flag=True):
        """While open, run() keeps waiting for submissions (from other threads) until its
        `until` has passed or the server is closed again."""
        _scheck(lib().bicadmm_server_set_open(self.s, int(bool(flag))), self.s)

    TIMING = ("arrival", "admitted", "setup_done", "retiring", "done", "iters", "rounds")
    PROFILE = ("rebuilds", "rebuild_s", "round_wait_s", "admit_s", "retire_s", "rounds", "clock")

    def timing(self, rid=-1):
        """Per request (rid >= 0, finished): arrival, admission (setup start), setup end,
        retirement start, completion (server clock, s), iterations and rounds.  rid = -1: the
        server's batch rebuilds and seconds spent rebuilding, waiting for rounds, admitting
        and retiring, its rounds and clock."""
        out = (ctypes.c_double * 7)()
        code = lib().bicadmm_server_timing(self.s, int(rid), out)
        if code != 0:
            raise BicadmmError(code, "request not finished" if code == -4 else "bad id")
        return dict(zip(self.PROFILE if rid < 0 else self.TIMING, list(out)))

    def stats(self):
        c = (ctypes.c_int64 * 5)()
        _scheck(lib().bicadmm_server_stats(self.s, c), self.s)
        return dict(submitted=c[0], finished=c[1], rounds=c[2], peak_bytes=c[3], launches=c[4])

    def close(self):
        if self.s:
            lib().bicadmm_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def destroy(h):
    if h:
        _check(lib().bicadmm_destroy(h))


def last_error(h=None) -> str:
    msg = lib().bicadmm_last_error(h)
    return msg.decode() if msg else ""


def create_path(params: Params, kappas, stream=None):
    """A sparsity path: len(kappas) instances of one problem (see include/bicadmm.h)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    k = (ctypes.c_int64 * len(kappas))(*[int(v) for v in kappas])
    h = _VP()
    _check(lib().bicadmm_create_path(ctypes.byref(params), len(kappas), k, _VP(stream or 0),
                                     ctypes.byref(h)))
    return h


class PathSolver:
    """Owner of a path handle: the instances of one problem at the given kappas, solved
    together on one copy of A."""

    def __init__(self, A, b, *, loss, N, M, kappas, gamma=10.0, rho_c=1.0, rho_b=0.0,
                 rho_l=0.0, precision=PREC_FP64, stream=None, **extra):
        m, n = A.shape
        self.n, self.m, self.N, self.kappas = int(n), int(m), int(N), [int(k) for k in kappas]
        self.params = default_params(loss=loss, precision=precision, m=m, n=n, N_shards=N,
                                     M_blocks=M, kappa=1, gamma=gamma, rho_c=rho_c,
                                     rho_b=rho_b, rho_l=rho_l, **extra)
        self.h = create_path(self.params, self.kappas, stream)
        try:
            setup(self.h, A, b)
        except Exception:
            destroy(self.h)
            self.h = None
            raise

    def step(self, n_iters, info=True):
        return step(self.h, n_iters, info)

    def solve(self):
        return solve(self.h)

    def info(self, q):
        inf = Info()
        _check(lib().bicadmm_path_info(self.h, int(q), ctypes.byref(inf)), self.h)
        return inf

    def x(self, q, with_support=False):
        """Instance q's z (n entries) and, optionally, its kappa-support."""
        x = np.zeros(self.n)
        sup = np.zeros(self.kappas[q], dtype=np.int64) if with_support else None
        sp = sup.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if with_support else None
        _check(lib().bicadmm_path_get_x(self.h, int(q), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        self.n, sp), self.h)
        return (x, sup) if with_support else x

    def state(self, q):
        """Instance q's x (N x n), u (N x n), z, s (n each) from the feature-major state."""
        R = len(self.kappas)
        N, n = self.N, self.n
        X = get_state(self.h, FIELD_X, N * n * R).reshape(N, n, R)
        U = get_state(self.h, FIELD_U, N * n * R).reshape(N, n, R)
        Z = get_state(self.h, FIELD_Z, n * R).reshape(n, R)
        S = get_state(self.h, FIELD_S, n * R).reshape(n, R)
        return dict(x=X[:, :, q].copy(), u=U[:, :, q].copy(), z=Z[:, q].copy(), s=S[:, q].copy())

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Convenience owner of one handle: create + setup on construction, destroy on close."""

    def __init__(self, A, b, *, loss, N, M, kappa, gamma=10.0, rho_c=1.0, rho_b=0.0,
                 rho_l=0.0, inner_iters=1, precision=PREC_FP64, stream=None, K=1, **extra):
        m, n = A.shape
        self.n, self.m, self.N, self.kappa, self.K = int(n), int(m), int(N), int(kappa), int(K)
        self.params = default_params(loss=loss, precision=precision, m=m, n=n, N_shards=N,
                                     M_blocks=M, kappa=kappa, gamma=gamma, rho_c=rho_c,
                                     rho_b=rho_b, rho_l=rho_l, inner_iters=inner_iters, K=K,
                                     **extra)
        self.h = create(self.params, stream)
        try:
            setup(self.h, A, b)
        except Exception:
            destroy(self.h)
            self.h = None
            raise

    def step(self, n_iters, info=True):
        return step(self.h, n_iters, info)

    def set_graph(self, iters_per_graph):
        set_graph(self.h, iters_per_graph)

    def solve(self):
        return solve(self.h)

    def x(self, polished=False):
        """The model (n entries; n*K, feature-major, for softmax)."""
        return get_x(self.h, self.n * self.K, polished)

    def state(self):
        """Full iteration state; with K > 1, x/u rows, z and s hold n*K entries
        (feature-major) and omega/nu are (m, K)."""
        N, n, m, K = self.N, self.n * self.K, self.m, self.K
        sc = get_state(self.h, FIELD_SCALARS, 3)
        om = get_state(self.h, FIELD_OMEGA, m * K)
        nu = get_state(self.h, FIELD_NU, m * K)
        if K > 1:
            om, nu = om.reshape(m, K), nu.reshape(m, K)
        return dict(x=get_state(self.h, FIELD_X, N * n).reshape(N, n),
                    u=get_state(self.h, FIELD_U, N * n).reshape(N, n),
                    z=get_state(self.h, FIELD_Z, n), s=get_state(self.h, FIELD_S, n),
                    omega=om, nu=nu, t=sc[0], v=sc[1], tau=sc[2])

    def block_inverses(self, blocks):
        """The setup's (rho_l A_ij'A_ij + c0 I)^-1 as a list (shards) of lists (blocks) of
        n_j x n_j arrays; `blocks` = the column ranges [(c0, c1), ...] of the M blocks."""
        sizes = [c1 - c0 for c0, c1 in blocks]
        flat = get_state(self.h, FIELD_P, self.N * sum(nj * nj for nj in sizes))
        out, o = [], 0
        for _ in range(self.N):
            row = []
            for nj in sizes:
                row.append(flat[o:o + nj * nj].reshape(nj, nj))
                o += nj * nj
            out.append(row)
        return out

    def close(self):
        if self.h:
            destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
