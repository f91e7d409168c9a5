"""Python binding of libbo_suggest.so (ctypes; argument marshalling only).

Every step of the suggest path runs in the library's CUDA kernels.  PyTorch
provides the device memory (its caching allocator, through the library's
allocation callback) and the stream.  There is no CPU fallback: if the
library cannot be loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbo_suggest.so")

BO_OK = 0
ERRORS = {1: "BO_ERR_ARG", 2: "BO_ERR_INDEX", 3: "BO_ERR_DUPLICATE", 4: "BO_ERR_EXHAUSTED",
          5: "BO_ERR_NUMERIC", 6: "BO_ERR_NOMEM", 7: "BO_ERR_CUDA", 8: "BO_ERR_TIMEOUT",
          9: "BO_ERR_NOT_POSITIVE", 10: "BO_ERR_STATE", 11: "BO_ERR_CAPACITY"}
AF = {"ei": 0, "poi": 1, "pi": 1, "lcb": 2, "multi": 3, "advanced_multi": 4}
AF_NAMES = {0: "ei", 1: "poi", 2: "lcb", -1: None}
PRECISION = {"fp64": 0, "fp16x3": 1, "bf16x3": 2, "tf32": 3, "tf32x3": 4}
INIT = {"random": 0, "lhs": 1, "maximin": 2}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class BOError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SpaceDesc(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_values", C.POINTER(C.c_int32)),
                ("values", C.POINTER(C.POINTER(C.c_double))), ("invalid_mask", C.POINTER(C.c_uint8)),
                ("nu", C.c_double), ("lengthscale", C.c_double), ("jitter", C.c_double),
                ("af", C.c_int32), ("explore", C.c_int32), ("lambda_const", C.c_double),
                ("skip_threshold", C.c_int32), ("rif", C.c_double), ("discount", C.c_double),
                ("y_norm", C.c_int32), ("precision", C.c_int32), ("n_max", C.c_int32),
                ("n_init", C.c_int32), ("seed", C.c_uint64), ("init_mode", C.c_int32),
                ("init_designs", C.c_int32), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_ctx", C.c_void_p), ("stream", C.c_void_p)]


class SuggestInfo(C.Structure):
    _fields_ = [("idx", C.c_int64), ("af", C.c_int32), ("predicted", C.c_int32),
                ("mu", C.c_double), ("sigma", C.c_double), ("score", C.c_double),
                ("lam", C.c_double), ("mean_var", C.c_double), ("n_scored", C.c_int64)]


class PassResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_fit", C.c_int32), ("n_scored", C.c_int64),
                ("sum_var", C.c_double), ("mean_var", C.c_double), ("lam", C.c_double),
                ("mean_var_s", C.c_double), ("top_idx", (C.c_int64 * 3) * 3),
                ("top_score", (C.c_double * 3) * 3), ("top_mu", (C.c_double * 3) * 3),
                ("top_sigma", (C.c_double * 3) * 3)]


class AcqParams(C.Structure):
    _fields_ = [("n_cand", C.c_int64), ("n_unvisited", C.c_int64), ("sum_var", C.c_double),
                ("n_af", C.c_int32), ("af", C.c_int32 * 3), ("explore", C.c_int32),
                ("n_fit", C.c_int32), ("lambda_const", C.c_double), ("fplus", C.c_double),
                ("fplus_raw", C.c_double), ("mu_s_raw", C.c_double), ("mean_var_s", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("stages_a", C.c_int32), ("b_slots", C.c_int32), ("b_resident", C.c_int32),
                ("tried", C.c_int32), ("best_ms", C.c_double), ("default_ms", C.c_double)]


def _tune_dict(r):
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("max_sessions", C.c_int32), ("pad", C.c_int32),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("session", C.c_int64), ("status", C.c_int32),
                ("observed", C.c_int32), ("idx", C.c_int64), ("info", SuggestInfo),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("admitted", C.c_int64), ("queued", C.c_int64), ("rejected", C.c_int64),
                ("closed", C.c_int64), ("requests", C.c_int64), ("completed", C.c_int64),
                ("iterations", C.c_int64), ("candidates_scored", C.c_int64),
                ("bytes_in_use", C.c_int64)]


class AluPeaks(C.Structure):
    _fields_ = [("fp64_fma_tflops", C.c_double), ("fp32_fma_tflops", C.c_double),
                ("fp32x2_fma_tflops", C.c_double), ("mufu_gops", C.c_double), ("sms", C.c_int32),
                ("pad", C.c_int32)]


# every symbol include/bo_suggest.h declares, with (restype, argtypes)
SIGNATURES = {
    "bo_space_desc_init": (None, [C.POINTER(SpaceDesc)]),
    "bo_initial_design": (C.c_int, [C.POINTER(SpaceDesc), C.c_int32, C.c_void_p]),
    "bo_space_create": (C.c_int, [C.POINTER(SpaceDesc), C.POINTER(C.c_void_p)]),
    "bo_space_destroy": (C.c_int, [C.c_void_p]),
    "bo_valid_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "bo_decode": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32)]),
    "bo_observe": (C.c_int, [C.c_void_p, C.c_int64, C.c_double]),
    "bo_suggest": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(SuggestInfo)]),
    "bo_predict": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]),
    "bo_predict_enqueue": (C.c_int, [C.c_void_p]),
    "bo_last_posterior": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]),
    "bo_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "bo_batch_destroy": (C.c_int, [C.c_void_p]),
    "bo_batch_observe": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bo_batch_suggest": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SuggestInfo)]),
    "bo_batch_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "bo_batch_suggest_some": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.POINTER(SuggestInfo)]),
    "bo_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(TuneResult)]),
    "bo_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(TuneResult)]),
    "bo_tuned_shape": (C.c_int, [C.c_void_p, C.POINTER(TuneResult)]),
    "bo_measure_alu_peaks": (C.c_int, [C.POINTER(AluPeaks)]),
    "bo_server_create": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]),
    "bo_server_open": (C.c_int, [C.c_void_p, C.POINTER(SpaceDesc), C.POINTER(C.c_int64)]),
    "bo_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.c_int32, C.c_uint64]),
    "bo_server_poll": (C.c_int, [C.c_void_p, C.POINTER(Completion), C.c_int32, C.POINTER(C.c_int32),
                                 C.c_int32]),
    "bo_server_close": (C.c_int, [C.c_void_p, C.c_int64]),
    "bo_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "bo_server_now": (C.c_double, [C.c_void_p]),
    "bo_server_destroy": (C.c_int, [C.c_void_p]),
    "bo_get_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "bo_sync": (C.c_int, [C.c_void_p]),
    "bo_replay_enqueue": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "bo_replay_fetch": (C.c_int, [C.c_void_p, C.POINTER(PassResult), C.c_int32]),
    "bo_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "bo_selftest_waits": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "bo_selftest_exp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "bo_acquire_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.POINTER(AcqParams), C.c_void_p, C.c_void_p]),
    "bo_last_error": (C.c_char_p, []),
}

_LIB = None


def lib():
    """Load libbo_suggest.so (built by paper_2111_14991_gb300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2111_14991_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(rc):
    if rc != BO_OK:
        raise BOError(rc, lib().bo_last_error().decode())


def _torch_allocator():
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:   # reported to the library as an allocation failure
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free)


def _as_ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def make_desc(grids, invalid_mask=None, *, nu=1.5, lengthscale=1.5, jitter=1e-10, af="ei",
              explore="cv", lambda_const=0.01, skip_threshold=5, rif=0.1, discount=None,
              normalize_y=True, precision="fp64", n_max=512, n_init=0, seed=0, init="maximin",
              init_designs=100):
    """A bo_space_desc for these arguments, and the arrays it points into."""
    grids = [np.ascontiguousarray(g, dtype=np.float64) for g in grids]
    d = len(grids)
    sizes = np.array([len(g) for g in grids], dtype=np.int32)
    vals = (C.POINTER(C.c_double) * d)(*[_as_ptr(g, C.c_double) for g in grids])
    desc = SpaceDesc()
    lib().bo_space_desc_init(C.byref(desc))
    desc.d = d
    desc.n_values = _as_ptr(sizes, C.c_int32)
    desc.values = vals
    mask = None
    if invalid_mask is not None:
        mask = np.ascontiguousarray(np.asarray(invalid_mask).reshape(-1), dtype=np.uint8)
        desc.invalid_mask = _as_ptr(mask, C.c_uint8)
    desc.nu, desc.lengthscale, desc.jitter = nu, lengthscale, jitter
    desc.af = AF[af]
    desc.explore = 0 if explore == "cv" else 1
    desc.lambda_const = lambda_const
    desc.skip_threshold = skip_threshold
    desc.rif = rif
    desc.discount = 0.0 if discount is None else discount
    desc.y_norm = 0 if normalize_y else 1
    desc.precision = PRECISION[precision]
    desc.n_max = n_max
    desc.n_init = n_init
    desc.seed = seed
    desc.init_mode = INIT[init]
    desc.init_designs = init_designs
    return desc, (grids, sizes, vals, mask)


def initial_design(grids, invalid_mask=None, count=20, *, init="maximin", init_designs=100, seed=0):
    """The initial sample (valid-list indices) a space with these arguments
    draws; host computation, no device needed."""
    desc, keep = make_desc(grids, invalid_mask, init=init, init_designs=init_designs, seed=seed)
    out = np.zeros(count, dtype=np.int64)
    _check(lib().bo_initial_design(C.byref(desc), count, out.ctypes.data))
    del keep
    return out


class Space:
    """One BO session on a discrete, normalized, constrained search space."""

    def __init__(self, grids, invalid_mask=None, *, precision="fp64", stream=None, torch_allocator=True,
                 **params):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the suggest library has no CPU path")
        L = lib()
        desc, self._keep = make_desc(grids, invalid_mask, precision=precision, **params)
        self.d = desc.d
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        desc.stream = C.c_void_p(stream.cuda_stream)
        if torch_allocator:
            self._alloc_cbs = _torch_allocator()
            desc.alloc, desc.free = self._alloc_cbs
        handle = C.c_void_p()
        _check(L.bo_space_create(C.byref(desc), C.byref(handle)))
        self._h = handle
        n = C.c_int64()
        _check(L.bo_valid_count(self._h, C.byref(n)))
        self.N = n.value
        self.precision = precision

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _check(lib().bo_space_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -----------------------------------------------------------------
    def decode(self, idx):
        out = (C.c_int32 * self.d)()
        _check(lib().bo_decode(self._h, int(idx), out))
        return list(out)

    def observe(self, idx, value):
        _check(lib().bo_observe(self._h, int(idx), float(value)))

    def suggest(self):
        idx = C.c_int64()
        info = SuggestInfo()
        _check(lib().bo_suggest(self._h, C.byref(idx), C.byref(info)))
        return _info_dict(info)

    def predict(self, begin=0, count=None):
        count = self.N - begin if count is None else count
        mu = np.empty(count, dtype=np.float64)
        var = np.empty(count, dtype=np.float64)
        _check(lib().bo_predict(self._h, begin, count, mu.ctypes.data, var.ctypes.data))
        return mu, var

    def last_posterior(self, begin=0, count=None):
        count = self.N - begin if count is None else count
        mu = np.empty(count, dtype=np.float64)
        var = np.empty(count, dtype=np.float64)
        _check(lib().bo_last_posterior(self._h, begin, count, mu.ctypes.data, var.ctypes.data))
        return mu, var

    def autotune(self, reps=3):
        r = TuneResult()
        _check(lib().bo_autotune(self._h, int(reps), C.byref(r)))
        return _tune_dict(r)

    def tuned_shape(self):
        """The autotuner's stored shape for this space's next launch key, or None."""
        r = TuneResult()
        rc = lib().bo_tuned_shape(self._h, C.byref(r))
        if rc == 10:                     # BO_ERR_STATE: nothing stored for the key
            return None
        _check(rc)
        return _tune_dict(r)

    def predict_enqueue(self):
        _check(lib().bo_predict_enqueue(self._h))

    def factor(self):
        n = C.c_int32()
        _check(lib().bo_get_factor(self._h, None, None, C.byref(n)))
        linv = np.zeros((n.value, n.value))
        beta = np.zeros(n.value)
        if n.value:
            _check(lib().bo_get_factor(self._h, linv.ctypes.data, beta.ctypes.data, C.byref(n)))
        return linv, beta

    def sync(self):
        _check(lib().bo_sync(self._h))

    def replay_enqueue(self, idx, y):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        _check(lib().bo_replay_enqueue(self._h, idx.ctypes.data, y.ctypes.data, len(idx)))
        return len(idx)

    def replay_fetch(self, steps):
        out = (PassResult * steps)()
        _check(lib().bo_replay_fetch(self._h, out, steps))
        return [pass_result_dict(r) for r in out]

    def launch_count(self):
        n = C.c_int64()
        _check(lib().bo_launch_count(self._h, C.byref(n)))
        return n.value


def _info_dict(info):
    return dict(idx=info.idx, af=AF_NAMES.get(info.af), predicted=bool(info.predicted), mu=info.mu,
                sigma=info.sigma, score=info.score, lam=info.lam, mean_var=info.mean_var,
                n_scored=info.n_scored)


class Batch:
    """Spaces observed and suggested together (one launch per phase for all)."""

    def __init__(self, spaces):
        self.spaces = list(spaces)
        arr = (C.c_void_p * len(self.spaces))(*[s._h for s in self.spaces])
        h = C.c_void_p()
        _check(lib().bo_batch_create(arr, len(self.spaces), C.byref(h)))
        self._h = h

    def observe(self, idx, values):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        values = np.ascontiguousarray(values, dtype=np.float64)
        status = np.zeros(len(self.spaces), dtype=np.int32)
        rc = lib().bo_batch_observe(self._h, idx.ctypes.data, values.ctypes.data, status.ctypes.data)
        if rc != BO_OK and not status.any():
            _check(rc)
        return status

    def suggest(self):
        n = len(self.spaces)
        idx = np.zeros(n, dtype=np.int64)
        status = np.zeros(n, dtype=np.int32)
        infos = (SuggestInfo * n)()
        rc = lib().bo_batch_suggest(self._h, idx.ctypes.data, status.ctypes.data, infos)
        if rc != BO_OK and not status.any():
            _check(rc)
        return idx, status, [_info_dict(i) for i in infos]

    def launch_count(self):
        n = C.c_int64()
        _check(lib().bo_batch_launch_count(self._h, C.byref(n)))
        return n.value

    def autotune(self, reps=3):
        r = TuneResult()
        _check(lib().bo_batch_autotune(self._h, int(reps), C.byref(r)))
        return _tune_dict(r)

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().bo_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over many sessions (native worker thread)."""

    def __init__(self, budget_bytes, max_sessions=1024, stream=None, torch_allocator=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the suggest library has no CPU path")
        cfg = ServerConfig()
        cfg.budget_bytes = int(budget_bytes)
        cfg.max_sessions = int(max_sessions)
        stream = torch.cuda.current_stream() if stream is None else stream
        self._stream = stream
        cfg.stream = C.c_void_p(stream.cuda_stream)
        if torch_allocator:
            self._alloc_cbs = _torch_allocator()
            cfg.alloc, cfg.free = self._alloc_cbs
        h = C.c_void_p()
        _check(lib().bo_server_create(C.byref(cfg), C.byref(h)))
        self._h = h

    def open(self, grids, invalid_mask=None, **params):
        desc, keep = make_desc(grids, invalid_mask, **params)
        sid = C.c_int64()
        _check(lib().bo_server_open(self._h, C.byref(desc), C.byref(sid)))
        del keep
        return sid.value

    def submit(self, session, observe_idx=-1, observe_value=0.0, tag=0, suggest=True):
        _check(lib().bo_server_submit(self._h, int(session), int(observe_idx), float(observe_value),
                                      1 if suggest else 0, int(tag)))

    def poll(self, max_n=1024, wait_ms=0):
        out = (Completion * max_n)()
        n = C.c_int32()
        _check(lib().bo_server_poll(self._h, out, max_n, C.byref(n), int(wait_ms)))
        return [dict(tag=c.tag, session=c.session, status=c.status, observed=bool(c.observed), idx=c.idx,
                     info=_info_dict(c.info), t_submit=c.t_submit, t_start=c.t_start, t_done=c.t_done)
                for c in out[:n.value]]

    def close_session(self, session):
        _check(lib().bo_server_close(self._h, int(session)))

    def stats(self):
        st = ServerStats()
        _check(lib().bo_server_stats_get(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def now(self):
        return lib().bo_server_now(self._h)

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().bo_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_waits():
    """bo_selftest_waits: (mbarrier wait status, grid barrier status), each
    BO_ERR_TIMEOUT when the bounded waits work (see include/bo_suggest.h)."""
    a, b = C.c_int32(), C.c_int32()
    _check(lib().bo_selftest_waits(C.byref(a), C.byref(b)))
    return a.value, b.value


def selftest_exp(t):
    """bo_selftest_exp: (the FP64 pass's e^-t, CUDA's exp(-t)) for the float64
    array t, computed on the current device (see include/bo_suggest.h)."""
    import numpy as np
    t = np.ascontiguousarray(t, dtype=np.float64)
    out, ref = np.empty_like(t), np.empty_like(t)
    _check(lib().bo_selftest_exp(t.ctypes.data, out.ctypes.data, ref.ctypes.data, int(t.size)))
    return out, ref


def acquire_noalloc(mu_ptr, var_ptr, visited_ptr, f64, params, result_ptr, stream_ptr):
    """bo_acquire_noalloc on caller-owned device pointers (see include/bo_suggest.h)."""
    _check(lib().bo_acquire_noalloc(C.c_void_p(mu_ptr), C.c_void_p(var_ptr), C.c_void_p(visited_ptr),
                                    int(f64), C.byref(params), C.c_void_p(result_ptr),
                                    C.c_void_p(stream_ptr)))


def pass_result_dict(r):
    return dict(status=r.status, n_fit=r.n_fit, n_scored=r.n_scored, sum_var=r.sum_var,
                mean_var=r.mean_var, lam=r.lam, mean_var_s=r.mean_var_s,
                top_idx=[[r.top_idx[q][k] for k in range(3)] for q in range(3)],
                top_score=[[r.top_score[q][k] for k in range(3)] for q in range(3)],
                top_mu=[[r.top_mu[q][k] for k in range(3)] for q in range(3)],
                top_sigma=[[r.top_sigma[q][k] for k in range(3)] for q in range(3)])


def measure_alu_peaks():
    """bo_measure_alu_peaks on the current device: FP64 / FP32 / f32x2 FMA rates
    (TFLOP/s) and the MUFU rate (Gop/s) of the units the prediction passes use."""
    r = AluPeaks()
    _check(lib().bo_measure_alu_peaks(C.byref(r)))
    return {f: getattr(r, f) for f, _ in AluPeaks._fields_ if f != "pad"}
