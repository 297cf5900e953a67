"""ctypes binding of include/pf.h (same names as the C ABI) and a small wrapper.

Argument marshalling only: every step of the filter runs in libpf_gb300.so's
CUDA kernels.  The library is built in-tree on first use if it is missing or
stale; if it cannot be built or loaded the import of any entry point raises,
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p
from typing import Optional, Sequence

import numpy as np

from . import build as _build
from . import workloads as W

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENUMERIC, PF_ETIMEOUT, PF_ESTATE, PF_EUNSUPPORTED = range(8)
STATUS_NAMES = ["PF_OK", "PF_EINVAL", "PF_ENOMEM", "PF_ECUDA", "PF_ENUMERIC", "PF_ETIMEOUT", "PF_ESTATE",
                "PF_EUNSUPPORTED"]
PF_STAT_MEAN, PF_STAT_LOG_EVIDENCE, PF_STAT_ESS, PF_STAT_LOG_Z, PF_STAT_FALLBACK = range(5)


class pf_model(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("dx", c_int32), ("J", c_int32), ("steps_per_obs", c_int32),
                ("params", POINTER(c_double)), ("n_params", c_int32)]


class pf_obs_op(ctypes.Structure):
    _fields_ = [("dy", c_int32), ("idx", POINTER(c_int32)), ("sigma_obs", c_double)]


class pf_noise(ctypes.Structure):
    _fields_ = [("sigma_dyn", c_double), ("x0_mean", POINTER(c_double)), ("sigma0", c_double), ("seed", c_uint64)]


class pf_stat(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("var", c_int32), ("per_filter", c_int32)]


PF_ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
PF_FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)

_SIGS = {
    "pf_version": (c_char_p, []),
    "pf_set_allocator": (c_int32, [PF_ALLOC_FN, PF_FREE_FN, c_void_p]),
    "pf_create": (c_int32, [POINTER(pf_model), c_int32, POINTER(c_int32), c_double, POINTER(pf_obs_op),
                            POINTER(pf_noise), POINTER(c_void_p)]),
    "pf_destroy": (None, [c_void_p]),
    "pf_last_error": (c_char_p, [c_void_p]),
    "pf_set_stream": (c_int32, [c_void_p, c_void_p]),
    "pf_step": (c_int32, [c_void_p, POINTER(c_float), c_int32]),
    "pf_step_device": (c_int32, [c_void_p, c_void_p, c_int32]),
    "pf_propagate": (c_int32, [c_void_p, POINTER(c_float), c_int32]),
    "pf_propagate_device": (c_int32, [c_void_p, c_void_p, c_int32]),
    "pf_resample": (c_int32, [c_void_p]),
    "pf_estimate": (c_int32, [c_void_p, POINTER(pf_stat), POINTER(c_double)]),
    "pf_get_time": (c_int32, [c_void_p, POINTER(c_int32)]),
    "pf_get_state": (c_int32, [c_void_p, POINTER(c_float)]),
    "pf_set_state": (c_int32, [c_void_p, POINTER(c_float), c_int32]),
    "pf_get_logw": (c_int32, [c_void_p, POINTER(c_float)]),
    "pf_set_logw": (c_int32, [c_void_p, POINTER(c_float)]),
    "pf_get_ancestors": (c_int32, [c_void_p, POINTER(c_int32)]),
    "pf_rng_philox": (c_int32, [c_int64, c_void_p, c_uint32, c_uint32, c_void_p, c_void_p]),
    "pf_rng_normals": (c_int32, [c_int64, c_void_p, c_uint64, c_void_p, c_void_p]),
    "pf_systematic_scratch_bytes": (c_size_t, [c_int32, c_int64]),
    "pf_systematic_resample": (c_int32, [c_int32, POINTER(c_int32), c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_size_t, c_void_p]),
    "pf_systematic_resample_noalloc": (c_int32, [c_int32, POINTER(c_int32), c_void_p, c_void_p, c_void_p,
                                                 c_void_p]),
    "pf_probe_bounded_wait": (c_int32, [c_int32, c_void_p]),
    "pf_set_schedule": (c_int32, [c_void_p, c_int32, c_int32, c_int32]),
    "pf_set_auxiliary": (c_int32, [c_void_p, c_int32]),
    "pf_estimate_async": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pf_estimate_wait": (c_int32, [c_void_p]),
    "pf_inject_error": (c_int32, [c_void_p, c_int32, c_int32]),
    "pf_step_timed": (c_int32, [c_void_p, c_void_p, c_int32, POINTER(c_float)]),
    "pf_ensemble_average": (c_int32, [c_int32, c_int32, POINTER(c_double), POINTER(c_double)]),
    "pf_step_kernels": (c_int32, [c_void_p, POINTER(c_int32)]),
    "pf_set_resampling": (c_int32, [c_void_p, c_double]),
    "pf_autotune": (c_int32, [c_void_p, POINTER(c_int32)]),
    "pf_set_proposal": (c_int32, [c_void_p, POINTER(c_float), c_int32, c_double]),
    "pf_set_proposal_span": (c_int32, [c_void_p, c_int32]),
    "pf_record_tuples": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32]),
    "pf_recorded_tuples": (c_int32, [c_void_p, POINTER(c_int64)]),
    "pf_proposal_forward": (c_int32, [c_int32, c_int64, c_void_p, c_int32, POINTER(c_int32), c_void_p, c_void_p,
                                      c_void_p, c_void_p]),
    "pf_mlp_forward": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_mlp_trainer_create": (c_int32, [POINTER(c_float), c_int32, c_int64, POINTER(c_void_p)]),
    "pf_mlp_train_step": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_float, POINTER(c_float),
                                    POINTER(c_double), c_void_p]),
    "pf_mlp_trainer_get": (c_int32, [c_void_p, POINTER(c_float)]),
    "pf_mlp_train_step_shuffled": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_int64, c_int64, c_uint64,
                                             c_float, POINTER(c_float), POINTER(c_double), c_void_p]),
    "pf_permutation": (c_int32, [c_int64, c_uint64, c_void_p, c_void_p]),
    "pf_mlp_trainer_destroy": (None, [c_void_p]),
    "pf_simulate": (c_int32, [POINTER(pf_model), c_double, POINTER(pf_obs_op), POINTER(pf_noise), c_int32, c_int32,
                              c_int32, POINTER(c_double), POINTER(c_float)]),
}

_lib = None


def lib():
    """Load libpf_gb300.so (building it in-tree first if needed)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols() -> list:
    return sorted(_SIGS)


class PFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _check(st: int, ctx=None):
    if st != PF_OK:
        raise PFError(st, (lib().pf_last_error(ctx) or b"").decode())


def _fp(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_float))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_int32))


# ---------------------------------------------------------------------------
# Thin wrappers with the C names
# ---------------------------------------------------------------------------
class _Structs:
    """Builds the pf_model / pf_obs_op / pf_noise structs of a ModelSpec and keeps their arrays alive."""

    def __init__(self, spec: W.ModelSpec, seed: int):
        self.params = np.ascontiguousarray(spec.params, dtype=np.float64)
        self.idx = np.ascontiguousarray(spec.obs_idx, dtype=np.int32)
        self.x0 = np.ascontiguousarray(spec.x0_mean, dtype=np.float64)
        self.model = pf_model(spec.kind, spec.dx, spec.J, spec.K, _dp(self.params), len(self.params))
        self.obs = pf_obs_op(len(self.idx), _ip(self.idx), spec.sigma_obs)
        self.noise = pf_noise(spec.sigma_dyn, _dp(self.x0), spec.sigma0, seed)


def pf_simulate(spec: W.ModelSpec, T: int, seed: int, record: int = 0):
    """Truth X_0..X_T (FP64) and observations (FP32) simulated on the GPU."""
    s = _Structs(spec, seed)
    x = np.empty((T + 1, spec.dx), dtype=np.float64)
    y = np.empty((T, spec.dy), dtype=np.float32)
    _check(lib().pf_simulate(ctypes.byref(s.model), spec.dt, ctypes.byref(s.obs), ctypes.byref(s.noise), T, record,
                             1 if spec.truth_init_random else 0, _dp(x), _fp(y)))
    return x, y


def pf_rng_philox(d_ctr, key0: int, key1: int, d_out, stream=None):
    n = d_ctr.shape[0]
    _check(lib().pf_rng_philox(n, d_ctr.data_ptr(), key0, key1, d_out.data_ptr(), stream))


def pf_rng_normals(d_ctr, seed: int, d_z, stream=None):
    n = d_ctr.shape[0]
    _check(lib().pf_rng_normals(n, d_ctr.data_ptr(), seed, d_z.data_ptr(), stream))


def pf_systematic_scratch_bytes(M: int, total: int) -> int:
    return int(lib().pf_systematic_scratch_bytes(M, total))


def pf_systematic_resample(N: Sequence[int], d_w, d_u, d_anc, d_scratch, stream=None):
    """Stateless systematic resampling of len(N) filters (device tensors)."""
    Nh = np.ascontiguousarray(N, dtype=np.int32)
    _check(lib().pf_systematic_resample(len(Nh), _ip(Nh), d_w.data_ptr(), d_u.data_ptr(), d_anc.data_ptr(),
                                        d_scratch.data_ptr(), d_scratch.numel() * d_scratch.element_size(), stream))


def pf_permutation(n: int, seed: int, d_perm, stream=None):
    """The library's keyed permutation of [0, n) into d_perm (n int64, device)."""
    _check(lib().pf_permutation(int(n), int(seed), d_perm.data_ptr(), stream))


def pf_ensemble_average(est) -> np.ndarray:
    """Definition 1's average of per-filter estimates (M x n_stat, host FP64):
    the exact sum over filters rounded once, divided by M (pf_ensemble_average)."""
    e = np.ascontiguousarray(est, dtype=np.float64)
    if e.ndim == 1:
        e = e[:, None]
    out = np.empty(e.shape[1], dtype=np.float64)
    _check(lib().pf_ensemble_average(e.shape[0], e.shape[1], _dp(e), _dp(out)))
    return out


def pf_systematic_resample_noalloc(N: Sequence[int], d_w, d_u, d_anc, stream=None):
    """Systematic resampling with the library's built-in scratch (no allocation)."""
    Nh = np.ascontiguousarray(N, dtype=np.int32)
    _check(lib().pf_systematic_resample_noalloc(len(Nh), _ip(Nh), d_w.data_ptr(), d_u.data_ptr(), d_anc.data_ptr(),
                                                stream))


def pf_probe_bounded_wait(arrive: bool, stream=None) -> int:
    """One bounded device wait on a barrier of the library's own (20 ms limit):
    the status it returns, PF_OK when the barrier was completed first,
    PF_ETIMEOUT when nothing completed it and the wait gave up."""
    return int(lib().pf_probe_bounded_wait(1 if arrive else 0, stream))


MLP_PARAMS = 23684


def pf_proposal_forward(J: int, d_x, obs_idx, d_y, d_theta, d_out, stream=None):
    """Network outputs for every (particle, observed node) of lattice states d_x
    (P x 2 J^2, device), rows built on the device; d_out: (P dy) x 4 FP32."""
    idx = np.ascontiguousarray(obs_idx, dtype=np.int32)
    _check(lib().pf_proposal_forward(int(J), d_x.shape[0], d_x.data_ptr(), len(idx), _ip(idx), d_y.data_ptr(),
                                     d_theta.data_ptr(), d_out.data_ptr(), stream))


def pf_mlp_forward(d_in, d_theta, d_out, stream=None):
    """Network forward of d_in (rows x 51 FP32, device) into d_out (rows x 4)."""
    _check(lib().pf_mlp_forward(d_in.shape[0], d_in.data_ptr(), d_theta.data_ptr(), d_out.data_ptr(), stream))


class MLPTrainer:
    """Adam training of the proposal network on the GPU (pf_mlp_trainer_*)."""

    def __init__(self, theta, max_batch: int):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == MLP_PARAMS
        h = c_void_p()
        _check(lib().pf_mlp_trainer_create(_fp(th), MLP_PARAMS, int(max_batch), ctypes.byref(h)))
        self.h = h

    def step(self, d_X, d_R, lr: float, want_grad: bool = False, want_loss: bool = True, stream=None):
        g = np.empty(MLP_PARAMS, dtype=np.float32) if want_grad else None
        loss = c_double(0.0)
        _check(lib().pf_mlp_train_step(self.h, d_X.shape[0], d_X.data_ptr(), d_R.data_ptr(), float(lr),
                                       _fp(g) if g is not None else POINTER(c_float)(),
                                       ctypes.byref(loss) if (want_loss or want_grad) else POINTER(c_double)(),
                                       stream))
        return loss.value, g

    def step_shuffled(self, d_X, d_R, batch: int, first: int, perm_seed: int, lr: float, want_grad: bool = False,
                      want_loss: bool = True, stream=None):
        """A step on rows pi(first .. first + batch - 1) of (d_X, d_R), pi = pf_permutation(n, perm_seed)."""
        g = np.empty(MLP_PARAMS, dtype=np.float32) if want_grad else None
        loss = c_double(0.0)
        _check(lib().pf_mlp_train_step_shuffled(self.h, d_X.shape[0], d_X.data_ptr(), d_R.data_ptr(), int(batch),
                                                int(first), int(perm_seed), float(lr),
                                                _fp(g) if g is not None else POINTER(c_float)(),
                                                ctypes.byref(loss) if (want_loss or want_grad) else POINTER(c_double)(),
                                                stream))
        return loss.value, g

    def theta(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(lib().pf_mlp_trainer_get(self.h, _fp(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().pf_mlp_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# torch caching allocator as the context allocator
# ---------------------------------------------------------------------------
_torch_hooks = None


def use_torch_allocator(enable: bool = True):
    """Route context device memory through torch's caching allocator."""
    global _torch_hooks
    if not enable:
        _check(lib().pf_set_allocator(PF_ALLOC_FN(), PF_FREE_FN(), None))
        _torch_hooks = None
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (PF_ALLOC_FN(_alloc), PF_FREE_FN(_free))
    _check(lib().pf_set_allocator(hooks[0], hooks[1], None))
    _torch_hooks = hooks


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
class _PendingEstimate:
    def __init__(self, f, buf, matrix):
        self.f, self.buf, self.matrix = f, buf, matrix

    def wait(self):
        _check(lib().pf_estimate_wait(self.f.h), self.f.h)
        out = self.buf.numpy().copy()
        return out.reshape(self.f.M, self.f.spec.dx) if self.matrix else out


class EnsembleFilter:
    """M independent bootstrap filters on the GPU (Sec. 3.1) behind the C ABI."""

    def __init__(self, spec: W.ModelSpec, M: int, N, seed: int):
        self.spec = spec
        self.M = int(M)
        self.N = np.ascontiguousarray(np.broadcast_to(np.asarray(N, dtype=np.int32), (self.M,)), dtype=np.int32)
        self.P = int(self.N.sum())
        self._s = _Structs(spec, seed)
        h = c_void_p()
        st = lib().pf_create(ctypes.byref(self._s.model), self.M, _ip(self.N), spec.dt, ctypes.byref(self._s.obs),
                             ctypes.byref(self._s.noise), ctypes.byref(h))
        _check(st)
        self.h = h

    # -- life cycle
    def close(self):
        if getattr(self, "h", None):
            lib().pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream_handle: Optional[int]):
        _check(lib().pf_set_stream(self.h, stream_handle), self.h)

    # -- hot path
    @staticmethod
    def _obs(y):
        return np.ascontiguousarray(y, dtype=np.float32)

    def step(self, y, per_filter: bool = False):
        y = self._obs(y)
        _check(lib().pf_step(self.h, _fp(y), self.spec.dy if per_filter else 0), self.h)

    def step_device(self, d_y, per_filter: bool = False):
        _check(lib().pf_step_device(self.h, d_y.data_ptr(), self.spec.dy if per_filter else 0), self.h)

    def step_timed(self, d_y, per_filter: bool = False):
        """A step without its graph, timed by halves: (propagation ms, resampling ms)."""
        ms = (c_float * 2)()
        _check(lib().pf_step_timed(self.h, d_y.data_ptr(), self.spec.dy if per_filter else 0, ms), self.h)
        return float(ms[0]), float(ms[1])

    def propagate(self, y, per_filter: bool = False):
        y = self._obs(y)
        _check(lib().pf_propagate(self.h, _fp(y), self.spec.dy if per_filter else 0), self.h)

    def propagate_device(self, d_y, per_filter: bool = False):
        _check(lib().pf_propagate_device(self.h, d_y.data_ptr(), self.spec.dy if per_filter else 0), self.h)

    def resample(self):
        _check(lib().pf_resample(self.h), self.h)

    def estimate(self, kind: int = PF_STAT_MEAN, var: int = -1, per_filter: bool = False) -> np.ndarray:
        n = 1
        if kind == PF_STAT_MEAN and var < 0:
            n = self.spec.dx
        if per_filter:
            n *= self.M
        out = np.empty(n, dtype=np.float64)
        st = pf_stat(kind, var, 1 if per_filter else 0)
        _check(lib().pf_estimate(self.h, ctypes.byref(st), _dp(out)), self.h)
        if per_filter and kind == PF_STAT_MEAN and var < 0:
            return out.reshape(self.M, self.spec.dx)
        return out

    def estimate_async(self, kind: int = PF_STAT_MEAN, var: int = -1, per_filter: bool = False):
        """Enqueue the copy of a statistic into pinned host memory without waiting
        (pf_estimate_async); the returned handle's wait() blocks until that copy
        alone is done (pf_estimate_wait) and gives the values.  Only the latest
        handle of a filter may be waited on."""
        import torch
        n = self.spec.dx if kind == PF_STAT_MEAN and var < 0 else 1
        if per_filter:
            n *= self.M
        buf = torch.empty(n, dtype=torch.float64, pin_memory=True)
        st = pf_stat(kind, var, 1 if per_filter else 0)
        _check(lib().pf_estimate_async(self.h, ctypes.byref(st), buf.data_ptr()), self.h)
        return _PendingEstimate(self, buf, per_filter and kind == PF_STAT_MEAN and var < 0)

    def inject_error(self, code: int, filter: int = 0):
        """Host-side failure injection (pf_inject_error): the next estimate reports `code`."""
        _check(lib().pf_inject_error(self.h, int(code), int(filter)), self.h)

    def step_kernels(self) -> int:
        """Kernels one step launches (kernel nodes of the captured step graph)."""
        n = c_int32(0)
        _check(lib().pf_step_kernels(self.h, ctypes.byref(n)), self.h)
        return n.value

    # -- inspection
    @property
    def t(self) -> int:
        v = c_int32()
        _check(lib().pf_get_time(self.h, ctypes.byref(v)), self.h)
        return v.value

    def get_state(self) -> np.ndarray:
        x = np.empty((self.P, self.spec.dx), dtype=np.float32)
        _check(lib().pf_get_state(self.h, _fp(x)), self.h)
        return x

    def set_state(self, x, t: int):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(self.P, self.spec.dx)
        _check(lib().pf_set_state(self.h, _fp(x), int(t)), self.h)

    def get_logw(self) -> np.ndarray:
        l = np.empty(self.P, dtype=np.float32)
        _check(lib().pf_get_logw(self.h, _fp(l)), self.h)
        return l

    def set_logw(self, l):
        l = np.ascontiguousarray(l, dtype=np.float32)
        _check(lib().pf_set_logw(self.h, _fp(l)), self.h)

    def get_ancestors(self) -> np.ndarray:
        a = np.empty(self.P, dtype=np.int32)
        _check(lib().pf_get_ancestors(self.h, _ip(a)), self.h)
        return a

    def autotune(self):
        """Pick the launch schedule by timing (cached per shape); returns (particles per lattice CTA,
        resample threads, lattice nodes per thread)."""
        ch = (c_int32 * 3)()
        _check(lib().pf_autotune(self.h, ch), self.h)
        return int(ch[0]), int(ch[1]), int(ch[2])

    def set_auxiliary(self, on: bool = True):
        """Auxiliary particle filters (Pitt & Shephard) instead of bootstrap filters."""
        _check(lib().pf_set_auxiliary(self.h, 1 if on else 0), self.h)

    def set_resampling(self, ess_threshold: float = -1.0):
        """Resample a filter only when its ESS < ess_threshold N (0..1); other values: every step."""
        _check(lib().pf_set_resampling(self.h, float(ess_threshold)), self.h)

    def set_schedule(self, nodes_per_thread: int = 0, particles_per_cta: int = 0, resample_threads: int = 0):
        """Set the launch schedule explicitly (0: default)."""
        _check(lib().pf_set_schedule(self.h, nodes_per_thread, particles_per_cta, resample_threads), self.h)

    def set_proposal(self, theta, ess_frac: float = 0.1):
        """Learned proposal on (theta: PF_MLP_PARAMS values) or off (None)."""
        if theta is None:
            _check(lib().pf_set_proposal(self.h, POINTER(c_float)(), 0, 0.0), self.h)
            return
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().pf_set_proposal(self.h, _fp(th), th.size, float(ess_frac)), self.h)

    def set_proposal_span(self, span: int = 1):
        """The learned proposal acts on the last `span` sub-steps of each interval (1: the last one)."""
        _check(lib().pf_set_proposal_span(self.h, int(span)), self.h)

    def record_tuples(self, d_X, d_R, stride: int = 1):
        """Record (inputs, standardised residual) training tuples into device tensors (None stops)."""
        if d_X is None:
            _check(lib().pf_record_tuples(self.h, None, None, 0, 1), self.h)
            return
        _check(lib().pf_record_tuples(self.h, d_X.data_ptr(), d_R.data_ptr(), d_X.shape[0], int(stride)), self.h)

    def recorded_tuples(self) -> int:
        n = c_int64()
        _check(lib().pf_recorded_tuples(self.h, ctypes.byref(n)), self.h)
        return n.value

    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N)]).astype(np.int64)
