"""ctypes binding of the C ABI in include/snn.h (argument marshalling only).

Every step of the simulation runs in the CUDA library libsnn.so; this module
converts Python/numpy arguments, checks return codes and raises SnnError.
There is no CPU path: if the library cannot be built or loaded, or no GPU is
present, the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# ---------------------------------------------------------------------------
# ABI structures (mirror include/snn.h field by field)
# ---------------------------------------------------------------------------
STDP_OFF = 1
DELIVERY_OFF = 2
FP64 = 4

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ETIMEOUT, ETRUNC, ESTATE, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7, -8
SNN_NOALLOC_MAX_SYNAPSES = 1 << 20   # staging size of snn_read_synapses_noalloc


class SnnConfig(ctypes.Structure):
    _fields_ = [
        ("grid_x", ctypes.c_uint32), ("grid_y", ctypes.c_uint32),
        ("neurons_per_col", ctypes.c_uint32), ("exc_per_col", ctypes.c_uint32),
        ("fanout", ctypes.c_uint32),
        ("pct_ring", ctypes.c_uint32 * 4),
        ("max_delay_ms", ctypes.c_uint32),
        ("w_exc0_q16", ctypes.c_int32), ("w_inh0_q16", ctypes.c_int32),
        ("wmax_q16", ctypes.c_int32),
        ("a_plus_mv", ctypes.c_double), ("a_minus_mv", ctypes.c_double),
        ("tau_plus_ms", ctypes.c_double), ("tau_minus_ms", ctypes.c_double),
        ("deriv_period_ms", ctypes.c_uint32),
        ("deriv_bias_q16", ctypes.c_int32), ("deriv_decay_q16", ctypes.c_int32),
        ("thal_per_col_per_ms", ctypes.c_uint32),
        ("thal_amp_q16", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("raster_capacity", ctypes.c_uint64),
    ]


class SnnSpike(ctypes.Structure):
    _fields_ = [("t_ms", ctypes.c_int32), ("gid", ctypes.c_int32)]


class SnnStimulus(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int32), ("gid", ctypes.c_int32), ("q16", ctypes.c_int32)]


class SnnCounters(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64), ("spikes", ctypes.c_int64), ("e_all", ctypes.c_int64),
                ("e_exc", ctypes.c_int64), ("l_exc", ctypes.c_int64), ("raster_kept", ctypes.c_int64),
                ("raster_dropped", ctypes.c_int64), ("error", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SnnLaunch(ctypes.Structure):
    _fields_ = [("deliver_block", ctypes.c_uint32), ("deliver_blocks_per_sm", ctypes.c_uint32),
                ("neuron_block", ctypes.c_uint32), ("ltp_block", ctypes.c_uint32),
                ("ltp_blocks_per_sm", ctypes.c_uint32), ("deriv_block", ctypes.c_uint32),
                ("graph_steps", ctypes.c_uint32), ("dense_block", ctypes.c_uint32),
                ("dense_rows", ctypes.c_uint32), ("dense_permille", ctypes.c_uint32),
                ("staged_permille", ctypes.c_uint32), ("ring_permille", ctypes.c_uint32)]


class SnnProfile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 5), ("ms", ctypes.c_double * 5),
                ("dense_steps", ctypes.c_int64), ("dense_deriv_steps", ctypes.c_int64),
                ("dense_events", ctypes.c_int64), ("dense_exc_events", ctypes.c_int64),
                ("dense_ltp_visits", ctypes.c_int64), ("kernels", ctypes.c_int64)]


class SnnAtomicRates(ctypes.Structure):
    _fields_ = [("red_global_random_gops", ctypes.c_double), ("red_global_window_gops", ctypes.c_double),
                ("red_global_coalesced_gops", ctypes.c_double), ("ld_global_random_gops", ctypes.c_double),
                ("atom_shared_window_gops", ctypes.c_double), ("array_bytes", ctypes.c_double),
                ("threads", ctypes.c_double)]


SPIKE_DTYPE = np.dtype([("t", np.int32), ("gid", np.int32)])
STIM_DTYPE = np.dtype([("t", np.int32), ("gid", np.int32), ("q16", np.int32)])
KERNELS = ("deliver", "neuron", "ltp", "deriv", "dense")

# every function the header declares, with its ctypes signature
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_SIGS = {
    "snn_build_network": (ctypes.c_int, [_P(SnnConfig), _vp, ctypes.c_size_t, _P(_vp)]),
    "snn_build_network_explicit": (ctypes.c_int, [_P(SnnConfig), _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                                  _P(_vp)]),
    "snn_set_stimulus": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "snn_set_thalamic": (ctypes.c_int, [_vp, ctypes.c_int]),
    "snn_set_launch": (ctypes.c_int, [_vp, _P(SnnLaunch)]),
    "snn_get_launch": (ctypes.c_int, [_vp, _P(SnnLaunch)]),
    "snn_step": (ctypes.c_int, [_vp]),
    "snn_run": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "snn_run_host": (ctypes.c_int, [_vp, ctypes.c_uint32, _vp, ctypes.c_size_t, _vp, ctypes.c_size_t,
                                    _P(ctypes.c_size_t)]),
    "snn_read_raster": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_size_t,
                                       _P(ctypes.c_size_t)]),
    "snn_raster_reset": (ctypes.c_int, [_vp]),
    "snn_read_synapses": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, _vp, _vp,
                                         ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "snn_read_synapses_noalloc": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, _vp, _vp,
                                                 ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "snn_read_weights": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "snn_read_neurons": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp]),
    "snn_read_counters": (ctypes.c_int, [_vp, _P(SnnCounters)]),
    "snn_read_neurons_f64": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp]),
    "snn_set_probe": (ctypes.c_int, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint32]),
    "snn_read_probe": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _P(ctypes.c_uint32)]),
    "snn_net_info": (ctypes.c_int, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_int64), _P(ctypes.c_size_t)]),
    "snn_set_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "snn_read_profile": (ctypes.c_int, [_vp, _P(SnnProfile)]),
    "snn_save_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _P(ctypes.c_size_t)]),
    "snn_load_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "snn_reset": (ctypes.c_int, [_vp]),
    "snn_autotune": (ctypes.c_int, [_vp, ctypes.c_uint32, _P(SnnLaunch)]),
    "snn_batch_create": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _P(_vp)]),
    "snn_batch_run": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "snn_batch_free": (None, [_vp]),
    "snn_batch_set_launch": (ctypes.c_int, [_vp, _P(SnnLaunch)]),
    "snn_batch_get_launch": (ctypes.c_int, [_vp, _P(SnnLaunch)]),
    "snn_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_uint32, _P(SnnLaunch)]),
    "snn_thalamic_events": (ctypes.c_int, [_P(SnnConfig), ctypes.c_int32, ctypes.c_uint32, _vp, ctypes.c_size_t,
                                           _P(ctypes.c_size_t)]),
    "snn_microbench_atomics": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_uint32, _vp, _P(SnnAtomicRates)]),
    "snn_set_tile": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
    "snn_inject_spikes": (ctypes.c_int, [_vp, _vp, ctypes.c_uint32]),
    "snn_free": (None, [_vp]),
    "snn_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "snn_last_error": (ctypes.c_char_p, []),
    "snn_set_allocator": (None, [_vp, _vp, _vp]),
}

_lib = None


def checked() -> bool:
    """SNN_CHECKED=1 in the environment selects the checked build."""
    return os.environ.get("SNN_CHECKED", "") == "1"


def library_path() -> str:
    return _build.CHECKED_LIB_PATH if checked() else _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libsnn.so, or libsnn_checked.so under SNN_CHECKED=1 (building it
    first if needed); raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("CUDA engine library missing: %s (run build())" % path)
        _build.build(checked=checked())
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SnnError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = load()
        msg = "%s: %s (%s)" % (what, lib.snn_strerror(code).decode(), lib.snn_last_error().decode())
        super().__init__(msg)
        self.code = code


def _check(code: int, what: str):
    if code != OK:
        raise SnnError(code, what)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_config(cfg: dict, raster_capacity: int | None = None) -> SnnConfig:
    c = SnnConfig()
    for name, _ in SnnConfig._fields_:
        if name == "pct_ring":
            for i, p in enumerate(cfg["pct_ring"]):
                c.pct_ring[i] = int(p)
        elif name == "reserved":
            c.reserved = 0
        elif name == "raster_capacity":
            c.raster_capacity = int(raster_capacity if raster_capacity is not None
                                    else cfg.get("raster_capacity", 0))
        else:
            setattr(c, name, cfg[name])
    return c


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))


# ---------------------------------------------------------------------------
# C-ABI mirrors (same names as include/snn.h)
# ---------------------------------------------------------------------------
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None          # the installed callbacks, kept alive while in use


def set_allocator(alloc=None, free=None):
    """snn_set_allocator with Python callables: alloc(nbytes, stream_handle) ->
    device pointer as int (0 on failure), free(ptr).  Nets built afterwards
    allocate through them (blocks must be 256-byte aligned); None restores
    cudaMalloc / cudaFree."""
    global _allocator_refs
    lib = load()
    if alloc is None:
        lib.snn_set_allocator(None, None, None)
        _allocator_refs = None
        return
    a = _ALLOC_FN(lambda n, stream, ctx: alloc(int(n), stream or 0) or None)
    f = _FREE_FN(lambda ptr, ctx: free(int(ptr)))
    lib.snn_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None)
    _allocator_refs = (a, f)


def torch_allocator():
    """(alloc, free) on PyTorch's caching allocator, for set_allocator."""
    import torch

    def alloc(n, stream):
        return torch.cuda.caching_allocator_alloc(n, torch.cuda.current_device(), stream)

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)
    return alloc, free


def snn_build_network(cfg: dict, stream=None, hbm_budget_bytes: int = 0, raster_capacity=None):
    lib = load()
    h = ctypes.c_void_p()
    c = make_config(cfg, raster_capacity)
    _check(lib.snn_build_network(ctypes.byref(c), _stream_handle(stream), hbm_budget_bytes, ctypes.byref(h)),
           "snn_build_network")
    return h


def snn_build_network_explicit(cfg: dict, row_off, tgt, delay, w, stream=None, hbm_budget_bytes: int = 0,
                               raster_capacity=None):
    lib = load()
    ro = np.ascontiguousarray(row_off, np.int64)
    tg = np.ascontiguousarray(tgt, np.int32)
    dl = np.ascontiguousarray(delay, np.uint8)
    ww = np.ascontiguousarray(w, np.int32)
    h = ctypes.c_void_p()
    c = make_config(cfg, raster_capacity)
    _check(lib.snn_build_network_explicit(ctypes.byref(c), _ptr(ro), _ptr(tg), _ptr(dl), _ptr(ww),
                                          _stream_handle(stream), hbm_budget_bytes, ctypes.byref(h)),
           "snn_build_network_explicit")
    return h


def snn_step(h):
    _check(load().snn_step(h), "snn_step")


def snn_run(h, n_ms: int):
    _check(load().snn_run(h, int(n_ms)), "snn_run")


def snn_free(h):
    load().snn_free(h)


def snn_read_raster(h, t0: int, t1: int):
    """(t, gid) numpy arrays of steps [t0, t1), sorted by (t, gid)."""
    lib = load()
    n = ctypes.c_size_t(0)
    rc = lib.snn_read_raster(h, t0, t1, None, 0, ctypes.byref(n))
    if rc not in (OK, ETRUNC):
        _check(rc, "snn_read_raster")
    buf = np.empty(max(n.value, 1), SPIKE_DTYPE)
    _check(lib.snn_read_raster(h, t0, t1, _ptr(buf), n.value, ctypes.byref(n)), "snn_read_raster")
    buf = buf[: n.value]
    return buf["t"].copy(), buf["gid"].copy()


def snn_read_weights(h, n_synapses: int):
    w = np.empty(max(n_synapses, 1), np.int32)
    sd = np.empty(max(n_synapses, 1), np.int32)
    n = ctypes.c_size_t(0)
    _check(load().snn_read_weights(h, _ptr(w), _ptr(sd), n_synapses, ctypes.byref(n)), "snn_read_weights")
    return w[: n.value], sd[: n.value]


def snn_thalamic_events(cfg: dict, t0: int, n_ms: int) -> np.ndarray:
    """Thalamic drive of cfg for steps [t0, t0 + n_ms) as host events (STIM_DTYPE)."""
    lib = load()
    c = make_config(cfg, 0)
    n = ctypes.c_size_t(0)
    rc = lib.snn_thalamic_events(ctypes.byref(c), int(t0), int(n_ms), None, 0, ctypes.byref(n))
    if rc not in (OK, ETRUNC):
        _check(rc, "snn_thalamic_events")
    out = np.empty(max(n.value, 1), STIM_DTYPE)
    _check(lib.snn_thalamic_events(ctypes.byref(c), int(t0), int(n_ms), _ptr(out), n.value, ctypes.byref(n)),
           "snn_thalamic_events")
    return out[: n.value]


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
def snn_microbench_atomics(array_bytes: int, ops_per_thread: int = 4096, stream=None) -> dict:
    """Rates (1e9 operations / s) of scattered L2 reductions, gathers and
    shared-memory atomics on this GPU (see include/snn.h)."""
    r = SnnAtomicRates()
    _check(load().snn_microbench_atomics(int(array_bytes), int(ops_per_thread), _stream_handle(stream),
                                         ctypes.byref(r)), "snn_microbench_atomics")
    return {name: getattr(r, name) for name, _ in SnnAtomicRates._fields_}


class Network:
    """One network on the device.  cfg: a parameter dictionary (workloads.py)."""

    def __init__(self, cfg: dict, stream=None, hbm_budget_bytes: int = 0, raster_capacity=None,
                 explicit: dict | None = None):
        self.cfg = dict(cfg)
        self._lib = load()
        self.stream = stream
        if explicit is None:
            self.h = snn_build_network(self.cfg, stream, hbm_budget_bytes, raster_capacity)
        else:
            self.h = snn_build_network_explicit(self.cfg, explicit["row_off"], explicit["tgt"], explicit["delay"],
                                                explicit["w"], stream, hbm_budget_bytes, raster_capacity)
        n = ctypes.c_uint32()
        s = ctypes.c_int64()
        b = ctypes.c_size_t()
        _check(self._lib.snn_net_info(self.h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(b)), "snn_net_info")
        self.n_neurons, self.n_synapses, self.device_bytes = n.value, s.value, b.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.snn_free(self.h)
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

    # simulation
    def step(self):
        snn_step(self.h)

    def run(self, n_ms: int):
        snn_run(self.h, n_ms)

    def run_host(self, n_ms: int, stimulus=None, cap: int | None = None):
        """End-to-end call on host buffers: returns (t, gid) of the window."""
        st = None if stimulus is None else np.ascontiguousarray(stimulus, STIM_DTYPE)
        cap = cap if cap is not None else int(self.cfg.get("raster_capacity", 0) or 1 << 20)
        out = np.empty(max(cap, 1), SPIKE_DTYPE)
        n = ctypes.c_size_t(0)
        _check(self._lib.snn_run_host(self.h, int(n_ms), _ptr(st), 0 if st is None else len(st), _ptr(out), cap,
                                      ctypes.byref(n)), "snn_run_host")
        out = out[: n.value]
        return out["t"].copy(), out["gid"].copy()

    def set_tile(self, first_col: int, n_cols: int):
        """Own (integrate, deliver to) columns [first_col, first_col + n_cols) only."""
        _check(self._lib.snn_set_tile(self.h, int(first_col), int(n_cols)), "snn_set_tile")

    def inject_spikes(self, gids):
        """Spikes of the last step of neurons owned by other tiles."""
        g = np.ascontiguousarray(gids, np.int32)
        _check(self._lib.snn_inject_spikes(self.h, _ptr(g) if len(g) else None, len(g)), "snn_inject_spikes")

    def set_thalamic(self, on: bool):
        _check(self._lib.snn_set_thalamic(self.h, int(bool(on))), "snn_set_thalamic")

    def autotune(self, probe_ms: int = 50) -> dict:
        """Pick the fastest launch shape (the net is left reset at t = 0)."""
        L = SnnLaunch()
        _check(self._lib.snn_autotune(self.h, int(probe_ms), ctypes.byref(L)), "snn_autotune")
        return {k: getattr(L, k) for k, _ in SnnLaunch._fields_}

    def reset(self):
        _check(self._lib.snn_reset(self.h), "snn_reset")

    def run_host_counts(self, n_ms: int, stimulus=None) -> int:
        """End-to-end call without raster read-back: spikes emitted in the window."""
        st = None if stimulus is None else np.ascontiguousarray(stimulus, STIM_DTYPE)
        n = ctypes.c_size_t(0)
        _check(self._lib.snn_run_host(self.h, int(n_ms), _ptr(st), 0 if st is None else len(st), None, 0,
                                      ctypes.byref(n)), "snn_run_host")
        return n.value

    def set_stimulus(self, t, gid, q16):
        ev = np.zeros(len(t), STIM_DTYPE)
        ev["t"], ev["gid"], ev["q16"] = t, gid, q16
        _check(self._lib.snn_set_stimulus(self.h, _ptr(ev), len(ev)), "snn_set_stimulus")

    def set_launch(self, **kw):
        L = SnnLaunch()
        for k, v in kw.items():
            setattr(L, k, int(v))
        _check(self._lib.snn_set_launch(self.h, ctypes.byref(L)), "snn_set_launch")

    def get_launch(self) -> dict:
        L = SnnLaunch()
        _check(self._lib.snn_get_launch(self.h, ctypes.byref(L)), "snn_get_launch")
        return {k: getattr(L, k) for k, _ in SnnLaunch._fields_}

    def set_profile(self, on: bool):
        _check(self._lib.snn_set_profile(self.h, int(bool(on))), "snn_set_profile")

    def profile(self) -> dict:
        p = SnnProfile()
        _check(self._lib.snn_read_profile(self.h, ctypes.byref(p)), "snn_read_profile")
        out = {k: (int(p.launches[i]), float(p.ms[i])) for i, k in enumerate(KERNELS)}
        for k in ("dense_steps", "dense_deriv_steps", "dense_events", "dense_exc_events", "dense_ltp_visits",
                  "kernels"):
            out[k] = int(getattr(p, k))
        return out

    # observables
    @property
    def t(self) -> int:
        return self.counters()["t"]

    def raster(self, t0: int = 0, t1: int | None = None):
        return snn_read_raster(self.h, t0, 2 ** 31 - 1 if t1 is None else t1)

    def raster_reset(self):
        _check(self._lib.snn_raster_reset(self.h), "snn_raster_reset")

    def synapses(self, first: int = 0, count: int | None = None, fields=("tgt", "delay", "w", "sd")):
        count = self.n_neurons - first if count is None else count
        n = ctypes.c_size_t(0)
        rc = self._lib.snn_read_synapses(self.h, first, count, None, None, None, None, 0, ctypes.byref(n))
        if rc not in (OK, ETRUNC):
            _check(rc, "snn_read_synapses")
        m = n.value
        out = {}
        out["tgt"] = np.empty(max(m, 1), np.int32) if "tgt" in fields else None
        out["delay"] = np.empty(max(m, 1), np.uint8) if "delay" in fields else None
        out["w"] = np.empty(max(m, 1), np.int32) if "w" in fields else None
        out["sd"] = np.empty(max(m, 1), np.int32) if "sd" in fields else None
        _check(self._lib.snn_read_synapses(self.h, first, count, _ptr(out["tgt"]), _ptr(out["delay"]),
                                           _ptr(out["w"]), _ptr(out["sd"]), m, ctypes.byref(n)), "snn_read_synapses")
        return {k: (v[:m] if v is not None else None) for k, v in out.items()}

    def weights(self):
        return snn_read_weights(self.h, self.n_synapses)

    def neurons(self, first: int = 0, count: int | None = None):
        count = self.n_neurons - first if count is None else count
        v = np.empty(max(count, 1), np.float32)
        u = np.empty(max(count, 1), np.float32)
        _check(self._lib.snn_read_neurons(self.h, first, count, _ptr(v), _ptr(u)), "snn_read_neurons")
        return dict(v=v[:count], u=u[:count])

    def neurons_f64(self, first: int = 0, count: int | None = None):
        count = self.n_neurons - first if count is None else count
        v = np.empty(max(count, 1), np.float64)
        u = np.empty(max(count, 1), np.float64)
        _check(self._lib.snn_read_neurons_f64(self.h, first, count, _ptr(v), _ptr(u)), "snn_read_neurons_f64")
        return dict(v=v[:count], u=u[:count])

    def set_probe(self, gids, max_steps: int):
        g = np.ascontiguousarray(gids, np.int32)
        _check(self._lib.snn_set_probe(self.h, _ptr(g) if len(g) else None, len(g), int(max_steps)), "snn_set_probe")
        self._probe_n = len(g)

    def probe(self):
        """(v, u) traces recorded so far, arrays of shape (steps, probed neurons)."""
        steps = ctypes.c_uint32(0)
        _check(self._lib.snn_read_probe(self.h, None, None, 0, ctypes.byref(steps)), "snn_read_probe")
        k = getattr(self, "_probe_n", 0)
        v = np.empty(max(steps.value * k, 1), np.float32)
        u = np.empty(max(steps.value * k, 1), np.float32)
        _check(self._lib.snn_read_probe(self.h, _ptr(v), _ptr(u), steps.value * k, ctypes.byref(steps)),
               "snn_read_probe")
        n = steps.value * k
        return v[:n].reshape(steps.value, k), u[:n].reshape(steps.value, k)

    def counters(self) -> dict:
        c = SnnCounters()
        _check(self._lib.snn_read_counters(self.h, ctypes.byref(c)), "snn_read_counters")
        return {k: getattr(c, k) for k, _ in SnnCounters._fields_ if k != "reserved"}

    def save_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(self._lib.snn_save_state(self.h, None, 0, ctypes.byref(n)), "snn_save_state")
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.snn_save_state(self.h, buf, n.value, ctypes.byref(n)), "snn_save_state")
        return buf.raw

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self._lib.snn_load_state(self.h, buf, len(data)), "snn_load_state")


class Batch:
    """Many independent nets advanced together: one CUDA graph per chunk of
    steps, one launch per kind of step kernel per step for all nets.  Does
    not own the nets."""

    def __init__(self, nets, graph_steps: int = 10):
        self._lib = load()
        self.nets = list(nets)
        arr = (ctypes.c_void_p * len(self.nets))(*[n.h.value for n in self.nets])
        self.h = ctypes.c_void_p()
        _check(self._lib.snn_batch_create(arr, len(self.nets), int(graph_steps), ctypes.byref(self.h)),
               "snn_batch_create")

    def run(self, n_ms: int):
        _check(self._lib.snn_batch_run(self.h, int(n_ms)), "snn_batch_run")

    def set_launch(self, **fields):
        L = SnnLaunch()
        for k, v in fields.items():
            setattr(L, k, int(v))
        _check(self._lib.snn_batch_set_launch(self.h, ctypes.byref(L)), "snn_batch_set_launch")

    def get_launch(self) -> dict:
        L = SnnLaunch()
        _check(self._lib.snn_batch_get_launch(self.h, ctypes.byref(L)), "snn_batch_get_launch")
        return {k: getattr(L, k) for k, _ in SnnLaunch._fields_}

    def autotune(self, probe_ms: int = 50) -> dict:
        """Pick the fastest batch launch shape; every net is left reset at t = 0."""
        L = SnnLaunch()
        _check(self._lib.snn_batch_autotune(self.h, int(probe_ms), ctypes.byref(L)), "snn_batch_autotune")
        return {k: getattr(L, k) for k, _ in SnnLaunch._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._lib.snn_batch_free(self.h)
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
