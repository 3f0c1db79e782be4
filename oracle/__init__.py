"""ctypes front end of the plain CPU simulator in oracle/oracle.c.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke check in
__graft_entry__ and the cpu_baseline / reference leg of bench.py may import
this package.  It does not import the CUDA path and the CUDA path does not
import it; both take the plain parameter dictionaries of workloads.py.

Every function of oracle.c is pinned against the paper and the mathematics
by tests/test_oracle_pins.py and tests/test_oracle_generator_pins.py (their
sensitivity: tests/test_oracle_mutants.py); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
# ORC_LIB names another build of oracle.c to load instead (the mutation test
# of the pins loads deliberately broken copies this way)
LIB_PATH = os.environ.get("ORC_LIB") or os.path.join(BUILD_DIR, "liborc.so")

STDP_OFF = 1
DELIVERY_OFF = 2
FP64 = 4
BRUTE_DELIVERY = 8


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("grid_x", ctypes.c_uint32), ("grid_y", ctypes.c_uint32),
        ("neurons_per_col", ctypes.c_uint32), ("exc_per_col", ctypes.c_uint32),
        ("fanout", ctypes.c_uint32),
        ("pct_ring", ctypes.c_uint32 * 4),
        ("max_delay_ms", ctypes.c_uint32),
        ("w_exc0_q16", ctypes.c_int32), ("w_inh0_q16", ctypes.c_int32), ("wmax_q16", ctypes.c_int32),
        ("a_plus_mv", ctypes.c_double), ("a_minus_mv", ctypes.c_double),
        ("tau_plus_ms", ctypes.c_double), ("tau_minus_ms", ctypes.c_double),
        ("deriv_period_ms", ctypes.c_uint32),
        ("deriv_bias_q16", ctypes.c_int32), ("deriv_decay_q16", ctypes.c_int32),
        ("thal_per_col_per_ms", ctypes.c_uint32),
        ("thal_amp_q16", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
    ]


class OrcStim(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int32), ("gid", ctypes.c_int32), ("q16", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liborc.so (gcc, no FMA contraction)."""
    if os.environ.get("ORC_LIB"):
        return LIB_PATH
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        c_sim = ctypes.c_void_p
        L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.orc_philox4x32_10.restype = None
        L.orc_stdp_q16.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        L.orc_stdp_q16.restype = ctypes.c_int32
        L.orc_neuron_step_f32.argtypes = [P(ctypes.c_float), P(ctypes.c_float), ctypes.c_int32, ctypes.c_int]
        L.orc_neuron_step_f32.restype = ctypes.c_int
        L.orc_neuron_step_f64.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int32, ctypes.c_int]
        L.orc_neuron_step_f64.restype = ctypes.c_int
        L.orc_deriv_q16.argtypes = [P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32]
        L.orc_deriv_q16.restype = None
        L.orc_generate_synapse.argtypes = [P(OrcConfig), ctypes.c_uint32, ctypes.c_uint32,
                                           P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.orc_generate_synapse.restype = None
        L.orc_thalamic_target.argtypes = [P(OrcConfig), ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_thalamic_target.restype = ctypes.c_uint32
        L.orc_create.argtypes = [P(OrcConfig), ctypes.c_char_p, ctypes.c_size_t]
        L.orc_create.restype = c_sim
        L.orc_create_explicit.argtypes = [P(OrcConfig), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
        L.orc_create_explicit.restype = c_sim
        L.orc_free.argtypes = [c_sim]
        L.orc_free.restype = None
        L.orc_set_stimulus.argtypes = [c_sim, ctypes.c_void_p, ctypes.c_int64]
        L.orc_set_stimulus.restype = ctypes.c_int
        L.orc_step.argtypes = [c_sim]
        L.orc_run.argtypes = [c_sim, ctypes.c_int32]
        L.orc_n_neurons.argtypes = [c_sim]
        L.orc_n_neurons.restype = ctypes.c_uint32
        L.orc_n_synapses.argtypes = [c_sim]
        L.orc_n_synapses.restype = ctypes.c_int64
        L.orc_time.argtypes = [c_sim]
        L.orc_time.restype = ctypes.c_int32
        L.orc_raster_size.argtypes = [c_sim]
        L.orc_raster_size.restype = ctypes.c_int64
        L.orc_error.argtypes = [c_sim]
        L.orc_error.restype = ctypes.c_char_p
        L.orc_read_raster.argtypes = [c_sim, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_read_synapses.argtypes = [c_sim, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.orc_read_row_offsets.argtypes = [c_sim, ctypes.c_void_p]
        L.orc_read_neurons.argtypes = [c_sim, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
        L.orc_read_counters.argtypes = [c_sim, ctypes.c_void_p]
        _lib = L
    return _lib


def make_config(cfg: dict) -> OrcConfig:
    c = OrcConfig()
    for name, _ in OrcConfig._fields_:
        if name == "pct_ring":
            for i, p in enumerate(cfg["pct_ring"]):
                c.pct_ring[i] = int(p)
        elif name == "flags":
            c.flags = int(cfg.get("oracle_flags", 0))
        else:
            setattr(c, name, cfg[name])
    return c


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# single functions of the oracle
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def stdp_q16(amplitude_mv: float, tau_ms: float, lag_ms: int) -> int:
    return int(lib().orc_stdp_q16(amplitude_mv, tau_ms, lag_ms))


def neuron_step(v, u, current_q16: int, excitatory: bool, fp64: bool = False):
    """One 1 ms neuron step; returns (v, u, fired)."""
    if fp64:
        vv, uu = ctypes.c_double(v), ctypes.c_double(u)
        fired = lib().orc_neuron_step_f64(ctypes.byref(vv), ctypes.byref(uu), int(current_q16), int(excitatory))
    else:
        vv, uu = ctypes.c_float(v), ctypes.c_float(u)
        fired = lib().orc_neuron_step_f32(ctypes.byref(vv), ctypes.byref(uu), int(current_q16), int(excitatory))
    return vv.value, uu.value, bool(fired)


def deriv_q16(w: int, sd: int, bias_q16: int, decay_q16: int, wmax_q16: int):
    ww, ss = ctypes.c_int32(w), ctypes.c_int32(sd)
    lib().orc_deriv_q16(ctypes.byref(ww), ctypes.byref(ss), bias_q16, decay_q16, wmax_q16)
    return ww.value, ss.value


def generate_synapse(cfg: dict, src: int, j: int):
    c = make_config(cfg)
    t, d = ctypes.c_uint32(), ctypes.c_uint32()
    lib().orc_generate_synapse(ctypes.byref(c), src, j, ctypes.byref(t), ctypes.byref(d))
    return t.value, d.value


def generate_row(cfg: dict, src: int):
    """(targets, delays) of one source neuron, canonical ordinal order."""
    c = make_config(cfg)
    L = lib()
    m = cfg["fanout"]
    tg = np.empty(m, np.int32)
    dl = np.empty(m, np.int32)
    t, d = ctypes.c_uint32(), ctypes.c_uint32()
    for j in range(m):
        L.orc_generate_synapse(ctypes.byref(c), src, j, ctypes.byref(t), ctypes.byref(d))
        tg[j] = t.value
        dl[j] = d.value
    return tg, dl


def thalamic_target(cfg: dict, t: int, col: int, k: int = 0) -> int:
    c = make_config(cfg)
    return int(lib().orc_thalamic_target(ctypes.byref(c), t, col, k))


# ---------------------------------------------------------------------------
# whole simulations
# ---------------------------------------------------------------------------
class Oracle:
    """A simulation in the oracle: generated from `cfg`, or from explicit
    synapse arrays (row_off[N+1], tgt, delay, w in canonical source order)."""

    def __init__(self, cfg: dict, explicit: dict | None = None, flags: int | None = None):
        self.cfg = dict(cfg)
        if flags is not None:
            self.cfg["oracle_flags"] = flags
        self._c = make_config(self.cfg)
        err = ctypes.create_string_buffer(256)
        L = lib()
        if explicit is None:
            h = L.orc_create(ctypes.byref(self._c), err, 256)
        else:
            self._keep = [np.ascontiguousarray(explicit["row_off"], np.int64),
                          np.ascontiguousarray(explicit["tgt"], np.int32),
                          np.ascontiguousarray(explicit["delay"], np.uint8),
                          np.ascontiguousarray(explicit["w"], np.int32)]
            h = L.orc_create_explicit(ctypes.byref(self._c), *[_ptr(a) for a in self._keep], err, 256)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self._h = ctypes.c_void_p(h)
        self.n_neurons = int(L.orc_n_neurons(self._h))
        self.n_synapses = int(L.orc_n_synapses(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_free(h)
            self._h = None

    @property
    def t(self) -> int:
        return int(lib().orc_time(self._h))

    def set_stimulus(self, t, gid, q16):
        ev = np.zeros(len(t), dtype=[("t", np.int32), ("gid", np.int32), ("q16", np.int32)])
        ev["t"], ev["gid"], ev["q16"] = t, gid, q16
        order = np.argsort(ev["t"], kind="stable")
        ev = np.ascontiguousarray(ev[order])
        self._stim = ev
        if lib().orc_set_stimulus(self._h, _ptr(ev), len(ev)) != 0:
            raise ValueError("oracle: bad stimulus")

    def run(self, n_ms: int):
        if lib().orc_run(self._h, int(n_ms)) != 0:
            raise RuntimeError("oracle: " + lib().orc_error(self._h).decode())

    def raster(self):
        n = int(lib().orc_raster_size(self._h))
        t = np.empty(n, np.int32)
        g = np.empty(n, np.int32)
        if n:
            lib().orc_read_raster(self._h, _ptr(t), _ptr(g))
        return t, g

    def synapses(self):
        s = self.n_synapses
        tgt = np.empty(s, np.int32)
        dly = np.empty(s, np.uint8)
        w = np.empty(s, np.int32)
        sd = np.empty(s, np.int32)
        lib().orc_read_synapses(self._h, _ptr(tgt), _ptr(dly), _ptr(w), _ptr(sd))
        ro = np.empty(self.n_neurons + 1, np.int64)
        lib().orc_read_row_offsets(self._h, _ptr(ro))
        return dict(row_off=ro, tgt=tgt, delay=dly, w=w, sd=sd)

    def neurons(self):
        n = self.n_neurons
        v = np.empty(n, np.float32)
        u = np.empty(n, np.float32)
        vd = np.empty(n, np.float64)
        ud = np.empty(n, np.float64)
        lib().orc_read_neurons(self._h, _ptr(v), _ptr(u), _ptr(vd), _ptr(ud))
        return dict(v=v, u=u, vd=vd, ud=ud)

    def counters(self):
        o = np.zeros(4, np.int64)
        lib().orc_read_counters(self._h, _ptr(o))
        return dict(spikes=int(o[0]), e_all=int(o[1]), e_exc=int(o[2]), l_exc=int(o[3]))
