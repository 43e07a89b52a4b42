"""Thin ctypes binding of the C ABI in include/ctaux.h (argument marshalling only).

Every computation runs in the CUDA library _ctaux.so; this module only builds
the parameter structs, passes pointers and converts results to numpy arrays.
Importing it raises ImportError when the library has not been built, so no
path can silently fall back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_ctaux.so")

CTAUX_FP64 = 0
CTAUX_MIXED = 1
CTAUX_GAMMA_INVERSE = 0
CTAUX_GAMMA_LU = 1
STATUS = {0: "CTAUX_OK", 1: "CTAUX_EINVAL", 2: "CTAUX_ENOMEM", 3: "CTAUX_ECUDA",
          4: "CTAUX_ECAPACITY", 5: "CTAUX_ESINGULAR", 6: "CTAUX_EDRIFT", 7: "CTAUX_ETIMEOUT",
          8: "CTAUX_ENUMERIC"}


class ChainParams(C.Structure):
    _fields_ = [("n_c", C.c_int), ("n_classes", C.c_int), ("n_tau", C.c_int),
                ("g0_table", C.POINTER(C.c_double)), ("dx_class", C.POINTER(C.c_int)),
                ("beta", C.c_double), ("U", C.c_double), ("K", C.c_double),
                ("k_max", C.c_int), ("capacity", C.c_int), ("seed", C.c_uint64),
                ("chain_id", C.c_uint32)]


class Params(C.Structure):
    _fields_ = [("n_chains", C.c_int), ("chains", C.POINTER(ChainParams)),
                ("precision", C.c_int), ("refresh_every", C.c_int),
                ("p_insert", C.c_double), ("p_flip", C.c_double),
                ("n_tau_bins", C.c_int), ("n_anchors", C.c_int),
                ("trace_capacity", C.c_int), ("device", C.c_int),
                ("mixed_flush_tc", C.c_int), ("tie_guard", C.c_double),
                ("tie_refine_iters", C.c_int), ("use_graph", C.c_int),
                ("refresh_df64", C.c_int), ("meas_bin_size", C.c_int),
                ("n_matsubara", C.c_int), ("drift_limit", C.c_double),
                ("mixed_prep_tc", C.c_int), ("tc_wait_limit", C.c_int),
                ("gamma_form", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("t", C.c_int64), ("proposals", C.c_int64 * 3),
                ("accepted", C.c_int64 * 3), ("sweeps", C.c_int64), ("measurements", C.c_int64),
                ("order_sum", C.c_int64), ("sign_sum", C.c_double),
                ("numeric_rejects", C.c_int64), ("near_ties", C.c_int64),
                ("tie_refreshes", C.c_int64),
                ("refreshes", C.c_int64),
                ("last_drift_max", C.c_double), ("last_drift_fro", C.c_double),
                ("last_drift_rel", C.c_double),
                ("logdet", C.c_double * 2), ("sign", C.c_int), ("status", C.c_int),
                ("tie_err_max", C.c_double), ("tie_guard_eff", C.c_double)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class TraceRec(C.Structure):
    _fields_ = [("t", C.c_int64), ("move", C.c_int32), ("n", C.c_int32), ("birth", C.c_int64),
                ("s_new", C.c_int32), ("accept", C.c_int32), ("ratio", C.c_double * 2),
                ("R", C.c_double), ("u", C.c_double)]


TRACE_DTYPE = np.dtype([("t", "<i8"), ("move", "<i4"), ("n", "<i4"), ("birth", "<i8"),
                        ("s_new", "<i4"), ("accept", "<i4"), ("ratio", "<f8", (2,)),
                        ("R", "<f8"), ("u", "<f8")])


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH} is missing "
                          "(run `python -m paper_1010_3690_gb300.build`)")
    lib = C.CDLL(_LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    sigs = {
        "ctaux_init": (C.c_int, [P(Params), P(vp)]),
        "ctaux_sweep": (C.c_int, [vp, C.c_int, C.c_int, vp]),
        "ctaux_measure_G": (C.c_int, [vp, C.c_int, P(C.c_double), P(C.c_double), P(C.c_int64)]),
        "ctaux_measure_G_matsubara": (C.c_int, [vp, C.c_int, P(C.c_double), P(C.c_double),
                                               P(C.c_int64)]),
        "ctaux_get_accumulators": (C.c_int, [vp, C.c_int, P(C.c_double), P(C.c_double),
                                            P(C.c_double), P(C.c_double), P(C.c_int64)]),
        "ctaux_reset_measurements": (C.c_int, [vp]),
        "ctaux_recompute": (C.c_int, [vp, P(C.c_double)]),
        "ctaux_get_stats": (C.c_int, [vp, C.c_int, P(Stats)]),
        "ctaux_get_trace": (C.c_int, [vp, C.c_int, P(TraceRec), C.c_int, P(C.c_int)]),
        "ctaux_get_config": (C.c_int, [vp, C.c_int, P(C.c_double), P(C.c_int), P(C.c_int),
                                       P(C.c_int64), C.c_int, P(C.c_int), P(C.c_int64)]),
        "ctaux_set_config": (C.c_int, [vp, C.c_int, P(C.c_double), P(C.c_int), P(C.c_int),
                                       P(C.c_int64), C.c_int, C.c_int64]),
        "ctaux_get_N": (C.c_int, [vp, C.c_int, C.c_int, P(C.c_double), C.c_int, P(C.c_int)]),
        "ctaux_set_profiling": (C.c_int, [vp, C.c_int]),
        "ctaux_get_phase_times": (C.c_int, [vp, P(C.c_double), P(C.c_int64)]),
        "ctaux_get_work": (C.c_int, [vp, P(C.c_double), P(C.c_double), P(C.c_double),
                                     P(C.c_double), P(C.c_double), P(C.c_double),
                                     P(C.c_double)]),
        "ctaux_philox_uniforms": (C.c_int, [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, C.c_int,
                                            P(C.c_double)]),
        "ctaux_set_kmax": (C.c_int, [vp, C.c_int, C.c_int]),
        "ctaux_autotune_k": (C.c_int, [vp, P(C.c_int), C.c_int, C.c_int, P(C.c_int),
                                       P(C.c_double)]),
        "ctaux_synchronize": (C.c_int, [vp]),
        "ctaux_autotune_tiles": (C.c_int, [vp, C.c_int, P(C.c_int8), P(C.c_double)]),
        "ctaux_get_tile_table": (C.c_int, [vp, P(C.c_int8)]),
        "ctaux_set_tile_table": (C.c_int, [vp, P(C.c_int8)]),
        "ctaux_invert_noalloc": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_int, vp, vp]),
        "ctaux_destroy": (None, [vp]),
        "ctaux_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()
EXPORTED = ("ctaux_init", "ctaux_sweep", "ctaux_measure_G", "ctaux_measure_G_matsubara",
            "ctaux_get_accumulators",
            "ctaux_reset_measurements",
            "ctaux_recompute", "ctaux_get_stats", "ctaux_get_trace", "ctaux_get_config",
            "ctaux_set_config", "ctaux_get_N", "ctaux_set_profiling", "ctaux_get_phase_times",
            "ctaux_get_work", "ctaux_philox_uniforms", "ctaux_synchronize", "ctaux_destroy",
            "ctaux_set_kmax", "ctaux_autotune_k", "ctaux_autotune_tiles", "ctaux_get_tile_table",
            "ctaux_set_tile_table",
            "ctaux_last_error", "ctaux_invert_noalloc")


class CtauxError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def ctaux_philox_uniforms(seed, chain, t0, count, purpose):
    out = np.empty((count, 2), dtype=np.float64)
    r = lib.ctaux_philox_uniforms(seed, chain, t0, count, purpose, _dp(out))
    if r:
        raise CtauxError(r, "philox")
    return out


def ctaux_invert_noalloc(d_a, lda, d_inv, ld_inv, m, d_logdet=None, stream=None):
    """Device pointers (ints) in, status code out; see include/ctaux.h."""
    return lib.ctaux_invert_noalloc(C.c_void_p(d_a), int(lda), C.c_void_p(d_inv), int(ld_inv),
                                    int(m), C.c_void_p(d_logdet or 0), C.c_void_p(stream or 0))


class Context:
    """One ctaux_ctx: a set of chains with their device state.

    `chains` is a sequence of objects with the attributes n_c, table
    ([2][n_classes][n_tau] float64), dx_class ([n_c][n_c] int), beta, U, K,
    k_max, capacity, seed and chain_id.
    """

    def __init__(self, chains, precision=CTAUX_FP64, refresh_every=32, p_insert=0.5, p_flip=0.0,
                 n_tau_bins=32, n_anchors=4, trace_capacity=0, device=0, mixed_flush_tc=1,
                 tie_guard=1e-4, tie_refine_iters=0, refresh_df64=0, use_graph=0,
                 meas_bin_size=0, n_matsubara=0, drift_limit=0.0, mixed_prep_tc=1,
                 tc_wait_limit=0, gamma_form=0):
        self._keep = []
        cps = (ChainParams * len(chains))()
        self.chain_inputs = list(chains)
        for i, ch in enumerate(chains):
            tab = np.ascontiguousarray(ch.table, dtype=np.float64)
            dxc = np.ascontiguousarray(ch.dx_class, dtype=np.int32)
            self._keep += [tab, dxc]
            cps[i] = ChainParams(int(ch.n_c), int(tab.shape[1]), int(tab.shape[2]), _dp(tab),
                                 _ip(dxc), float(ch.beta), float(ch.U), float(ch.K),
                                 int(ch.k_max), int(ch.capacity), int(ch.seed),
                                 int(ch.chain_id))
        self.params = Params(len(chains), cps, precision, refresh_every, p_insert, p_flip,
                             n_tau_bins, n_anchors, trace_capacity, device, mixed_flush_tc,
                             tie_guard, tie_refine_iters, int(use_graph), int(refresh_df64),
                             int(meas_bin_size), int(n_matsubara), float(drift_limit),
                             int(mixed_prep_tc), int(tc_wait_limit), int(gamma_form))
        self.n_tau_bins = n_tau_bins
        self.n_matsubara = n_matsubara
        self.trace_capacity = trace_capacity
        h = C.c_void_p()
        r = lib.ctaux_init(C.byref(self.params), C.byref(h))
        if r:
            raise CtauxError(r, "ctaux_init failed")
        self.h = h
        # the library copied everything it needs
        self._keep = []

    def _check(self, r, what):
        if r:
            raise CtauxError(r, f"{what}: {lib.ctaux_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib.ctaux_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sweep(self, n_sweeps=1, measure=False, stream=None):
        self._check(lib.ctaux_sweep(self.h, int(n_sweeps), int(bool(measure)),
                                    C.c_void_p(stream or 0)), "ctaux_sweep")

    def synchronize(self):
        self._check(lib.ctaux_synchronize(self.h), "ctaux_synchronize")

    def measure_G(self, chain=0):
        ch = self.chain_inputs[chain]
        shape = (2, np.asarray(ch.table).shape[1], self.n_tau_bins)
        G = np.empty(shape)
        E = np.empty(shape)
        nm = C.c_int64()
        self._check(lib.ctaux_measure_G(self.h, chain, _dp(G), _dp(E), C.byref(nm)), "measure_G")
        return G, E, nm.value

    def measure_G_matsubara(self, chain=0):
        """(mean G_xy(i w_n) [2, n_c, n_c, n_matsubara] complex, standard errors of the
        real and imaginary parts [2, n_c, n_c, n_matsubara, 2], measurements)."""
        n_c = int(self.chain_inputs[chain].n_c)
        shape = (2, n_c, n_c, self.n_matsubara, 2)
        G = np.empty(shape)
        E = np.empty(shape)
        nm = C.c_int64()
        self._check(lib.ctaux_measure_G_matsubara(self.h, chain, _dp(G), _dp(E), C.byref(nm)),
                    "measure_G_matsubara")
        return G[..., 0] + 1j * G[..., 1], E, nm.value

    def accumulators(self, chain=0):
        """Raw sums for merging chains or ranks: dict of sum, sumsq, bin_sum,
        bin_sumsq ([2, n_classes, n_tau_bins]) and n_meas, n_bins, bin_size."""
        ch = self.chain_inputs[chain]
        shape = (2, np.asarray(ch.table).shape[1], self.n_tau_bins)
        arrs = [np.empty(shape) for _ in range(4)]
        cnt = np.zeros(3, np.int64)
        self._check(lib.ctaux_get_accumulators(self.h, chain, *(_dp(a) for a in arrs), _lp(cnt)),
                    "get_accumulators")
        return dict(sum=arrs[0], sumsq=arrs[1], bin_sum=arrs[2], bin_sumsq=arrs[3],
                    n_meas=int(cnt[0]), n_bins=int(cnt[1]), bin_size=int(cnt[2]))

    def reset_measurements(self):
        self._check(lib.ctaux_reset_measurements(self.h), "reset_measurements")

    def recompute(self):
        d = C.c_double()
        self._check(lib.ctaux_recompute(self.h, C.byref(d)), "recompute")
        return d.value

    def stats(self, chain=0):
        s = Stats()
        self._check(lib.ctaux_get_stats(self.h, chain, C.byref(s)), "get_stats")
        return s.as_dict()

    def trace(self, chain=0, cap=None):
        cap = cap or max(1, self.trace_capacity)
        buf = (TraceRec * cap)()
        n = C.c_int()
        self._check(lib.ctaux_get_trace(self.h, chain, buf, cap, C.byref(n)), "get_trace")
        arr = np.frombuffer(buf, dtype=TRACE_DTYPE, count=n.value).copy()
        return arr

    def get_config(self, chain=0):
        cap = int(self.chain_inputs[chain].capacity)
        tau = np.empty(cap)
        site = np.empty(cap, np.int32)
        s = np.empty(cap, np.int32)
        birth = np.empty(cap, np.int64)
        n = C.c_int()
        t = C.c_int64()
        self._check(lib.ctaux_get_config(self.h, chain, _dp(tau), _ip(site), _ip(s), _lp(birth),
                                         cap, C.byref(n), C.byref(t)), "get_config")
        k = n.value
        return dict(tau=tau[:k].copy(), site=site[:k].copy(), s=s[:k].copy(),
                    birth=birth[:k].copy(), t=t.value)

    def set_config(self, chain, tau, site, s, birth, t):
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        site = np.ascontiguousarray(site, dtype=np.int32)
        s = np.ascontiguousarray(s, dtype=np.int32)
        birth = np.ascontiguousarray(birth, dtype=np.int64)
        self._check(lib.ctaux_set_config(self.h, chain, _dp(tau), _ip(site), _ip(s), _lp(birth),
                                         len(tau), int(t)), "set_config")

    def get_N(self, chain=0, spin=0):
        m = C.c_int()
        self._check(lib.ctaux_get_N(self.h, chain, spin, None, 0, C.byref(m)), "get_N")
        k = m.value
        out = np.zeros((max(k, 1), max(k, 1)), order="F")
        self._check(lib.ctaux_get_N(self.h, chain, spin, _dp(out), max(k, 1), C.byref(m)), "get_N")
        return out[:k, :k]

    def set_kmax(self, chain, k_max):
        self._check(lib.ctaux_set_kmax(self.h, int(chain), int(k_max)), "set_kmax")

    def autotune_k(self, candidates=(16, 32, 64, 128), n_blocks=8):
        """Choose k_max per chain on the device; returns (k per chain, proposals/s)."""
        cand = np.ascontiguousarray(candidates, dtype=np.int32)
        k = np.zeros(len(self.chain_inputs), np.int32)
        rate = C.c_double()
        self._check(lib.ctaux_autotune_k(self.h, _ip(cand), len(cand), int(n_blocks), _ip(k),
                                         C.byref(rate)), "autotune_k")
        return k, rate.value

    TILE_TABLE_SIZE = 720

    def autotune_tiles(self, n_blocks=4):
        """Tile shape per (product, order octave, k octave) timed on the device;
        returns (table [720] int8, gain of the chosen shapes over the defaults)."""
        t = np.zeros(self.TILE_TABLE_SIZE, np.int8)
        g = C.c_double()
        self._check(lib.ctaux_autotune_tiles(self.h, int(n_blocks),
                                             t.ctypes.data_as(C.POINTER(C.c_int8)), C.byref(g)),
                    "autotune_tiles")
        return t, g.value

    def tile_table(self):
        t = np.zeros(self.TILE_TABLE_SIZE, np.int8)
        self._check(lib.ctaux_get_tile_table(self.h, t.ctypes.data_as(C.POINTER(C.c_int8))),
                    "get_tile_table")
        return t

    def set_tile_table(self, table):
        t = np.ascontiguousarray(table, dtype=np.int8)
        self._check(lib.ctaux_set_tile_table(self.h, t.ctypes.data_as(C.POINTER(C.c_int8))),
                    "set_tile_table")

    def set_profiling(self, on=True):
        self._check(lib.ctaux_set_profiling(self.h, int(bool(on))), "set_profiling")

    PHASES = ("plan_gather", "prep", "proposals", "flush_gemm", "flush_support", "measure",
              "refresh", "tie_refine")

    def phase_times(self):
        """(ms per phase while profiling was on, kernels launched per phase)."""
        ms = np.zeros(len(self.PHASES))
        ln = np.zeros(len(self.PHASES), np.int64)
        self._check(lib.ctaux_get_phase_times(self.h, _dp(ms), _lp(ln)), "phase_times")
        return ms, ln

    def work(self):
        a, b, c, g, me, rf, mw = (C.c_double() for _ in range(7))
        self._check(lib.ctaux_get_work(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(g),
                                       C.byref(me), C.byref(rf), C.byref(mw)), "get_work")
        return dict(prep_flop=a.value, flush_flop=b.value, flush_bytes=c.value,
                    gamma_flop=g.value, meas_flop=me.value, refresh_flop=rf.value,
                    mats_flop=mw.value)
