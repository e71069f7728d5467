"""ctypes binding of libecpic (``include/ecpic.h``): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays to pointers and status codes to exceptions.  There is no fallback: if
``libecpic.so`` cannot be built or loaded the import of ``lib()`` raises.
The module-level functions carry the C names (``ecpic_create`` ...); ``Run``
is a convenience wrapper over them.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libecpic.so")

ECPIC_OK = 0
ECPIC_ERR_ARG, ECPIC_ERR_STATE, ECPIC_ERR_NOMEM = -1, -2, -3
ECPIC_ERR_CAPACITY, ECPIC_ERR_CUDA, ECPIC_ERR_TIMEOUT, ECPIC_ERR_NAN = -4, -5, -6, -7
ECPIC_MAX_SPECIES, ECPIC_MAX_PROC, ECPIC_MAX_CELLS = 4, 8, 2048
ECPIC_DIRICHLET_RF, ECPIC_PERIODIC = 0, 1
ECPIC_SCHEME_EC, ECPIC_SCHEME_MC, ECPIC_SCHEME_EC2, ECPIC_SCHEME_MC2 = 0, 1, 2, 3
ECPIC_ELASTIC, ECPIC_EXCITATION, ECPIC_IONIZATION, ECPIC_ION_ELASTIC, ECPIC_CX = 0, 1, 2, 3, 4

_STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_STATE", -3: "ERR_NOMEM", -4: "ERR_CAPACITY",
           -5: "ERR_CUDA", -6: "ERR_TIMEOUT", -7: "ERR_NAN"}


class EcpicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class ecpic_diag(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("time", C.c_double), ("n_species", C.c_int), ("n_cells", C.c_int),
        ("n_live", C.c_int64 * 4), ("absorbed", (C.c_int64 * 2) * 4), ("births", C.c_int64 * 4),
        ("lost", C.c_int64 * 4), ("candidates", C.c_int64 * 4), ("clamps", C.c_int64 * 4),
        ("collisions", (C.c_int64 * 8) * 4), ("ke", C.c_double * 4), ("fe", C.c_double),
        ("n_samples", C.c_int64), ("density", C.c_void_p), ("phi", C.c_void_p),
        ("temp_x", C.c_void_p), ("temp_x_mom", C.c_void_p),
        ("eedf_bins", C.c_int), ("iedf_bins", C.c_int), ("iad_bins", C.c_int),
        ("eedf_cell0", C.c_int), ("eedf_cell1", C.c_int), ("eedf_dE", C.c_double),
        ("iedf_dE", C.c_double), ("impacts_dropped", C.c_int64 * 4), ("eedf", C.c_void_p),
        ("iedf", C.c_void_p), ("iad", C.c_void_p), ("power", C.c_void_p),
        ("rb_merged", C.c_int64 * 4), ("rb_split", C.c_int64 * 4), ("rb_skipped", C.c_int64 * 4),
    ]


# default tally shape: (eedf, iedf, iad) bins
TALLY_DEFAULT = dict(eedf_center=-1.0, eedf_halfwidth=0.5e-3, eedf_dE=0.5, eedf_bins=100,
                     iedf_dE=2.0, iedf_bins=256, iad_bins=90)


class ecpic_process_desc(C.Structure):
    _fields_ = [("species", C.c_int), ("kind", C.c_int), ("threshold_eV", C.c_double),
                ("dE_eV", C.c_double), ("n", C.c_int), ("sigma_m2", C.c_void_p),
                ("product_species", C.c_int)]


class ecpic_run_config(C.Structure):
    _fields_ = [
        ("edges", C.c_void_p), ("n_edges", C.c_int), ("bc", C.c_int), ("v0", C.c_double),
        ("freq_hz", C.c_double), ("phase_rad", C.c_double), ("v_dc", C.c_double),
        ("scheme", C.c_int), ("n_species", C.c_int), ("q", C.c_double * 4), ("m", C.c_double * 4),
        ("w", C.c_double * 4), ("capacity", C.c_int64 * 4), ("n_init", C.c_int64 * 4),
        ("T_eV", C.c_double * 4), ("n_gas", C.c_double), ("T_gas", C.c_double),
        ("m_gas", C.c_double), ("n_proc", C.c_int), ("procs", C.c_void_p), ("seed", C.c_uint64),
        ("dt", C.c_double), ("sample_every", C.c_int), ("quiet_start", C.c_int),
        ("eedf_center", C.c_double), ("eedf_halfwidth", C.c_double), ("eedf_dE", C.c_double),
        ("eedf_bins", C.c_int), ("iedf_dE", C.c_double), ("iedf_bins", C.c_int),
        ("iad_bins", C.c_int),
        ("rb_every", C.c_int), ("rb_target", C.c_int), ("rb_lo", C.c_int), ("rb_hi", C.c_int),
        ("rb_m0", C.c_uint32),
    ]


# name -> (restype, argtypes); the exported symbols of include/ecpic.h
vp, i32, i64, u32, u64, d = C.c_void_p, C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
SIGNATURES = {
    "ecpic_engine_create": (i32, [C.POINTER(vp), i32, vp, C.c_size_t, i32, i32, i32]),
    "ecpic_engine_destroy": (None, [vp]),
    "ecpic_engine_last_error": (C.c_char_p, [vp]),
    "ecpic_engine_submit": (i32, [vp, C.POINTER(ecpic_run_config), i64, C.POINTER(u64)]),
    "ecpic_engine_pump": (i32, [vp, i64, C.POINTER(i32), C.POINTER(i32)]),
    "ecpic_engine_poll": (i32, [vp, u64, C.POINTER(i32), C.POINTER(ecpic_diag), C.POINTER(i64),
                                C.POINTER(i64)]),
    "ecpic_engine_release": (i32, [vp, u64]),
    "ecpic_engine_stats": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]),
    "ecpic_engine_tune": (i32, [vp, i32, i32]),
    "ecpic_engine_profile": (i32, [vp, i64, vp, vp]),
    "ecpic_engine_autotune": (i32, [vp, i64, vp, vp, vp]),
    "ecpic_engine_autotune_ks": (i32, [vp, i64, vp, i32, vp, vp, vp]),
    "ecpic_engine_set_phase_timing": (i32, [vp, i32]),
    "ecpic_engine_phase_times": (i32, [vp, vp, vp, C.POINTER(i64), C.POINTER(i64)]),
    "ecpic_engine_sort_state": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
    "ecpic_autotune_ks": (i32, [vp, i64, vp, i32, vp, vp, vp]),
    "ecpic_set_phase_timing": (i32, [vp, i32]),
    "ecpic_phase_times": (i32, [vp, vp, vp, C.POINTER(i64), C.POINTER(i64)]),
    "ecpic_sort_state": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
    "ecpic_autotune": (i32, [vp, i64, vp, vp, vp]),
    "ecpic_set_quiet_start": (i32, [vp, i32]),
    "ecpic_set_rebalance": (i32, [vp, i32, i32, i32, i32, u32]),
    "ecpic_rebalance_now": (i32, [vp]),
    "ecpic_get_weights": (i32, [vp, i32, vp, i64, C.POINTER(i64)]),
    "ecpic_set_weights": (i32, [vp, i32, vp, i64]),
    "ecpic_set_tallies": (i32, [vp, d, d, d, i32, d, i32, i32]),
    "ecpic_create": (i32, [C.POINTER(vp), i32, vp]),
    "ecpic_destroy": (None, [vp]),
    "ecpic_last_error": (C.c_char_p, [vp]),
    "ecpic_set_grid": (i32, [vp, vp, i32, i32, d, d, d, d]),
    "ecpic_set_scheme": (i32, [vp, i32]),
    "ecpic_add_species": (i32, [vp, d, d, d, i64, C.POINTER(i32)]),
    "ecpic_set_gas": (i32, [vp, d, d, d]),
    "ecpic_add_process": (i32, [vp, i32, i32, d, d, i32, vp, i32]),
    "ecpic_init": (i32, [vp, u64, d, vp, vp]),
    "ecpic_step": (i32, [vp, i64]),
    "ecpic_sync": (i32, [vp]),
    "ecpic_reset_averages": (i32, [vp, i32]),
    "ecpic_diagnostics": (i32, [vp, C.POINTER(ecpic_diag)]),
    "ecpic_get_particles": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, i64, C.POINTER(i64)]),
    "ecpic_set_particles": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, i64]),
    "ecpic_get_fields": (i32, [vp, vp, vp]),
    "ecpic_nu_max": (i32, [vp, i32, C.POINTER(d), C.POINTER(u32)]),
    "ecpic_set_sort_every": (i32, [vp, i32]),
    "ecpic_sort_now": (i32, [vp]),
    "ecpic_reserve": (i32, [vp, i32, i64]),
    "ecpic_set_auto_grow": (i32, [vp, i32]),
    "ecpic_profile_step": (i32, [vp, i64, vp, vp]),
    "ecpic_set_pass_grid": (i32, [vp, i32]),
    "ecpic_doubling_grid": (i32, [i32, d, d, i32, i32, vp, i32]),
    "ecpic_deposit_device": (i32, [i32, i64, vp, vp, vp, vp]),
    "ecpic_deposit_device_noalloc": (i32, [i32, i64, vp, vp, vp, vp]),
    "ecpic_deposit_device2": (i32, [i32, i32, i64, vp, vp, vp, vp]),
    "ecpic_philox_device": (i32, [i64, vp, vp, vp, vp]),
    "ecpic_debug_checks": (i32, [vp]),
}

_lock = threading.Lock()
_lib = None


def lib(build_if_missing: bool = True):
    """Load libecpic.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _build
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libecpic.so not found at {LIB_PATH}; run build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _phase_times(call):
    ms = np.zeros(4)
    cnt = np.zeros(4, np.int64)
    st, so = C.c_int64(), C.c_int64()
    call(_p(ms), _p(cnt), C.byref(st), C.byref(so))
    return dict(pass_ms=float(ms[0]), field_ms=float(ms[1]), sort_ms=float(ms[2]),
                collide_ms=float(ms[3]), launches=cnt.tolist(), steps=st.value, sorts=so.value)


def _chk(h, rc, what):
    if rc != ECPIC_OK:
        msg = lib().ecpic_last_error(h).decode() if h else ""
        raise EcpicError(rc, f"{what}: {msg}")
    return rc


# ---------------------------------------------------------------- C names
def ecpic_create(device=0, stream=None):
    h = C.c_void_p()
    rc = lib().ecpic_create(C.byref(h), device, stream)
    if rc != ECPIC_OK:
        raise EcpicError(rc, "ecpic_create (no CUDA device?)")
    return h


def ecpic_destroy(h):
    lib().ecpic_destroy(h)


def ecpic_doubling_grid(n_ref, L, L_buff, dx_min, dx_max):
    e = np.zeros(n_ref + 1)
    n = lib().ecpic_doubling_grid(n_ref, L, L_buff, dx_min, dx_max, _p(e), e.size)
    if n < 0:
        raise EcpicError(n, "ecpic_doubling_grid")
    return e[: n + 1].copy()


def ecpic_deposit_device(N, n, d_cell, d_xi, d_S, stream=None):
    rc = lib().ecpic_deposit_device(N, n, d_cell, d_xi, d_S, stream)
    if rc != ECPIC_OK:
        raise EcpicError(rc, "ecpic_deposit_device")


def ecpic_deposit_device2(N, bc, n, d_cell, d_xi, d_S, stream=None):
    rc = lib().ecpic_deposit_device2(N, bc, n, d_cell, d_xi, d_S, stream)
    if rc != ECPIC_OK:
        raise EcpicError(rc, "ecpic_deposit_device2")


def ecpic_deposit_device_noalloc(N, n, d_cell, d_xi, d_S, stream=None):
    rc = lib().ecpic_deposit_device_noalloc(N, n, d_cell, d_xi, d_S, stream)
    if rc != ECPIC_OK:
        raise EcpicError(rc, "ecpic_deposit_device_noalloc")


def ecpic_philox_device(n, d_ctr, d_key, d_out, stream=None):
    rc = lib().ecpic_philox_device(n, d_ctr, d_key, d_out, stream)
    if rc != ECPIC_OK:
        raise EcpicError(rc, "ecpic_philox_device")


class Run:
    """One discharge on the GPU, driven through the C ABI."""

    def __init__(self, device=0, stream=None):
        self._L = lib()
        self.h = ecpic_create(device, stream)
        self.ns = 0
        self.N = 0
        self.scheme = ECPIC_SCHEME_EC
        self.tally = dict(TALLY_DEFAULT)

    @classmethod
    def from_config(cls, cfg, device=0, stream=None, sort_every=None, init=True):
        r = cls(device, stream)
        r.set_grid(cfg.edges, cfg.bc, cfg.v0, cfg.freq, cfg.phase, cfg.vdc)
        r.set_scheme(cfg.scheme)
        for s in cfg.species:
            r.add_species(s.q, s.m, s.w, s.capacity)
        if cfg.processes or cfg.n_gas:
            r.set_gas(cfg.n_gas, cfg.T_gas, cfg.m_gas)
        for p in cfg.processes:
            r.add_process(p.species, p.kind, p.threshold, p.dE, p.sigma, p.product)
        if sort_every:
            r.set_sort_every(sort_every)
        if getattr(cfg, "quiet", False):
            r.set_quiet_start(True)
        if getattr(cfg, "tallies", None):
            r.set_tallies(**cfg.tallies)
        if getattr(cfg, "rebalance", None):
            r.set_rebalance(**cfg.rebalance)
        if init:
            r.init(cfg.seed, cfg.dt, [s.n0 for s in cfg.species], [s.T_eV for s in cfg.species])
            if cfg.sample_every:
                r.reset_averages(cfg.sample_every)
        return r

    def close(self):
        if getattr(self, "h", None):
            self._L.ecpic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_grid(self, edges, bc=ECPIC_DIRICHLET_RF, v0=0.0, freq=0.0, phase=0.0, vdc=0.0):
        e = np.ascontiguousarray(edges, dtype=np.float64)
        _chk(self.h, self._L.ecpic_set_grid(self.h, _p(e), e.size, bc, v0, freq, phase, vdc),
             "ecpic_set_grid")
        self.N = e.size - 1

    def set_scheme(self, scheme):
        _chk(self.h, self._L.ecpic_set_scheme(self.h, scheme), "ecpic_set_scheme")
        self.scheme = scheme

    def add_species(self, q, m, w, capacity):
        out = C.c_int()
        _chk(self.h, self._L.ecpic_add_species(self.h, q, m, w, int(capacity), C.byref(out)),
             "ecpic_add_species")
        self.ns += 1
        return out.value

    def set_gas(self, n_g, T_g, m_g):
        _chk(self.h, self._L.ecpic_set_gas(self.h, n_g, T_g, m_g), "ecpic_set_gas")

    def add_process(self, species, kind, threshold, dE, sigma, product=-1):
        s = np.ascontiguousarray(sigma, dtype=np.float32)
        _chk(self.h, self._L.ecpic_add_process(self.h, species, kind, threshold, dE, s.size,
                                               _p(s), product), "ecpic_add_process")

    def init(self, seed, dt, n_per_species, T_eV):
        n = np.ascontiguousarray(n_per_species, dtype=np.int64)
        T = np.ascontiguousarray(T_eV, dtype=np.float64)
        _chk(self.h, self._L.ecpic_init(self.h, int(seed), dt, _p(n), _p(T)), "ecpic_init")

    def step(self, n=1):
        _chk(self.h, self._L.ecpic_step(self.h, int(n)), "ecpic_step")

    def sync(self, allow=()):
        rc = self._L.ecpic_sync(self.h)
        if rc in allow:
            return rc
        return _chk(self.h, rc, "ecpic_sync")

    def reset_averages(self, sample_every):
        _chk(self.h, self._L.ecpic_reset_averages(self.h, sample_every), "ecpic_reset_averages")

    def set_sort_every(self, k):
        _chk(self.h, self._L.ecpic_set_sort_every(self.h, k), "ecpic_set_sort_every")

    def sort_now(self):
        _chk(self.h, self._L.ecpic_sort_now(self.h), "ecpic_sort_now")

    def reserve(self, species, capacity):
        """Raise one species' particle capacity (keeps the run's state)."""
        _chk(self.h, self._L.ecpic_reserve(self.h, int(species), int(capacity)), "ecpic_reserve")

    def set_auto_grow(self, on=True):
        """Double a species' capacity when it is 3/4 full (checked every ~64 steps)."""
        _chk(self.h, self._L.ecpic_set_auto_grow(self.h, 1 if on else 0), "ecpic_set_auto_grow")

    def profile_step(self, n):
        ms = np.zeros(4)
        cnt = np.zeros(4, np.int64)
        _chk(self.h, self._L.ecpic_profile_step(self.h, int(n), _p(ms), _p(cnt)),
             "ecpic_profile_step")
        return dict(pass_ms=ms[0], field_ms=ms[1], sort_ms=ms[2], collide_ms=ms[3],
                    launches=cnt.tolist())

    def set_pass_grid(self, ctas):
        _chk(self.h, self._L.ecpic_set_pass_grid(self.h, int(ctas)), "ecpic_set_pass_grid")

    def set_rebalance(self, every, target, lo, hi, m0=1):
        """Particle rebalancing (before init): see ecpic_set_rebalance."""
        _chk(self.h, self._L.ecpic_set_rebalance(self.h, int(every), int(target), int(lo), int(hi),
                                                 int(m0)), "ecpic_set_rebalance")

    def rebalance_now(self):
        _chk(self.h, self._L.ecpic_rebalance_now(self.h), "ecpic_rebalance_now")

    def get_weights(self, species):
        n = C.c_int64()
        rc = self._L.ecpic_get_weights(self.h, species, None, 0, C.byref(n))
        if rc not in (ECPIC_OK, ECPIC_ERR_ARG):
            _chk(self.h, rc, "ecpic_get_weights")
        k = np.zeros(max(1, n.value), dtype=np.uint32)
        _chk(self.h, self._L.ecpic_get_weights(self.h, species, _p(k), k.size, C.byref(n)),
             "ecpic_get_weights")
        return k[: n.value]

    def set_weights(self, species, k):
        k = np.ascontiguousarray(k, dtype=np.uint32)
        _chk(self.h, self._L.ecpic_set_weights(self.h, species, _p(k), k.size), "ecpic_set_weights")

    def set_phase_timing(self, on=True):
        _chk(self.h, self._L.ecpic_set_phase_timing(self.h, 1 if on else 0), "ecpic_set_phase_timing")

    def phase_times(self):
        """Read and clear the per-phase device times of the timed steps."""
        return _phase_times(lambda *a: _chk(self.h, self._L.ecpic_phase_times(self.h, *a),
                                            "ecpic_phase_times"))

    def sort_state(self):
        k, since = C.c_int(), C.c_int()
        _chk(self.h, self._L.ecpic_sort_state(self.h, C.byref(k), C.byref(since)), "ecpic_sort_state")
        return dict(sort_every=k.value, since_sort=since.value)

    def set_quiet_start(self, quiet=True):
        _chk(self.h, self._L.ecpic_set_quiet_start(self.h, 1 if quiet else 0),
             "ecpic_set_quiet_start")

    def set_tallies(self, **kw):
        t = dict(TALLY_DEFAULT)
        t.update(kw)
        _chk(self.h, self._L.ecpic_set_tallies(self.h, t["eedf_center"], t["eedf_halfwidth"],
                                               t["eedf_dE"], t["eedf_bins"], t["iedf_dE"],
                                               t["iedf_bins"], t["iad_bins"]), "ecpic_set_tallies")
        self.tally = t

    def autotune(self, steps_per_trial=64, ks=None):
        k, g, ns = C.c_int(), C.c_int(), C.c_double()
        if ks is None:
            _chk(self.h, self._L.ecpic_autotune(self.h, int(steps_per_trial), C.byref(k), C.byref(g),
                                                C.byref(ns)), "ecpic_autotune")
        else:
            kk = np.ascontiguousarray(ks, dtype=np.int32)
            _chk(self.h, self._L.ecpic_autotune_ks(self.h, int(steps_per_trial), _p(kk), int(kk.size),
                                                   C.byref(k), C.byref(g), C.byref(ns)),
                 "ecpic_autotune_ks")
        return dict(sort_every=k.value, pass_ctas=g.value, ns_per_particle_step=ns.value)

    def nu_max(self, species):
        nu = C.c_double()
        t = C.c_uint32()
        _chk(self.h, self._L.ecpic_nu_max(self.h, species, C.byref(nu), C.byref(t)), "ecpic_nu_max")
        return nu.value, int(t.value)

    def get_particles(self, species):
        n = C.c_int64()
        rc = self._L.ecpic_get_particles(self.h, species, None, None, None, None, None, None, 0,
                                         C.byref(n))
        if rc not in (ECPIC_OK, ECPIC_ERR_ARG):
            _chk(self.h, rc, "ecpic_get_particles")
        m = n.value
        cell = np.zeros(m, np.int32)
        xi, vx, vy, vz = (np.zeros(m, np.float32) for _ in range(4))
        ids = np.zeros(m, np.uint64)
        _chk(self.h, self._L.ecpic_get_particles(self.h, species, _p(cell), _p(xi), _p(vx),
                                                 _p(vy), _p(vz), _p(ids), m, C.byref(n)),
             "ecpic_get_particles")
        return dict(cell=cell, xi=xi, vx=vx, vy=vy, vz=vz, id=ids)

    def set_particles(self, species, cell, xi, vx, vy, vz, ids):
        c = np.ascontiguousarray(cell, dtype=np.int32)
        f = [np.ascontiguousarray(a, dtype=np.float32) for a in (xi, vx, vy, vz)]
        i = np.ascontiguousarray(ids, dtype=np.uint64)
        _chk(self.h, self._L.ecpic_set_particles(self.h, species, _p(c), *[_p(a) for a in f], _p(i),
                                                 c.size), "ecpic_set_particles")

    def fields(self):
        phi = np.zeros(self.N + 1)
        E = np.zeros(self.N + 1 if self.scheme in (ECPIC_SCHEME_MC, ECPIC_SCHEME_MC2) else self.N,
                     np.float32)
        _chk(self.h, self._L.ecpic_get_fields(self.h, _p(phi), _p(E)), "ecpic_get_fields")
        return dict(phi=phi, E=E)

    def diagnostics(self, profiles=True):
        dg = ecpic_diag()
        arrs = _diag_arrays(dg, self.ns, self.N, self.tally) if profiles else None
        _chk(self.h, self._L.ecpic_diagnostics(self.h, C.byref(dg)), "ecpic_diagnostics")
        return _diag_dict(dg, self.ns, self.N, arrs)

def _diag_arrays(dg, ns, N, tally=None):
    t = TALLY_DEFAULT if tally is None else tally
    M = N + 1
    arrs = dict(density=np.zeros(ns * M), phi=np.zeros(M), temp_x=np.zeros(ns * M),
                temp_x_mom=np.zeros(ns * M), eedf=np.zeros(ns * t["eedf_bins"]),
                iedf=np.zeros(ns * t["iedf_bins"]), iad=np.zeros(ns * t["iad_bins"]),
                power=np.zeros(ns * N))
    for k, a in arrs.items():
        setattr(dg, k, _p(a))
    return arrs


def _diag_dict(dg, ns, N, arrs=None):
    out = dict(step=dg.step, time=dg.time, n_samples=dg.n_samples, fe=dg.fe,
               ke=np.array(dg.ke[:ns]), species=[])
    for s in range(ns):
        out["species"].append(dict(
            n=dg.n_live[s], absorbed_left=dg.absorbed[s][0], absorbed_right=dg.absorbed[s][1],
            births=dg.births[s], lost=dg.lost[s], candidates=dg.candidates[s],
            clamps=dg.clamps[s], collisions=list(dg.collisions[s])))
    for s in range(ns):
        out["species"][s]["impacts_dropped"] = dg.impacts_dropped[s]
        out["species"][s]["rb_merged"] = dg.rb_merged[s]
        out["species"][s]["rb_split"] = dg.rb_split[s]
        out["species"][s]["rb_skipped"] = dg.rb_skipped[s]
    if arrs:
        M = N + 1
        out["density"] = arrs["density"].reshape(ns, M)
        out["phi"] = arrs["phi"]
        out["Tx"] = arrs["temp_x"].reshape(ns, M)
        out["Tx_mom"] = arrs["temp_x_mom"].reshape(ns, M)
        out["eedf"] = arrs["eedf"].reshape(ns, dg.eedf_bins)
        out["iedf"] = arrs["iedf"].reshape(ns, dg.iedf_bins)
        out["iad"] = arrs["iad"].reshape(ns, dg.iad_bins)
        out["power"] = arrs["power"].reshape(ns, N)
        out["eedf_cells"] = (dg.eedf_cell0, dg.eedf_cell1)
        out["eedf_dE"], out["iedf_dE"] = dg.eedf_dE, dg.iedf_dE
    return out


class Engine:
    """Batched / served runs on one GPU (ecpic_engine_* of the C ABI)."""

    QUEUED, RESIDENT, FINISHED = 0, 1, 2

    def __init__(self, device=0, stream=None, mem_budget=0, max_slots=256, max_cells=1024,
                 species_per_run=2):
        self._L = lib()
        h = C.c_void_p()
        rc = self._L.ecpic_engine_create(C.byref(h), device, stream, int(mem_budget), max_slots,
                                         max_cells, species_per_run)
        if rc != ECPIC_OK:
            raise EcpicError(rc, "ecpic_engine_create")
        self.h = h
        self._meta = {}

    def close(self):
        if getattr(self, "h", None):
            self._L.ecpic_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, what):
        if rc != ECPIC_OK:
            raise EcpicError(rc, f"{what}: {self._L.ecpic_engine_last_error(self.h).decode()}")

    def submit(self, cfg, n_steps=None):
        keep = []
        rc = ecpic_run_config()
        e = np.ascontiguousarray(cfg.edges, dtype=np.float64)
        keep.append(e)
        rc.edges = _p(e)
        rc.n_edges = e.size
        rc.bc, rc.v0, rc.freq_hz, rc.phase_rad, rc.v_dc = cfg.bc, cfg.v0, cfg.freq, cfg.phase, cfg.vdc
        rc.scheme = cfg.scheme
        rc.n_species = len(cfg.species)
        for i, s in enumerate(cfg.species):
            rc.q[i], rc.m[i], rc.w[i] = s.q, s.m, s.w
            rc.capacity[i], rc.n_init[i], rc.T_eV[i] = s.capacity, s.n0, s.T_eV
        rc.n_gas = cfg.n_gas if cfg.processes else 0.0
        rc.T_gas, rc.m_gas = cfg.T_gas, cfg.m_gas
        procs = (ecpic_process_desc * max(1, len(cfg.processes)))()
        for i, p in enumerate(cfg.processes):
            sg = np.ascontiguousarray(p.sigma, dtype=np.float32)
            keep.append(sg)
            procs[i] = ecpic_process_desc(p.species, p.kind, p.threshold, p.dE, sg.size, _p(sg),
                                          p.product)
        rc.n_proc = len(cfg.processes)
        rc.procs = C.cast(procs, C.c_void_p)
        rc.seed, rc.dt, rc.sample_every = int(cfg.seed), cfg.dt, int(cfg.sample_every)
        rc.quiet_start = 1 if getattr(cfg, "quiet", False) else 0
        rb = getattr(cfg, "rebalance", None)
        if rb:
            rc.rb_every, rc.rb_target, rc.rb_lo, rc.rb_hi = (int(rb["every"]), int(rb["target"]),
                                                             int(rb["lo"]), int(rb["hi"]))
            rc.rb_m0 = int(rb.get("m0", 1))
        tally = dict(TALLY_DEFAULT)
        tally.update(getattr(cfg, "tallies", None) or {})
        for k, v in tally.items():
            setattr(rc, k, v)
        t = C.c_uint64()
        n = int(cfg.n_steps if n_steps is None else n_steps)
        self._chk(self._L.ecpic_engine_submit(self.h, C.byref(rc), n, C.byref(t)),
                  "ecpic_engine_submit")
        self._meta[t.value] = (len(cfg.species), cfg.N, tally)
        return t.value

    def pump(self, max_steps):
        r, q = C.c_int(), C.c_int()
        self._chk(self._L.ecpic_engine_pump(self.h, int(max_steps), C.byref(r), C.byref(q)),
                  "ecpic_engine_pump")
        return r.value, q.value

    def poll(self, ticket, diagnostics=False, profiles=False):
        st = C.c_int()
        steps, ps = C.c_int64(), C.c_int64()
        dg = ecpic_diag()
        ns, N, tally = self._meta.get(ticket, (0, 0, None))
        arrs = _diag_arrays(dg, ns, N, tally) if (diagnostics and profiles) else None
        self._chk(self._L.ecpic_engine_poll(self.h, ticket, C.byref(st),
                                            C.byref(dg) if diagnostics else None,
                                            C.byref(steps), C.byref(ps)), "ecpic_engine_poll")
        out = dict(state=st.value, steps=steps.value, particle_steps=ps.value)
        if diagnostics and st.value in (self.RESIDENT, self.FINISHED):
            out["diag"] = _diag_dict(dg, ns, N, arrs)
        return out

    def release(self, ticket):
        self._chk(self._L.ecpic_engine_release(self.h, ticket), "ecpic_engine_release")
        self._meta.pop(ticket, None)

    def stats(self):
        ps, rf, by = C.c_int64(), C.c_int64(), C.c_int64()
        self._chk(self._L.ecpic_engine_stats(self.h, C.byref(ps), C.byref(rf), C.byref(by)),
                  "ecpic_engine_stats")
        return dict(particle_steps=ps.value, runs_finished=rf.value, bytes_resident=by.value)

    def profile(self, n):
        ms = np.zeros(4)
        cnt = np.zeros(4, np.int64)
        self._chk(self._L.ecpic_engine_profile(self.h, int(n), _p(ms), _p(cnt)),
                  "ecpic_engine_profile")
        return dict(pass_ms=ms[0], field_ms=ms[1], sort_ms=ms[2], collide_ms=ms[3],
                    launches=cnt.tolist())

    def autotune(self, steps_per_trial=64, ks=None):
        k, g, ns = C.c_int(), C.c_int(), C.c_double()
        if ks is None:
            self._chk(self._L.ecpic_engine_autotune(self.h, int(steps_per_trial), C.byref(k),
                                                    C.byref(g), C.byref(ns)), "ecpic_engine_autotune")
        else:
            kk = np.ascontiguousarray(ks, dtype=np.int32)
            self._chk(self._L.ecpic_engine_autotune_ks(self.h, int(steps_per_trial), _p(kk),
                                                       int(kk.size), C.byref(k), C.byref(g),
                                                       C.byref(ns)), "ecpic_engine_autotune_ks")
        return dict(sort_every=k.value, pass_ctas=g.value, ns_per_particle_step=ns.value)

    def set_phase_timing(self, on=True):
        self._chk(self._L.ecpic_engine_set_phase_timing(self.h, 1 if on else 0),
                  "ecpic_engine_set_phase_timing")

    def phase_times(self):
        """Read and clear the per-phase device times of the timed steps."""
        return _phase_times(lambda *a: self._chk(self._L.ecpic_engine_phase_times(self.h, *a),
                                                 "ecpic_engine_phase_times"))

    def sort_state(self):
        k, since = C.c_int(), C.c_int()
        self._chk(self._L.ecpic_engine_sort_state(self.h, C.byref(k), C.byref(since)),
                  "ecpic_engine_sort_state")
        return dict(sort_every=k.value, since_sort=since.value)

    def tune(self, pass_ctas=0, sort_every=16):
        self._chk(self._L.ecpic_engine_tune(self.h, int(pass_ctas), int(sort_every)),
                  "ecpic_engine_tune")
