"""ctypes binding of the plain FP64 C oracle (``ecpic_oracle.c``).

TEST INFRASTRUCTURE ONLY.  ``build()`` compiles the C source with gcc into
``oracle/libecpic_oracle.so`` (git-ignored) when it is missing or stale.
Every numeric routine lives in the C file; this module only marshals arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ecpic_oracle.c")
_HDR = os.path.join(_HERE, "ecpic_oracle.h")
_SO = os.path.join(_HERE, "libecpic_oracle.so")

ELASTIC, EXCITATION, IONIZATION, ION_ELASTIC, CX = 0, 1, 2, 3, 4
DIRICHLET, PERIODIC = 0, 1
EC, MC, EC2, MC2 = 0, 1, 2, 3  # EC2 / MC2: quadratic-spline deposit, linear face / quadratic node gather
MAX_SPECIES, MAX_PROC = 4, 8

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction) if needed."""
    stale = (not os.path.exists(_SO) or
             os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


def _load(path):
    L = C.CDLL(path)
    P = C.POINTER
    d, i32, i64, u32, u64 = C.c_double, C.c_int, C.c_int64, C.c_uint32, C.c_uint64
    vp = C.c_void_p
    sig = {
        "oracle_philox4x32_10": (None, [P(u32), P(u32), P(u32)]),
        "oracle_child_id": (u64, [u64, i64, u64]),
        "oracle_deposit_fixed": (i32, [i32, i64, vp, vp, vp]),
        "oracle_deposit_fixed2": (i32, [i32, i32, i64, vp, vp, vp]),
        "oracle_poisson_thomas": (i32, [i32, vp, vp, d, d, vp]),
        "oracle_poisson_dense": (i32, [i32, vp, vp, d, d, vp]),
        "oracle_field": (i32, [i32, vp, vp, i32, i32, vp]),
        "oracle_doubling_grid": (i32, [i32, d, d, i32, i32, vp, i32]),
        "oracle_create": (i32, [P(vp)]),
        "oracle_destroy": (None, [vp]),
        "oracle_set_grid": (i32, [vp, vp, i32, i32, d, d, d, d]),
        "oracle_set_scheme": (i32, [vp, i32]),
        "oracle_add_species": (i32, [vp, d, d, d, i64, P(i32)]),
        "oracle_set_gas": (i32, [vp, d, d, d]),
        "oracle_add_process": (i32, [vp, i32, i32, d, d, i32, vp, i32]),
        "oracle_init": (i32, [vp, u64, d, vp, vp]),
        "oracle_set_quiet_start": (i32, [vp, i32]),
        "oracle_set_tallies": (i32, [vp, d, d, d, i32, d, i32, i32]),
        "oracle_get_tally_shape": (i32, [vp, vp]),
        "oracle_get_tallies": (i64, [vp, vp, vp, vp, vp]),
        "oracle_set_particles": (i32, [vp, i32, vp, vp, vp, vp, vp, i64]),
        "oracle_get_particles": (i32, [vp, i32, vp, vp, vp, vp, vp, i64, P(i64)]),
        "oracle_set_particles_cell": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, i64]),
        "oracle_get_particles_cell": (i32, [vp, i32, vp, vp, i64, P(i64)]),
        "oracle_step": (i32, [vp, i64]),
        "oracle_set_step": (i32, [vp, i64]),
        "oracle_reset_averages": (i32, [vp, i32]),
        "oracle_get_counters": (i32, [vp, vp, i32]),
        "oracle_get_fields": (i32, [vp, vp, vp, vp]),
        "oracle_get_energy": (i32, [vp, vp, vp]),
        "oracle_get_averages": (i64, [vp, vp, vp, vp, vp]),
        "oracle_nu_max": (i32, [vp, i32, P(d), P(u32)]),
        "oracle_set_rebalance": (i32, [vp, i32, i32, i32, i32, u32]),
        "oracle_rebalance_now": (i32, [vp]),
        "oracle_get_weights": (i32, [vp, i32, vp, i64, P(i64)]),
        "oracle_set_weights": (i32, [vp, i32, vp, i64]),
        "oracle_get_rebalance_counters": (i32, [vp, vp]),
        "oracle_deposit_fixed_w": (i32, [i32, i64, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _chk(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def child_id(parent: int, step: int, tag: int) -> int:
    return int(lib().oracle_child_id(parent, step, tag))


def deposit_fixed(N, cell, xi, S=None):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    xi = np.ascontiguousarray(xi, dtype=np.float32)
    if S is None:
        S = np.zeros(N + 1, dtype=np.uint64)
    _chk(lib().oracle_deposit_fixed(N, cell.size, _ptr(cell), _ptr(xi), _ptr(S)),
         "oracle_deposit_fixed")
    return S


def deposit_fixed_w(N, cell, xi, k, S=None):
    """Weighted fixed-point CIC rule: S[cell] += k (2^32 - r), S[cell+1] += k r."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    xi = np.ascontiguousarray(xi, dtype=np.float32)
    k = np.ascontiguousarray(k, dtype=np.uint32)
    if S is None:
        S = np.zeros(N + 1, dtype=np.uint64)
    _chk(lib().oracle_deposit_fixed_w(N, cell.size, _ptr(cell), _ptr(xi), _ptr(k), _ptr(S)),
         "oracle_deposit_fixed_w")
    return S


def deposit_fixed2(N, bc, cell, xi, S=None):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    xi = np.ascontiguousarray(xi, dtype=np.float32)
    if S is None:
        S = np.zeros(N + 1, dtype=np.uint64)
    _chk(lib().oracle_deposit_fixed2(N, bc, cell.size, _ptr(cell), _ptr(xi), _ptr(S)),
         "oracle_deposit_fixed2")
    return S


def poisson_thomas(x, Q, phi0, phiN):
    x = np.ascontiguousarray(x, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    phi = np.zeros_like(x)
    _chk(lib().oracle_poisson_thomas(x.size - 1, _ptr(x), _ptr(Q), phi0, phiN, _ptr(phi)),
         "oracle_poisson_thomas")
    return phi


def poisson_dense(x, Q, phi0, phiN):
    x = np.ascontiguousarray(x, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    phi = np.zeros_like(x)
    _chk(lib().oracle_poisson_dense(x.size - 1, _ptr(x), _ptr(Q), phi0, phiN, _ptr(phi)),
         "oracle_poisson_dense")
    return phi


def field(x, phi, bc, scheme):
    x = np.ascontiguousarray(x, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    N = x.size - 1
    E = np.zeros(N if scheme == EC else N + 1)
    _chk(lib().oracle_field(N, _ptr(x), _ptr(phi), bc, scheme, _ptr(E)), "oracle_field")
    return E


def doubling_grid(n_ref, L, L_buff, dx_min, dx_max):
    cap = n_ref + 1
    e = np.zeros(cap)
    n = lib().oracle_doubling_grid(n_ref, L, L_buff, dx_min, dx_max, _ptr(e), cap)
    if n < 0:
        raise RuntimeError(f"oracle_doubling_grid failed with code {n}")
    return e[: n + 1].copy()


# ---------------------------------------------------------------- simulation
class OracleRun:
    """One discharge simulation held by the C oracle (host memory)."""

    def __init__(self):
        self._L = lib()
        h = C.c_void_p()
        _chk(self._L.oracle_create(C.byref(h)), "oracle_create")
        self.h = h
        self.N = 0
        self.ns = 0
        self.scheme = EC
        self.caps = []

    def close(self):
        if self.h:
            self._L.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_grid(self, edges, bc=DIRICHLET, v0=0.0, freq=0.0, phase=0.0, vdc=0.0):
        e = np.ascontiguousarray(edges, dtype=np.float64)
        _chk(self._L.oracle_set_grid(self.h, _ptr(e), e.size, bc, v0, freq, phase, vdc),
             "oracle_set_grid")
        self.N = e.size - 1
        self.edges = e.copy()

    def set_scheme(self, scheme):
        _chk(self._L.oracle_set_scheme(self.h, scheme), "oracle_set_scheme")
        self.scheme = scheme

    def add_species(self, q, m, w, capacity):
        out = C.c_int()
        _chk(self._L.oracle_add_species(self.h, q, m, w, int(capacity), C.byref(out)),
             "oracle_add_species")
        self.ns += 1
        self.caps.append(int(capacity))
        return out.value

    def set_gas(self, n_g, T_g, m_g):
        _chk(self._L.oracle_set_gas(self.h, n_g, T_g, m_g), "oracle_set_gas")

    def add_process(self, species, kind, threshold, dE, sigma, product=-1):
        s = np.ascontiguousarray(sigma, dtype=np.float32)
        _chk(self._L.oracle_add_process(self.h, species, kind, threshold, dE, s.size,
                                        _ptr(s), product), "oracle_add_process")

    def set_tallies(self, eedf_center=-1.0, eedf_halfwidth=0.5e-3, eedf_dE=0.5, eedf_bins=100,
                    iedf_dE=2.0, iedf_bins=256, iad_bins=90):
        _chk(self._L.oracle_set_tallies(self.h, eedf_center, eedf_halfwidth, eedf_dE, eedf_bins,
                                        iedf_dE, iedf_bins, iad_bins), "oracle_set_tallies")

    def tallies(self):
        sh = np.zeros(5, dtype=np.int32)
        _chk(self._L.oracle_get_tally_shape(self.h, _ptr(sh)), "oracle_get_tally_shape")
        ne, ni, na = int(sh[0]), int(sh[1]), int(sh[2])
        e = np.zeros(self.ns * ne)
        i = np.zeros(self.ns * ni)
        a = np.zeros(self.ns * na)
        p = np.zeros(self.ns * self.N)
        n = self._L.oracle_get_tallies(self.h, _ptr(e), _ptr(i), _ptr(a), _ptr(p))
        if n < 0:
            raise RuntimeError("oracle_get_tallies failed")
        return dict(n_samples=int(n), eedf=e.reshape(self.ns, ne), iedf=i.reshape(self.ns, ni),
                    iad=a.reshape(self.ns, na), power=p.reshape(self.ns, self.N),
                    eedf_cells=(int(sh[3]), int(sh[4])))

    def set_quiet_start(self, quiet=True):
        _chk(self._L.oracle_set_quiet_start(self.h, 1 if quiet else 0), "oracle_set_quiet_start")

    def init(self, seed, dt, n_per_species, T_eV):
        n = np.ascontiguousarray(n_per_species, dtype=np.int64)
        T = np.ascontiguousarray(T_eV, dtype=np.float64)
        _chk(self._L.oracle_init(self.h, int(seed), dt, _ptr(n), _ptr(T)), "oracle_init")

    def set_particles(self, species, X, vx, vy, vz, ids):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (X, vx, vy, vz)]
        i = np.ascontiguousarray(ids, dtype=np.uint64)
        _chk(self._L.oracle_set_particles(self.h, species, *[_ptr(v) for v in a], _ptr(i),
                                          a[0].size), "oracle_set_particles")

    def get_particles(self, species):
        cap = self.caps[species]
        X, vx, vy, vz = (np.zeros(cap) for _ in range(4))
        ids = np.zeros(cap, dtype=np.uint64)
        n = C.c_int64()
        _chk(self._L.oracle_get_particles(self.h, species, _ptr(X), _ptr(vx), _ptr(vy),
                                          _ptr(vz), _ptr(ids), cap, C.byref(n)),
             "oracle_get_particles")
        k = n.value
        return dict(X=X[:k], vx=vx[:k], vy=vy[:k], vz=vz[:k], id=ids[:k])

    def set_particles_cell(self, species, cell, xi, vx, vy, vz, ids):
        c = np.ascontiguousarray(cell, dtype=np.int32)
        f = [np.ascontiguousarray(v, dtype=np.float32) for v in (xi, vx, vy, vz)]
        i = np.ascontiguousarray(ids, dtype=np.uint64)
        _chk(self._L.oracle_set_particles_cell(self.h, species, _ptr(c), *[_ptr(v) for v in f],
                                               _ptr(i), c.size), "oracle_set_particles_cell")

    def get_particles_cell(self, species):
        cap = self.caps[species]
        cell = np.zeros(cap, dtype=np.int32)
        xi = np.zeros(cap)
        n = C.c_int64()
        _chk(self._L.oracle_get_particles_cell(self.h, species, _ptr(cell), _ptr(xi), cap,
                                               C.byref(n)), "oracle_get_particles_cell")
        k = n.value
        return cell[:k], xi[:k]

    def set_rebalance(self, every, target, lo, hi, m0=1):
        """Particle rebalancing (before init): see oracle_set_rebalance."""
        _chk(self._L.oracle_set_rebalance(self.h, int(every), int(target), int(lo), int(hi),
                                          int(m0)), "oracle_set_rebalance")

    def rebalance_now(self):
        rc = self._L.oracle_rebalance_now(self.h)
        _chk(rc, "oracle_rebalance_now")

    def get_weights(self, species):
        cap = self.caps[species]
        k = np.zeros(cap, dtype=np.uint32)
        n = C.c_int64()
        _chk(self._L.oracle_get_weights(self.h, species, _ptr(k), cap, C.byref(n)),
             "oracle_get_weights")
        return k[: n.value].copy()

    def set_weights(self, species, k):
        k = np.ascontiguousarray(k, dtype=np.uint32)
        _chk(self._L.oracle_set_weights(self.h, species, _ptr(k), k.size), "oracle_set_weights")

    def rebalance_counters(self):
        out = np.zeros(3 * MAX_SPECIES, dtype=np.int64)
        _chk(self._L.oracle_get_rebalance_counters(self.h, _ptr(out)),
             "oracle_get_rebalance_counters")
        return [dict(merged=int(out[3 * s]), split=int(out[3 * s + 1]), skipped=int(out[3 * s + 2]))
                for s in range(self.ns)]

    def step(self, n=1, allow_capacity=False):
        rc = self._L.oracle_step(self.h, int(n))
        if rc == -4 and allow_capacity:
            return rc
        _chk(rc, "oracle_step")
        return rc

    def set_step(self, k):
        """Time level k: the RF phase and the random stream follow it."""
        _chk(self._L.oracle_set_step(self.h, int(k)), "oracle_set_step")

    def reset_averages(self, sample_every):
        _chk(self._L.oracle_reset_averages(self.h, sample_every), "oracle_reset_averages")

    def counters(self):
        out = np.zeros(1 + 16 * MAX_SPECIES, dtype=np.int64)
        _chk(self._L.oracle_get_counters(self.h, _ptr(out), out.size), "oracle_get_counters")
        res = {"step": int(out[0]), "species": []}
        for s in range(self.ns):
            o = out[1 + 16 * s: 1 + 16 * (s + 1)]
            res["species"].append(dict(
                n=int(o[0]), absorbed_left=int(o[1]), absorbed_right=int(o[2]),
                births=int(o[3]), lost=int(o[4]), clamps=int(o[5]), candidates=int(o[6]),
                collisions=[int(v) for v in o[7:15]]))
        return res

    def fields(self):
        N = self.N
        phi = np.zeros(N + 1)
        E = np.zeros(N + 1 if self.scheme in (MC, MC2) else N)
        Q = np.zeros(N + 1)
        _chk(self._L.oracle_get_fields(self.h, _ptr(phi), _ptr(E), _ptr(Q)),
             "oracle_get_fields")
        return dict(phi=phi, E=E, Q=Q)

    def energy(self):
        ke = np.zeros(MAX_SPECIES)
        fe = C.c_double()
        _chk(self._L.oracle_get_energy(self.h, _ptr(ke), C.byref(fe)), "oracle_get_energy")
        return ke[: self.ns].copy(), fe.value

    def averages(self):
        N = self.N
        dens = np.zeros(self.ns * (N + 1))
        phi = np.zeros(N + 1)
        T = np.zeros(self.ns * (N + 1))
        Tm = np.zeros(self.ns * (N + 1))
        ns = self._L.oracle_get_averages(self.h, _ptr(dens), _ptr(phi), _ptr(T), _ptr(Tm))
        if ns < 0:
            raise RuntimeError("oracle_get_averages failed")
        sh = (self.ns, N + 1)
        return dict(n_samples=int(ns), density=dens.reshape(sh), phi=phi,
                    Tx=T.reshape(sh), Tx_mom=Tm.reshape(sh))

    def nu_max(self, species):
        nu = C.c_double()
        t = C.c_uint32()
        _chk(self._L.oracle_nu_max(self.h, species, C.byref(nu), C.byref(t)), "oracle_nu_max")
        return nu.value, int(t.value)
