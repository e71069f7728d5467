"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This module holds workload recipes only: the geometry, plasma, gas and
cross-section inputs of each discharge, the seeded run manifests of the batched
and served workloads, and seeded particle states for parity tests.  It holds
none of the method's arithmetic (no deposit, field, push or collision).

Helium-like discharge of Sec. 2b / Table 1 (L = 0.3 m, 13.56 MHz, 300 K gas),
with synthetic analytic cross sections in place of the Turner et al. tables
that this project does not have:
  e-n elastic    5e-20 m^2, constant
  excitation     1e-21 m^2 above 20 eV
  ionisation     25 eV threshold, 3e-21 (E-25)/75 up to 100 eV, then 3e-21*100/E
  ion-n elastic  2e-19 m^2, constant
  charge exch.   3e-19 m^2, constant
tabulated every 0.5 eV from 0 to 1000 eV (2001 entries).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# CODATA 2018 (input recipes only)
QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
TORR = 133.322368421

ELASTIC, EXCITATION, IONIZATION, ION_ELASTIC, CX = 0, 1, 2, 3, 4
DIRICHLET, PERIODIC = 0, 1
EC, MC, EC2, MC2 = 0, 1, 2, 3  # EC2 / MC2: quadratic-spline deposit, linear face / quadratic node gather

F_RF = 13.56e6
L_GAP = 0.3
T_GAS = 300.0
M_ION = 4.0 * AMU

DE_TABLE = 0.5
N_TABLE = 2001


@dataclasses.dataclass
class Species:
    q: float
    m: float
    w: float
    capacity: int
    n0: int
    T_eV: float


@dataclasses.dataclass
class Process:
    species: int
    kind: int
    threshold: float
    dE: float
    sigma: np.ndarray  # float32
    product: int = -1


@dataclasses.dataclass
class RunConfig:
    name: str
    edges: np.ndarray  # float64, N+1, edges[0] == 0
    bc: int
    v0: float
    freq: float
    phase: float
    vdc: float
    scheme: int
    species: List[Species]
    n_gas: float
    T_gas: float
    m_gas: float
    processes: List[Process]
    seed: int
    dt: float
    n_steps: int
    sample_every: int = 0
    quiet: bool = False  # loader: evenly spaced positions (quiet start)
    tallies: Optional[dict] = None  # diagnostic tally set-up (None: defaults)
    # particle rebalancing: dict(every, target, lo, hi, m0) or None (off)
    rebalance: Optional[dict] = None

    @property
    def N(self) -> int:
        return int(self.edges.size - 1)

    @property
    def n_particles(self) -> int:
        return int(sum(s.n0 for s in self.species))


# ------------------------------------------------------------ cross sections
def synthetic_cross_sections(dE: float = DE_TABLE, n: int = N_TABLE):
    E = np.arange(n, dtype=np.float64) * dE
    el = np.full(n, 5e-20)
    exc = np.where(E >= 20.0, 1e-21, 0.0)
    iz = np.where(E < 25.0, 0.0,
                  np.where(E <= 100.0, 3e-21 * (E - 25.0) / 75.0,
                           3e-21 * 100.0 / np.maximum(E, 1e-30)))
    ion_el = np.full(n, 2e-19)
    cx = np.full(n, 3e-19)
    f = lambda a: a.astype(np.float32)  # noqa: E731
    return dict(elastic=f(el), excitation=f(exc), ionization=f(iz),
                ion_elastic=f(ion_el), cx=f(cx))


def gas_density(p_mtorr: float, T: float = T_GAS) -> float:
    return p_mtorr * 1e-3 * TORR / (KB * T)


def uniform_edges(N: int, L: float) -> np.ndarray:
    e = np.arange(N + 1, dtype=np.float64) * (L / N)
    e[0] = 0.0
    e[-1] = L
    return e


def tanh_edges(N: int, L: float, edge_cell: float) -> np.ndarray:
    """x_i = (L/2)(1 + tanh(beta(2i/N - 1))/tanh(beta)), beta chosen so that the
    first cell has width edge_cell (bisection)."""
    def first(beta):
        return 0.5 * L * (1.0 + math.tanh(beta * (2.0 / N - 1.0)) / math.tanh(beta))
    lo, hi = 1e-6, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if first(mid) > edge_cell:
            lo = mid
        else:
            hi = mid
    beta = 0.5 * (lo + hi)
    i = np.arange(N + 1, dtype=np.float64)
    e = 0.5 * L * (1.0 + np.tanh(beta * (2.0 * i / N - 1.0)) / math.tanh(beta))
    e[0] = 0.0
    e[-1] = L
    return e


# ------------------------------------------------------------ discharges
def ccp(name: str, N: int, n0: float, dt: float, ppc: int, v0: float, p_mtorr: float,
        n_steps: int, seed: int = 0, scheme: int = EC, edges: Optional[np.ndarray] = None,
        L: float = L_GAP, Te: float = 2.0, Ti: float = 0.03, collisions: bool = True,
        headroom: float = 2.0, n_per_species: Optional[int] = None) -> RunConfig:
    """A two-species (electron, 4 amu ion) RF-CCP: grounded at x = L, RF at x = 0."""
    if edges is None:
        edges = uniform_edges(N, L)
    N = edges.size - 1
    L = float(edges[-1])
    np_s = int(n_per_species if n_per_species is not None else ppc * N)
    w = n0 * L / np_s
    cap = int(headroom * np_s) + 4096
    sp = [Species(-QE, ME, w, cap, np_s, Te), Species(QE, M_ION, w, cap, np_s, Ti)]
    procs: List[Process] = []
    ng = gas_density(p_mtorr)
    if collisions:
        xs = synthetic_cross_sections()
        procs = [
            Process(0, ELASTIC, 0.0, DE_TABLE, xs["elastic"]),
            Process(0, EXCITATION, 20.0, DE_TABLE, xs["excitation"]),
            Process(0, IONIZATION, 25.0, DE_TABLE, xs["ionization"], product=1),
            Process(1, ION_ELASTIC, 0.0, DE_TABLE, xs["ion_elastic"]),
            Process(1, CX, 0.0, DE_TABLE, xs["cx"]),
        ]
    return RunConfig(name=name, edges=edges, bc=DIRICHLET, v0=v0, freq=F_RF, phase=0.0,
                     vdc=0.0, scheme=scheme, species=sp, n_gas=ng, T_gas=T_GAS, m_gas=M_ION,
                     processes=procs, seed=seed, dt=dt, n_steps=n_steps)


def config_small(seed: int = 0, scheme: int = EC) -> RunConfig:
    """128 uniform cells, 64 particles/cell/species, 200 steps per RF period,
    300 V, 30 mTorr, n0 = 5e13 m^-3, 2000 steps."""
    return ccp("small-128", N=128, n0=5e13, dt=1.0 / (200 * F_RF), ppc=64, v0=300.0,
               p_mtorr=30.0, n_steps=2000, seed=seed, scheme=scheme)


def config_resolved(seed: int = 0, scheme: int = EC, periods: int = 50) -> RunConfig:
    """1024 uniform cells at dx = lambda_De (n0 = 1.288e15, Te = 2 eV),
    256 particles/cell/species (524,288 total), w_pe dt = 0.2, 300 V, 30 mTorr."""
    return ccp("resolved-1024", N=1024, n0=1.288e15, dt=1.0 / (750 * F_RF), ppc=256,
               v0=300.0, p_mtorr=30.0, n_steps=750 * periods, seed=seed, scheme=scheme)


def config_sweep(dx_over_lambda: int, seed: int = 0, scheme: int = EC) -> RunConfig:
    """The resolved plasma at dx = 2, 4, 8, 16 lambda_De (512..64 cells),
    particles per cell held at 256."""
    N = 1024 // dx_over_lambda
    return ccp(f"sweep-{N}", N=N, n0=1.288e15, dt=1.0 / (750 * F_RF), ppc=256, v0=300.0,
               p_mtorr=30.0, n_steps=750 * 50, seed=seed, scheme=scheme)


def config_tanh(seed: int = 0, scheme: int = EC, N: int = 114) -> RunConfig:
    """tanh-stretched grid with N cells, first cell 4 dx_ref (dx_ref = L/1024)."""
    e = tanh_edges(N, L_GAP, 4.0 * L_GAP / 1024)
    return ccp(f"tanh-{N}", N=N, n0=1.288e15, dt=1.0 / (750 * F_RF), ppc=0, v0=300.0,
               p_mtorr=30.0, n_steps=750 * 50, seed=seed, scheme=scheme, edges=e,
               n_per_species=256 * 1024 // 9)


def config_nonuniform(edges: np.ndarray, seed: int = 0, scheme: int = EC) -> RunConfig:
    """The resolved plasma on caller-provided (e.g. doubling) edges, with the
    particle count of a 9x reduced grid."""
    return ccp(f"grid-{edges.size - 1}", N=edges.size - 1, n0=1.288e15,
               dt=1.0 / (750 * F_RF), ppc=0, v0=300.0, p_mtorr=30.0, n_steps=750 * 50,
               seed=seed, scheme=scheme, edges=edges, n_per_species=256 * 1024 // 9)


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def growth_headroom(steps: int) -> float:
    """Particle capacity per species, as a multiple of the initial load, for a
    manifest run of ``steps`` steps.  The discharges grow by ionisation from
    n0 = 1e14; the fastest of the 256-run manifest has 1.1x its electrons
    after 256 steps, 2.05x after 1024 and 2.9x after 2048, so 2 + steps/500
    (at most 8) keeps about twice that margin."""
    return min(8.0, 2.0 + steps / 500.0)


def with_headroom(cfg: RunConfig, headroom: float) -> RunConfig:
    """Resize every species' capacity to ``headroom`` x its initial load
    (plus the loader's 4096 spare slots)."""
    for sp in cfg.species:
        sp.capacity = int(headroom * sp.n0) + 4096
    return cfg


def batched_manifest(n_runs: int = 256, seed: int = 0, steps: int = 4400,
                     scale: float = 1.0, headroom: Optional[float] = None) -> List[RunConfig]:
    """Independent CCP runs: cells ~ logU[64,1024], particles ~ logU[1e4,1e6]
    (split evenly between species), V0 ~ logU[100,500] V, p ~ logU[10,100] mTorr,
    dx ~ U[0.5,1.0] mm, n0 = 1e14, dt = 1/(400 f).  ``scale`` shrinks particle
    counts for quick tests.  Capacity: ``headroom`` x the initial load, by
    default ``growth_headroom(steps)`` so that no run fills it in ``steps``."""
    if headroom is None:
        headroom = growth_headroom(steps)
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(n_runs):
        N = int(round(_log_uniform(rng, 64, 1024)))
        npart = int(round(_log_uniform(rng, 1e4, 1e6) * scale))
        v0 = float(_log_uniform(rng, 100, 500))
        p = float(_log_uniform(rng, 10, 100))
        dx = float(rng.uniform(0.5e-3, 1.0e-3))
        L = N * dx
        nps = max(npart // 2, 16)
        cfg = ccp(f"batch-{r}", N=N, n0=1e14, dt=1.0 / (400 * F_RF), ppc=0, v0=v0,
                  p_mtorr=p, n_steps=steps, seed=seed * 1000003 + r, L=L,
                  n_per_species=nps, headroom=headroom)
        runs.append(cfg)
    return runs


def appendix_b_sweep(ratios=(0.5, 1.0, 2.0, 4.0, 8.0, 16.0), ppc: int = 64, N: int = 2048,
                     steps: int = 100_000, seed: int = 0, schemes=(EC, MC),
                     sample_every: int = 1000, quiet: bool = True) -> List[RunConfig]:
    """App. B heating-rate sweep: collisionless periodic electrons on an
    immobile neutralising background with the Table 1 plasma (n0 = 7e15 m^-3,
    Te = 2.585 eV), N cells of dx = r * lambda_De (L grows with r),
    dt = 0.1/w_pe, 10,000/w_pe = 100,000 steps; one run per (scheme, r),
    energies sampled every `sample_every` steps.  Quiet start by default: a
    random load at dx >> lambda_De starts with long-wavelength charge noise
    whose field energy exceeds the kinetic energy and relaxes into it."""
    runs = []
    for scheme in schemes:
        for i, r in enumerate(ratios):
            c = periodic_plasma(N=N, dx_lambda=float(r), ppc=ppc, dt_wpe=0.1, n_steps=steps,
                                seed=seed * 1000 + 10 * i + scheme, scheme=scheme,
                                n0=7e15, Te=2.585, quiet=quiet)
            c.name = f"appB-{'EC' if scheme == EC else 'MC'}-dx{r:g}"
            c.sample_every = sample_every
            runs.append(c)
    return runs


@dataclasses.dataclass
class Request:
    arrival: float  # seconds after the stream starts
    config: RunConfig


def served_stream(n_requests: int = 2000, seed: int = 1, rate: float = 1.0,
                  scale: float = 1.0, period_range=(5, 50)) -> List[Request]:
    """Poisson arrivals (rate per second) of CCP runs drawn as in
    ``batched_manifest``, each for U{5..50} RF periods of 400 steps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    base = batched_manifest(n_requests, seed=seed + 7, steps=1, scale=scale)
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        periods = int(rng.integers(period_range[0], period_range[1] + 1))
        cfg = with_headroom(base[i], growth_headroom(400 * periods))
        cfg.n_steps = 400 * periods
        cfg.name = f"req-{i}"
        out.append(Request(arrival=t, config=cfg))
    return out


# ------------------------------------------------------------ particle states
def random_state(rng: np.random.Generator, N: int, n: int, vth: float, cells_per_step: float,
                 dt: float, dx_min: float, tail: float = 0.02, near_face: float = 0.01,
                 id_base: int = 0):
    """A particle state in cell-relative form (int32 cell, float32 xi in [0,1),
    float32 velocities, unique uint64 ids): Maxwellian core of thermal speed
    ``vth``, a fraction ``tail`` of fast particles that cross several cells,
    and a fraction ``near_face`` placed within a few ulps of a cell face."""
    cell = rng.integers(0, N, n).astype(np.int32)
    xi = rng.random(n).astype(np.float32)
    k = int(n * near_face)
    if k:
        idx = rng.choice(n, k, replace=False)
        xi[idx[: k // 2]] = np.float32(1.0) - np.float32(2.0 ** -24) * rng.integers(
            1, 5, k // 2).astype(np.float32)
        xi[idx[k // 2:]] = np.float32(2.0 ** -24) * rng.integers(0, 4, k - k // 2).astype(
            np.float32)
    xi = np.minimum(xi, np.float32(1.0 - 2.0 ** -24)).astype(np.float32)
    v = rng.normal(0.0, vth, (3, n))
    m = int(n * tail)
    if m:
        idx = rng.choice(n, m, replace=False)
        fast = cells_per_step * dx_min / dt
        v[0, idx] = rng.uniform(-fast, fast, m)
    ids = (np.uint64(id_base) + rng.permutation(np.arange(n, dtype=np.uint64) * np.uint64(3)
                                                + np.uint64(11))).astype(np.uint64)
    return dict(cell=cell, xi=xi, vx=v[0].astype(np.float32), vy=v[1].astype(np.float32),
                vz=v[2].astype(np.float32), id=ids)


def periodic_plasma(N: int = 64, dx_lambda: float = 4.0, ppc: int = 64, dt_wpe: float = 0.1,
                    n_steps: int = 1000, seed: int = 0, scheme: int = EC, ions: bool = False,
                    n0: float = 1e14, Te: float = 2.0, Ti: float = 0.5,
                    quiet: bool = False) -> RunConfig:
    """Collisionless periodic Maxwellian of App. B: electrons (and optionally
    mobile ions) on a uniform neutralising background, dx = dx_lambda * lambda_De,
    dt = dt_wpe / w_pe."""
    lam = math.sqrt(EPS0 * Te / (n0 * QE))
    wpe = math.sqrt(n0 * QE ** 2 / (EPS0 * ME))
    L = N * dx_lambda * lam
    npart = N * ppc
    w = n0 * L / npart
    sp = [Species(-QE, ME, w, npart, npart, Te)]
    if ions:
        sp.append(Species(QE, M_ION, w, npart, npart, Ti))
    return RunConfig(name=f"periodic-{N}", edges=uniform_edges(N, L), bc=PERIODIC, v0=0.0,
                     freq=0.0, phase=0.0, vdc=0.0, scheme=scheme, species=sp, n_gas=0.0,
                     T_gas=T_GAS, m_gas=M_ION, processes=[], seed=seed, dt=dt_wpe / wpe,
                     n_steps=n_steps, quiet=quiet)
