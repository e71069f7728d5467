"""Element-wise parity of the sampled moments (Sec. 3a: density, potential,
x temperature; the energy diagnostics) on one sample step from an identical
state, GPU through the C ABI against the FP64 oracle, node by node.

Bounds, from the arithmetic of the GPU path:
* density: the deposit is an integer sum of floor(xi 2^32) shares of the FP32
  offsets, which differ from the oracle's FP64 offsets by a few FP32
  roundings after the push, so |dn| <= 1e-5 n + (w / V_n) 2^-20 at every
  node, plus a whole particle's share w / V_n for each particle that one side
  absorbs at a wall and the other keeps (counted from the ids);
* potential (and the field energy): 1e-5 of the potential's scale (as the
  field parity), field energy to relative 1e-6;
* T_x and T_x of the averaged moments: the vx moments are FP32 products
  summed in FP32 per block and in FP64 across blocks; with a relative error
  eps <= 1e-5 on <v> and <v^2> the temperature m (<v^2> - <v>^2) / e is off
  by at most 3 eps m <v^2> / e (Cauchy-Schwarz), so
  |dT_n| <= 3e-5 m <v^2>_n / e, with <v^2>_n the CIC-weighted mean square
  of the oracle's particles at node n;
* kinetic energy of the sampled push: every term v^- v^+ + vy^2 + vz^2 is
  formed in FP32 (a few roundings) and the terms are summed in FP64 by quads,
  so relative 2e-6 per species.
Collisionless cases (EC, MC on uniform and doubling grids, EC2 and MC2 on a
uniform grid, a periodic EC case) compare everything; the collisional case
compares density, potential and the energies (the process choice of a
near-tie candidate may differ, which moves a velocity but no position).
"""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I
from helpers import require_gpu
from test_gpu_parity import _pair, _set_same_state, _small

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _node_v2(edges, bc, X, v):
    """CIC-weighted mean square of v at every node (for the temperature
    bound's scale), from particle positions X."""
    N = edges.size - 1
    j = np.clip(np.searchsorted(edges, X, side="right") - 1, 0, N - 1)
    xi = (X - edges[j]) / (edges[j + 1] - edges[j])
    D = np.zeros(N + 1)
    S2 = np.zeros(N + 1)
    np.add.at(D, j, 1 - xi)
    np.add.at(D, j + 1, xi)
    np.add.at(S2, j, (1 - xi) * v * v)
    np.add.at(S2, j + 1, xi * v * v)
    if bc == I.PERIODIC:
        D[0] += D[N]
        D[N] = D[0]
        S2[0] += S2[N]
        S2[N] = S2[0]
    return np.where(D > 0, S2 / np.maximum(D, 1e-300), 0.0)


def _volumes(edges, bc):
    dx = np.diff(edges)
    V = np.empty(edges.size)
    V[1:-1] = 0.5 * (dx[:-1] + dx[1:])
    if bc == I.PERIODIC:
        V[0] = V[-1] = 0.5 * (dx[0] + dx[-1])
    else:
        V[0], V[-1] = 0.5 * dx[0], 0.5 * dx[-1]
    return V


def _sample_step(cfg, tail=0.05):
    g, o = _pair(cfg)
    _set_same_state(cfg, g, o, tail=tail)
    g.reset_averages(1)
    o.reset_averages(1)
    g.step(1)
    g.sync()
    o.step(1)
    return g, o


def _only_counts(g, o, ns):
    out = []
    for s in range(ns):
        gi = g.get_particles(s)["id"]
        oi = o.get_particles(s)["id"]
        out.append(int(np.setxor1d(gi, oi).size))
    return out


def _check(cfg, g, o, temperatures=True):
    dg = g.diagnostics(profiles=True)
    ao = o.averages()
    assert dg["n_samples"] == 1 and ao["n_samples"] == 1
    edges, bc = cfg.edges, cfg.bc
    V = _volumes(edges, bc)
    ns = len(cfg.species)
    only = _only_counts(g, o, ns)
    report = {}
    for s, sp in enumerate(cfg.species):
        dn = np.abs(dg["density"][s] - ao["density"][s])
        share = sp.w / V
        tol = 1e-5 * np.abs(ao["density"][s]) + share * 2.0 ** -20 + only[s] * share
        assert np.all(dn <= tol), (s, int(np.argmax(dn - tol)), float(np.max(dn / np.maximum(tol, 1e-300))))
        report[f"density_{s}"] = float(np.max(dn / tol))
        if temperatures:
            p = o.get_particles(s)
            v2 = _node_v2(edges, bc, p["X"], p["vx"])
            scale = sp.m * v2 / I.QE
            for key in ("Tx", "Tx_mom"):
                dT = np.abs(dg[key][s] - ao[key][s])
                tolT = 3e-5 * scale + 1e-12
                assert np.all(dT <= tolT), (s, key, int(np.argmax(dT - tolT)),
                                            float(np.max(dT / tolT)))
                report[f"{key}_{s}"] = float(np.max(dT / tolT))
        ke_o = o.energy()[0][s]
        assert abs(dg["ke"][s] - ke_o) <= 2e-6 * abs(ke_o), (s, dg["ke"][s], ke_o)
        report[f"ke_{s}"] = abs(dg["ke"][s] / ke_o - 1.0)
    phi_scale = max(np.max(np.abs(ao["phi"])), 1e-3)
    dphi = np.abs(dg["phi"] - ao["phi"])
    assert np.all(dphi <= 1e-5 * phi_scale), float(np.max(dphi) / phi_scale)
    fe_o = o.energy()[1]
    assert abs(dg["fe"] - fe_o) <= 1e-6 * abs(fe_o) + 1e-30, (dg["fe"], fe_o)
    report["phi"] = float(np.max(dphi) / phi_scale)
    report["fe"] = abs(dg["fe"] / max(fe_o, 1e-300) - 1.0)
    return report


@pytest.mark.parametrize("scheme,grid", [(I.EC, "uniform"), (I.EC, "doubling"), (I.MC, "uniform"),
                                         (I.MC, "doubling"), (I.EC2, "uniform"), (I.MC2, "uniform")])
def test_sample_step_moments_match_oracle_node_by_node(scheme, grid):
    edges = None if grid == "uniform" else oracle.doubling_grid(128, 0.05, 0.01, 1, 8)
    cfg = _small(scheme=scheme, edges=edges, collisions=False, n=6000, seed=5)
    g, o = _sample_step(cfg)
    rep = _check(cfg, g, o)
    assert rep["density_0"] <= 1.0 and rep["density_1"] <= 1.0


def test_sample_step_moments_periodic():
    cfg = _small(scheme=I.EC, collisions=False, bc=I.PERIODIC, n=6000, seed=6)
    g, o = _sample_step(cfg)
    _check(cfg, g, o)


def test_sample_step_density_potential_energy_with_collisions():
    cfg = _small(scheme=I.EC, collisions=True, n=6000, seed=7)
    g, o = _sample_step(cfg)
    _check(cfg, g, o, temperatures=False)


def test_density_of_quiet_neutral_cold_load_is_n0_on_the_gpu():
    """The oracle's closed-form pin, on the GPU: evenly spaced electrons and
    ions at the same positions, zero temperature, no bias -- density n0 at
    every node (half-cell Dirichlet end nodes included) to the 2^-32 share
    quantum, zero temperature."""
    L, N, ppc, n0 = 0.05, 128, 8, 3.0e14
    cfg = I.ccp("quiet-cold", N=N, n0=n0, dt=1e-10, ppc=ppc, v0=0.0, p_mtorr=30.0, n_steps=3,
                seed=1, L=L, Te=0.0, Ti=0.0, collisions=False)
    cfg.quiet = True
    cfg.sample_every = 1
    from helpers import gpu_from_config
    g = gpu_from_config(cfg)
    g.step(3)
    g.sync()
    d = g.diagnostics(profiles=True)
    assert d["n_samples"] == 3
    for s in range(2):
        assert np.max(np.abs(d["density"][s] / n0 - 1.0)) < 1e-8, d["density"][s][:3]
        assert np.all(np.abs(d["Tx"][s]) < 1e-12)


def _set_sorted_state(cfg, g, o, seed=12, weights=False):
    """Cell-sorted particles, as the counting sort leaves them, most of them
    slow enough to stay in their cell over the step: whole warps then share a
    cell, so the sample step's warp-segmented sums carry most of the moments
    and of J.E; a 5 % tail of fast particles crosses cells, and those lanes
    add their own runs (the other path).  With weights, multipliers 1..16 on
    both sides."""
    rng = np.random.default_rng(seed)
    dx = np.diff(cfg.edges)
    for s, sp in enumerate(cfg.species):
        vth = np.sqrt(I.QE * (1.0 if s == 0 else 0.1) / sp.m)
        st = I.random_state(rng, cfg.N, sp.n0, vth, cells_per_step=2.5, dt=cfg.dt,
                            dx_min=dx.min(), tail=0.05, id_base=1000000 * s)
        order = np.argsort(st["cell"], kind="stable")
        st = {k: v[order] for k, v in st.items()}
        g.set_particles(s, st["cell"], st["xi"], st["vx"], st["vy"], st["vz"], st["id"])
        o.set_particles_cell(s, st["cell"], st["xi"], st["vx"], st["vy"], st["vz"], st["id"])
        if weights:
            k = rng.integers(1, 17, st["cell"].size).astype(np.uint32)
            g.set_weights(s, k)
            o.set_weights(s, k)


@pytest.mark.parametrize("scheme,grid,weights", [(I.EC, "uniform", False), (I.MC, "doubling", False),
                                                 (I.EC, "uniform", True), (I.EC2, "uniform", False)])
def test_sample_step_moments_on_cell_sorted_particles(scheme, grid, weights):
    edges = None if grid == "uniform" else oracle.doubling_grid(128, 0.05, 0.01, 1, 8)
    cfg = _small(scheme=scheme, edges=edges, collisions=False, n=20000, seed=8)
    if weights:
        cfg.rebalance = dict(every=0, target=512, lo=64, hi=1024, m0=16)
    g, o = _pair(cfg)
    _set_sorted_state(cfg, g, o, weights=weights)
    g.reset_averages(1)
    o.reset_averages(1)
    g.step(1)
    g.sync()
    o.step(1)
    rep = _check(cfg, g, o)
    assert rep["density_0"] <= 1.0 and rep["density_1"] <= 1.0
    # J.E of the sampled push per cell (the tally test's bound)
    d = g.diagnostics()
    t = o.tallies()
    for s in range(len(cfg.species)):
        gp, op = d["power"][s], t["power"][s]
        scale = np.abs(op).max()
        assert scale > 0
        np.testing.assert_allclose(gp, op, rtol=0, atol=2e-4 * scale)
