"""Pins for the oracle's sampled and time-averaged moments (Sec. 3a: density,
potential and the x temperature, the standard deviation of the velocity
distribution), against closed forms that do not come from the oracle:

* a quiet, neutral, cold load of n0 on a uniform, a doubling (Sec. 3c) and a
  periodic grid: the density diagnostic equals n0 at every node -- interior
  nodes, the half-cell Dirichlet end nodes and the merged periodic node --
  to FP64 rounding, and stays so when averaged over samples;
* no charge: the averaged potential is the straight line between the
  electrode values averaged over the sample levels t_k = k dt;
* three particles at known offsets: the node temperatures are the weighted
  population variances of their velocities with CIC weights (numpy's
  weighted covariance), m var / e;
* a drifting Maxwellian: T_x returns the set temperature within its sampling
  error and not the drift (m u^2 / e = 16 T here);
* two samples of the same spread at different drifts: T_x (mean of the
  per-sample temperatures) keeps the spread, T_x of the averaged moments adds
  m ((u1 - u2)/2)^2 / e (law of total variance).
"""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I

QE, ME = I.QE, I.ME


def _run(edges, bc=I.DIRICHLET, species=(), vdc=0.0, v0=0.0, freq=0.0, dt=1e-10, sample_every=1,
         quiet=False, n=None, T=None, seed=0):
    """An oracle run with the given species (q, m, w, cap) and no gas."""
    o = oracle.OracleRun()
    o.set_grid(edges, bc, v0, freq, 0.0, vdc)
    o.set_scheme(I.EC)
    for q, m, w, cap in species:
        o.add_species(q, m, w, cap)
    o.set_gas(0.0, 300.0, I.M_ION)
    o.reset_averages(sample_every)
    if quiet:
        o.set_quiet_start(True)
    ns = len(species)
    o.init(seed, dt, list(n) if n is not None else [0] * ns, list(T) if T is not None else [0.0] * ns)
    return o


@pytest.mark.parametrize("grid,bc", [("uniform", I.DIRICHLET), ("doubling", I.DIRICHLET),
                                     ("uniform", I.PERIODIC)])
def test_quiet_neutral_cold_load_density_is_n0_at_every_node(grid, bc):
    """Evenly spaced electrons and ions at the same positions, zero
    temperature: no charge, no field, no motion.  Every cell of width m dx_ref
    holds m ppc particles at offsets (k + 1/2)/(m ppc), so each node receives
    (m_left + m_right) ppc / 2 particles of CIC share over a control volume of
    (m_left + m_right) dx_ref / 2: the density is w ppc / dx_ref = n0 at every
    node, a half cell at a Dirichlet end node, the two end nodes merged when
    periodic."""
    L, n_ref, ppc, n0 = 0.05, 256, 8, 3.0e14
    if grid == "uniform":
        edges = I.uniform_edges(n_ref, L)
    else:
        edges = oracle.doubling_grid(n_ref, L, L / 8, 1, 4)
        assert edges.size - 1 < n_ref  # a real non-uniform grid
    n = ppc * n_ref
    w = n0 * L / n
    o = _run(edges, bc=bc, species=[(-QE, ME, w, n), (QE, I.M_ION, w, n)], quiet=True,
             n=[n, n], T=[0.0, 0.0])
    f = o.fields()
    assert np.all(f["Q"] == 0.0) and np.all(f["E"] == 0.0)
    o.step(3)
    a = o.averages()
    assert a["n_samples"] == 3
    for s in range(2):
        d = a["density"][s]
        assert np.max(np.abs(d / n0 - 1.0)) < 1e-12, (s, d[:3], d[-3:])
        assert np.all(a["Tx"][s] == 0.0)


def test_density_planted_end_volume_error_is_caught():
    """The same load read with full-cell end volumes would give n0/2 at the
    Dirichlet end nodes: the pin above separates the two readings."""
    L, N, ppc, n0 = 0.05, 64, 8, 3.0e14
    n = ppc * N
    w = n0 * L / n
    o = _run(I.uniform_edges(N, L), species=[(-QE, ME, w, n), (QE, I.M_ION, w, n)], quiet=True,
             n=[n, n], T=[0.0, 0.0])
    o.step(1)
    d = o.averages()["density"][0]
    dx = L / N
    # full-cell reading: w D / dx at the ends
    D_end = d[0] * (0.5 * dx) / w
    assert abs(w * D_end / dx / n0 - 0.5) < 1e-12
    assert abs(d[0] / n0 - 1.0) < 1e-12


@pytest.mark.parametrize("grid", ["uniform", "doubling"])
def test_averaged_potential_without_charge_is_the_electrode_line(grid):
    """No particles: phi_n = phi_0(t_k) (1 - x_n / L) at every sampled level
    k = 1..K (phi_0 = v_dc + v0 sin(2 pi f t_k), grounded at x = L), so the
    average is the line of the averaged electrode value."""
    L = 0.05
    edges = I.uniform_edges(40, L) if grid == "uniform" else oracle.doubling_grid(128, L, L / 8, 1, 4)
    v0, vdc, f, dt, K = 150.0, 20.0, 13.56e6, 1.0 / (40 * 13.56e6), 7
    o = _run(edges, species=[(-QE, ME, 1.0, 16)], v0=v0, vdc=vdc, freq=f, dt=dt, n=[0])
    o.step(K)
    a = o.averages()
    assert a["n_samples"] == K
    k = np.arange(1, K + 1)
    phi0 = np.mean(vdc + v0 * np.sin(2 * np.pi * f * k * dt))
    expect = phi0 * (1.0 - edges / L)
    assert np.max(np.abs(a["phi"] - expect)) < 1e-12 * (abs(vdc) + v0)


def _place(o, edges, species, cell, xi, vx, dt, vy=None, vz=None, ids=None):
    """Put particles so that after one push (no field) they sit at
    x[cell] + xi dx[cell] with velocity vx (the start wrapped into [0, L)
    on a periodic grid)."""
    dx = np.diff(edges)
    X1 = edges[cell] + xi * dx[cell]
    L = edges[-1]
    X0 = np.mod(X1 - vx * dt, L)
    X0[X0 >= L] = 0.0
    n = len(cell)
    vy = np.zeros(n) if vy is None else vy
    vz = np.zeros(n) if vz is None else vz
    ids = np.arange(n, dtype=np.uint64) if ids is None else ids
    o.set_particles(species, X0, vx, vy, vz, ids)


def test_three_particle_node_temperatures_are_weighted_variances():
    """Particles A (cell 1, xi 1/4), B (cell 1, xi 3/4), C (cell 2, xi 1/2):
    node 1 sees A, B with weights 3/4, 1/4; node 2 sees A, B, C with 1/4,
    3/4, 1/2; node 3 sees C alone (T = 0).  T_n = m var_w(vx) / e, the
    weighted population variance with the CIC shares as weights."""
    edges = I.uniform_edges(4, 0.04)
    dt = 1e-11
    o = _run(edges, bc=I.PERIODIC, species=[(-QE, ME, 1e-6, 8)], dt=dt, n=[0])
    v = np.array([1.0e6, -3.0e5, 2.2e6])
    _place(o, edges, 0, np.array([1, 1, 2]), np.array([0.25, 0.75, 0.5]), v, dt)
    o.step(1)
    T = o.averages()["Tx"][0]

    def var(vals, wts):
        return float(np.cov(np.asarray(vals), aweights=np.asarray(wts), bias=True)) * ME / QE

    assert T[0] == 0.0 and T[4] == 0.0
    assert np.isclose(T[1], var(v[:2], [0.75, 0.25]), rtol=1e-9)
    assert np.isclose(T[2], var(v, [0.25, 0.75, 0.5]), rtol=1e-9)
    assert abs(T[3]) <= 1e-9 * var(v, [0.25, 0.75, 0.5])
    # the same numbers from the two-point closed form a b (vA - vB)^2 / (a + b)^2
    assert np.isclose(T[1], 0.1875 * (v[0] - v[1]) ** 2 * ME / QE, rtol=1e-9)


def test_drifting_maxwellian_gives_its_temperature_not_its_drift():
    rng = np.random.default_rng(4)
    N, ppc, L, dt = 32, 4000, 0.032, 1e-12
    edges = I.uniform_edges(N, L)
    T0 = 3.0
    sd = np.sqrt(QE * T0 / ME)
    u = 4.0 * sd
    n = N * ppc
    o = _run(edges, bc=I.PERIODIC, species=[(-QE, ME, 1e-6, n)], dt=dt, n=[0])
    cell = rng.integers(0, N, n)
    xi = rng.random(n)
    vx = u + sd * rng.standard_normal(n)
    _place(o, edges, 0, cell, xi, vx, dt)
    o.step(1)
    a = o.averages()
    Tn = a["Tx"][0][:N]  # node N is node 0
    n_eff = ppc * 1.5  # (sum w)^2 / sum w^2 of uniform CIC shares: 2 ppc / (4/3)
    se = T0 * np.sqrt(2.0 / n_eff)
    assert np.all(np.abs(Tn - T0) < 5 * se), np.max(np.abs(Tn - T0)) / se
    assert abs(Tn.mean() - T0) < 4 * se / np.sqrt(N / 2)
    assert np.allclose(a["Tx_mom"][0], a["Tx"][0], rtol=1e-12)  # one sample
    drift_T = ME * u * u / QE
    assert drift_T > 10 * T0 and np.all(Tn < T0 + 0.5 * drift_T)


def test_two_sample_average_separates_tx_and_tx_of_averaged_moments():
    rng = np.random.default_rng(9)
    N, ppc, L, dt = 16, 500, 0.016, 1e-12
    edges = I.uniform_edges(N, L)
    n = N * ppc
    sd = np.sqrt(QE * 2.0 / ME)
    u1, u2 = 3.0e6, -1.0e6
    cell = rng.integers(0, N, n)
    xi = rng.random(n)
    z = rng.standard_normal(n)
    o = _run(edges, bc=I.PERIODIC, species=[(-QE, ME, 1e-6, n)], dt=dt, n=[0])
    for u in (u1, u2):
        _place(o, edges, 0, cell, xi, u + sd * z, dt)
        o.step(1)
    a = o.averages()
    assert a["n_samples"] == 2
    # per-sample temperature: the same deviates about either drift
    o1 = _run(edges, bc=I.PERIODIC, species=[(-QE, ME, 1e-6, n)], dt=dt, n=[0])
    _place(o1, edges, 0, cell, xi, u1 + sd * z, dt)
    o1.step(1)
    Ts = o1.averages()["Tx"][0]
    assert np.allclose(a["Tx"][0], Ts, rtol=1e-6)
    extra = ME * (0.5 * (u1 - u2)) ** 2 / QE
    assert np.allclose(a["Tx_mom"][0], Ts + extra, rtol=1e-6)
    assert extra > 10 * Ts.max()


def test_sample_step_kinetic_energy_without_field():
    """No field: the leapfrog-average kinetic energy of the sampled push is
    sum 1/2 m w (vx^2 + vy^2 + vz^2) of the loaded state."""
    rng = np.random.default_rng(2)
    edges = I.uniform_edges(8, 0.008)
    dt, w, n = 1e-12, 1e-6, 300
    o = _run(edges, bc=I.PERIODIC, species=[(-QE, ME, w, n)], dt=dt, n=[0])
    v = rng.normal(0, 1e6, (3, n))
    _place(o, edges, 0, rng.integers(0, 8, n), rng.random(n), v[0], dt, v[1], v[2])
    o.step(1)
    ke, fe = o.energy()
    assert np.isclose(ke[0], 0.5 * ME * w * np.sum(v * v), rtol=1e-12)
