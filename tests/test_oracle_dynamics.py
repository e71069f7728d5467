"""Pins for the oracle's time step: leapfrog push (Eq. 8-9) against the exact
constant-acceleration orbit, EC gather (Eq. 6-7), momentum conservation of the
MC scheme and energy conservation of the EC scheme on periodic grids
(Sec. 1 and App. B), wall absorption, and independence of particle order."""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I
from helpers import oracle_from_config


def _single(scheme, X0, v0x, V, N=32, L=0.05, dt=1e-10, edges=None):
    o = oracle.OracleRun()
    e = I.uniform_edges(N, L) if edges is None else edges
    o.set_grid(e, oracle.DIRICHLET, v0=0.0, freq=0.0, phase=0.0, vdc=V)
    o.set_scheme(scheme)
    o.add_species(-I.QE, I.ME, 0.0, 4)  # zero weight: no self field
    o.init(0, dt, [0], [0.0])
    o.set_particles(0, [X0], [v0x], [3.0], [-4.0], np.array([7], np.uint64))
    return o


@pytest.mark.parametrize("scheme", [oracle.EC, oracle.MC])
@pytest.mark.parametrize("grid", ["uniform", "doubling"])
def test_push_exact_in_uniform_field(scheme, grid):
    """Charge-free gap with phi_0 = V, phi_L = 0: E = V/L everywhere and the
    leapfrog orbit is X^k = X^0 + k dt v^{-1/2} + a dt^2 k(k+1)/2 exactly."""
    L, V, dt = 0.05, 20.0, 1e-10
    edges = None if grid == "uniform" else oracle.doubling_grid(64, L, 0.01, 1, 4)
    X0, u0 = 0.02, 2.0e5
    o = _single(scheme, X0, u0, V, L=L, dt=dt, edges=edges)
    a = -I.QE / I.ME * (V / L)
    for k in range(1, 41):
        o.step(1)
        p = o.get_particles(0)
        if p["X"].size == 0:
            break
        X = X0 + k * dt * u0 + a * dt * dt * k * (k + 1) / 2
        v = u0 + k * a * dt
        assert np.isclose(p["X"][0], X, rtol=1e-12, atol=1e-15)
        assert np.isclose(p["vx"][0], v, rtol=1e-12, atol=1e-9)
        assert p["vy"][0] == 3.0 and p["vz"][0] == -4.0


def test_ec_gather_uses_cell_face_field():
    """Eq. 6-7: a probe at rest in cell j gains exactly (q/m) E_j dt, with
    E_j = -(phi_{j+1}-phi_j)/dx_j from the charge of other particles."""
    rng = np.random.default_rng(2)
    e = oracle.doubling_grid(128, 0.02, 0.003, 1, 4)
    N = e.size - 1
    o = oracle.OracleRun()
    o.set_grid(e, oracle.DIRICHLET, vdc=5.0)
    o.set_scheme(oracle.EC)
    o.add_species(I.QE, I.M_ION, 1e9, 2000)
    o.add_species(-I.QE, I.ME, 0.0, 200)
    o.init(0, 1e-10, [0, 0], [0.0, 0.0])
    n = 1500
    X = rng.uniform(0, 0.02, n)
    z = np.zeros(n)
    o.set_particles(0, X, z, z, z, np.arange(n, dtype=np.uint64))
    probes = np.array([0.001, 0.0051, 0.0099, 0.0123, 0.019])
    zp = np.zeros(probes.size)
    o.set_particles(1, probes, zp, zp, zp, np.arange(probes.size, dtype=np.uint64))
    f = o.fields()
    o.step(1)
    p = o.get_particles(1)
    for X0, v in zip(probes, p["vx"]):
        j = np.searchsorted(e, X0, side="right") - 1
        Ej = -(f["phi"][j + 1] - f["phi"][j]) / (e[j + 1] - e[j])
        assert np.isclose(v, -I.QE / I.ME * Ej * 1e-10, rtol=1e-12)


def test_mc_gather_is_cic_of_node_field():
    rng = np.random.default_rng(3)
    e = I.uniform_edges(64, 0.02)
    o = oracle.OracleRun()
    o.set_grid(e, oracle.DIRICHLET, vdc=5.0)
    o.set_scheme(oracle.MC)
    o.add_species(I.QE, I.M_ION, 1e9, 2000)
    o.add_species(-I.QE, I.ME, 0.0, 200)
    o.init(0, 1e-10, [0, 0], [0.0, 0.0])
    X = rng.uniform(0, 0.02, 1000)
    z = np.zeros(1000)
    o.set_particles(0, X, z, z, z, np.arange(1000, dtype=np.uint64))
    probes = np.array([0.0007, 0.0101, 0.0199])
    zp = np.zeros(3)
    o.set_particles(1, probes, zp, zp, zp, np.arange(3, dtype=np.uint64))
    E = o.fields()["E"]
    o.step(1)
    p = o.get_particles(1)
    for X0, v in zip(probes, p["vx"]):
        j = int(X0 // (0.02 / 64))
        xi = (X0 - e[j]) / (e[j + 1] - e[j])
        Ei = (1 - xi) * E[j] + xi * E[j + 1]
        assert np.isclose(v, -I.QE / I.ME * Ei * 1e-10, rtol=1e-10)


def _periodic_plasma(scheme, N, dx_lambda, ppc, dt_wpe, seed, ions=False):
    n0, Te = 1e14, 2.0
    lam = np.sqrt(I.EPS0 * Te / (n0 * I.QE))
    wpe = np.sqrt(n0 * I.QE ** 2 / (I.EPS0 * I.ME))
    L = N * dx_lambda * lam
    o = oracle.OracleRun()
    o.set_grid(I.uniform_edges(N, L), oracle.PERIODIC)
    o.set_scheme(scheme)
    npart = N * ppc
    w = n0 * L / npart
    o.add_species(-I.QE, I.ME, w, npart)
    if ions:
        o.add_species(I.QE, I.M_ION, w, npart)
    o.init(seed, dt_wpe / wpe, [npart] + ([npart] if ions else []),
           [Te] + ([0.5] if ions else []))
    return o


def test_mc_momentum_conserved_uniform_periodic():
    """MC-PIC on a uniform periodic grid conserves total momentum to round-off
    (Sec. 1): CIC gather is the transpose of the CIC deposit."""
    o = _periodic_plasma(oracle.MC, 32, 3.0, 64, 0.2, seed=4, ions=True)
    masses = [I.ME, I.M_ION]

    def mom():
        tot, scale = 0.0, 0.0
        for s in range(2):
            v = o.get_particles(s)["vx"]
            tot += masses[s] * v.sum()
            scale += masses[s] * np.abs(v).sum()
        return tot, scale
    p0, sc = mom()
    for _ in range(60):
        o.step(1)
    p1, _ = mom()
    assert abs(p1 - p0) <= 1e-11 * sc
    # the EC scheme does not conserve it (Sec. 1)
    o2 = _periodic_plasma(oracle.EC, 32, 3.0, 64, 0.2, seed=4, ions=True)
    q0 = sum(masses[s] * o2.get_particles(s)["vx"].sum() for s in range(2))
    o2.step(60)
    q1 = sum(masses[s] * o2.get_particles(s)["vx"].sum() for s in range(2))
    assert abs(q1 - q0) > 1e3 * 1e-11 * sc


def _energy_error(scheme, dt_wpe, T_wpe, seed, dx_lambda=4.0, ppc=512, N=64):
    o = _periodic_plasma(scheme, N, dx_lambda, ppc, dt_wpe, seed)
    W = []
    for _ in range(int(round(T_wpe / dt_wpe))):
        o.step(1)
        ke, fe = o.energy()
        W.append(ke.sum() + fe)
    W = np.array(W)
    return np.max(np.abs(W - W[0])) / W[0]


def test_ec_energy_converges_with_dt():
    """Collisionless periodic Maxwellian at dx = 4 lambda_De: the EC total
    energy error over 50/w_pe falls about 4x when dt halves (0.2 -> 0.1/w_pe),
    the second-order regime above the finite-particle floor."""
    r = []
    for seed in (5, 6):
        a = _energy_error(oracle.EC, 0.2, 50.0, seed)
        b = _energy_error(oracle.EC, 0.1, 50.0, seed)
        r.append(a / b)
        assert b < 1e-4
    assert np.mean(r) >= 3.0


def test_mc_heats_where_ec_does_not():
    """App. B: at dx = 8 lambda_De the MC scheme heats (finite-grid instability)
    while the EC error stays small."""
    ec = _energy_error(oracle.EC, 0.1, 1000.0, 1, dx_lambda=8.0, ppc=64)
    mc = _energy_error(oracle.MC, 0.1, 1000.0, 1, dx_lambda=8.0, ppc=64)
    assert mc > 0.05
    assert mc > 8 * ec


def test_wall_absorption_and_counts():
    e = I.uniform_edges(16, 0.01)
    o = oracle.OracleRun()
    o.set_grid(e, oracle.DIRICHLET)
    o.add_species(-I.QE, I.ME, 0.0, 8)
    o.init(0, 1e-9, [0], [0.0])
    X = np.array([1e-6, 0.01 - 1e-6, 0.005, 0.0003])
    vx = np.array([-2e3, 2e3, 0.0, -0.2e6])
    z = np.zeros(4)
    o.set_particles(0, X, vx, z, z, np.arange(4, dtype=np.uint64))
    o.step(1)
    c = o.counters()["species"][0]
    assert (c["absorbed_left"], c["absorbed_right"], c["n"]) == (1, 1, 2)
    # a particle landing exactly on x = 0 is absorbed (X <= 0)
    o.set_particles(0, [0.0005], [-0.0005 / 1e-9], [0.0], [0.0], np.array([9], np.uint64))
    o.step(1)
    assert o.counters()["species"][0]["absorbed_left"] == 2


def test_result_independent_of_particle_order():
    """Random numbers are keyed on (particle id, step), so permuting the arrays
    permutes the result; only the FP64 summation order of the deposit changes,
    which moves values at round-off level."""
    cfg = I.config_small()
    cfg.species[0].n0 = cfg.species[1].n0 = 3000
    a = oracle_from_config(cfg)
    b = oracle_from_config(cfg)
    rng = np.random.default_rng(0)
    for s in range(2):
        p = a.get_particles(s)
        perm = rng.permutation(p["X"].size)
        b.set_particles(s, *(p[k][perm] for k in ("X", "vx", "vy", "vz", "id")))
    a.step(60)
    b.step(60)
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
        assert np.array_equal(pa["id"][ia], pb["id"][ib])
        for k in ("X", "vx", "vy", "vz"):
            assert np.allclose(pa[k][ia], pb[k][ib], rtol=1e-8, atol=0)
    assert a.counters() == b.counters()
