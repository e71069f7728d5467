"""Pins for the oracle's higher-order schemes on uniform grids: EC2 (quadratic-
spline charge deposit, field interpolated one order lower, i.e. linearly
between faces: the EC construction of Sec. 2a carried one order up) and its
momentum-conserving partner MC2 (the same deposit and a quadratic-spline
gather of the centred node field):

* fixed-point quadratic shares: exact integers within one 2^-32 quantum of
  the B-spline weights, exactly 2^32 per particle (charge conserved also at
  Dirichlet walls, where the share beyond the wall folds into the wall node),
  periodic wrap;
* the gathered field is -dPhi/dX of the quadratic-spline potential
  Phi(X) = sum_n phi_n S2(X/dx - n) (ghost node beyond a wall = wall node):
  the EC property that makes the scheme energy conserving;
* energy error second order in dt on a periodic Maxwellian, no grid heating at
  dx = 8 lambda_De where MC heats (App. B, quiet start);
* MC2 conserves total momentum on a uniform periodic grid to round-off (its
  gather is the transpose of the deposit, folds included), EC2 does not; MC2
  heats at dx = 8 lambda_De, less than MC, while EC2 does not."""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I
from helpers import oracle_from_config

TWO32 = 2.0 ** 32


def _spline_shares(xi):
    xi = np.asarray(xi, np.float64)
    u = np.where(xi < 0.5, xi, xi - 1.0)
    return 0.5 * (0.5 - u) ** 2, 0.75 - u * u, 0.5 * (0.5 + u) ** 2


@pytest.mark.parametrize("bc", [oracle.DIRICHLET, oracle.PERIODIC])
def test_fixed2_shares_exact_and_conserving(bc):
    rng = np.random.default_rng(8)
    N, n = 16, 400
    cell = rng.integers(0, N, n).astype(np.int32)
    xi = rng.random(n).astype(np.float32)
    edge = np.array([0.0, 0.5, np.nextafter(np.float32(0.5), np.float32(0)), 1 - 2.0 ** -24,
                     2.0 ** -30], np.float32)
    xi[:edge.size] = edge
    cell[:edge.size] = [0, N - 1, 0, N - 1, 3]
    S = oracle.deposit_fixed2(N, bc, cell, xi)
    assert int(S[:N].sum(dtype=np.uint64)) + (int(S[N]) if bc == oracle.DIRICHLET else 0) == n * 2 ** 32
    if bc == oracle.PERIODIC:
        assert S[N] == S[0]
    # one particle at a time against the B-spline weights
    a, m, b = _spline_shares(xi)
    for k in range(n):
        Sk = oracle.deposit_fixed2(N, bc, cell[k:k + 1], xi[k:k + 1]).astype(np.float64)
        n0 = cell[k] + (0 if xi[k] < 0.5 else 1)
        want = np.zeros(N + 1)
        for node, w in ((n0 - 1, a[k]), (n0, m[k]), (n0 + 1, b[k])):
            if bc == oracle.PERIODIC:
                node %= N
            else:
                node = min(max(node, 0), N)
            want[node] += w * TWO32
        if bc == oracle.PERIODIC:
            want[N] = want[0]
        assert np.all(np.abs(Sk - want) <= 2.0), (k, cell[k], xi[k])


def test_ec2_needs_a_uniform_grid():
    o = oracle.OracleRun()
    o.set_grid(oracle.doubling_grid(128, 0.02, 0.003, 1, 4), oracle.DIRICHLET)
    with pytest.raises(RuntimeError):
        o.set_scheme(oracle.EC2)


@pytest.mark.parametrize("bc", [oracle.DIRICHLET, oracle.PERIODIC])
def test_ec2_gather_is_derivative_of_quadratic_potential(bc):
    rng = np.random.default_rng(6)
    N, L = 32, 0.02
    e = I.uniform_edges(N, L)
    dx = L / N
    o = oracle.OracleRun()
    o.set_grid(e, bc, vdc=5.0 if bc == oracle.DIRICHLET else 0.0)
    o.set_scheme(oracle.EC2)
    o.add_species(I.QE, I.M_ION, 1e9, 2000)
    o.add_species(-I.QE, I.ME, 0.0, 200)
    o.init(0, 1e-10, [0, 0], [0.0, 0.0])
    n = 1200
    X = rng.uniform(0, L, n)
    z = np.zeros(n)
    o.set_particles(0, X, z, z, z, np.arange(n, dtype=np.uint64))
    probes = np.array([0.2, 0.45, 0.55, 3.3, 7.5, 15.49, 15.51, 30.9, 31.6]) * dx
    zp = np.zeros(probes.size)
    o.set_particles(1, probes, zp, zp, zp, np.arange(probes.size, dtype=np.uint64))
    phi = o.fields()["phi"]
    o.step(1)
    v = o.get_particles(1)["vx"]

    def S2(t):
        t = np.abs(t)
        return np.where(t <= 0.5, 0.75 - t * t, np.where(t <= 1.5, 0.5 * (1.5 - t) ** 2, 0.0))

    def Phi(Xp):
        p = Xp / dx
        tot = 0.0
        for n_ in range(-1, N + 2):
            if bc == oracle.PERIODIC:
                ph = phi[n_ % N]
            else:
                ph = phi[min(max(n_, 0), N)]  # ghost node = wall node
            tot += ph * S2(p - n_)  # periodic: nodes -1, N, N+1 are images
        return tot

    h = 1e-7 * dx
    for X0, v0 in zip(probes, v):
        Ei = -(Phi(X0 + h) - Phi(X0 - h)) / (2 * h)
        assert np.isclose(v0, -I.QE / I.ME * Ei * 1e-10, rtol=1e-6, atol=1e-9 * abs(v).max()), X0


def test_ec2_charge_conserved_at_walls():
    rng = np.random.default_rng(2)
    N, L = 16, 0.01
    o = oracle.OracleRun()
    o.set_grid(I.uniform_edges(N, L), oracle.DIRICHLET)
    o.set_scheme(oracle.EC2)
    o.add_species(I.QE, I.M_ION, 3e9, 500)
    o.init(0, 1e-10, [0], [0.0])
    X = np.concatenate([rng.uniform(0, 0.5 * L / N, 50), rng.uniform(0, L, 200),
                        L - rng.uniform(0, 0.5 * L / N, 50)])
    z = np.zeros(X.size)
    o.set_particles(0, X, z, z, z, np.arange(X.size, dtype=np.uint64))
    Q = o.fields()["Q"]
    assert np.isclose(Q.sum(), I.QE * 3e9 * X.size, rtol=1e-13)


def _energy_error(scheme, dt_wpe, T_wpe, seed, dx_lambda=4.0, ppc=512, N=64, quiet=False):
    cfg = I.periodic_plasma(N=N, dx_lambda=dx_lambda, ppc=ppc, dt_wpe=dt_wpe, seed=seed,
                            scheme=scheme, quiet=quiet)
    o = oracle_from_config(cfg)
    W = []
    for _ in range(int(round(T_wpe / dt_wpe))):
        o.step(1)
        ke, fe = o.energy()
        W.append(ke.sum() + fe)
    W = np.array(W)
    return np.max(np.abs(W - W[0])) / W[0]


def test_ec2_energy_second_order_in_dt():
    r = []
    for seed in (5, 6):
        a = _energy_error(oracle.EC2, 0.2, 50.0, seed)
        b = _energy_error(oracle.EC2, 0.1, 50.0, seed)
        r.append(a / b)
        assert b < 1e-4
    assert np.mean(r) >= 3.0, r


def test_ec2_does_not_heat_where_mc_does():
    ec2 = _energy_error(oracle.EC2, 0.1, 250.0, 1, dx_lambda=8.0, ppc=64, N=128, quiet=True)
    mc = _energy_error(oracle.MC, 0.1, 250.0, 1, dx_lambda=8.0, ppc=64, N=128, quiet=True)
    assert ec2 < 2e-3, ec2
    assert mc > 0.1 and mc > 50 * ec2, (mc, ec2)


def test_mc2_conserves_momentum_ec2_does_not():
    masses = [I.ME, I.M_ION]
    drift = {}
    for scheme in (oracle.MC2, oracle.EC2):
        cfg = I.periodic_plasma(N=32, dx_lambda=3.0, ppc=64, dt_wpe=0.2, seed=4, scheme=scheme,
                                ions=True)
        o = oracle_from_config(cfg)
        v0 = [o.get_particles(k)["vx"] for k in range(2)]
        p0 = sum(m * v.sum() for m, v in zip(masses, v0))
        scale = sum(m * np.abs(v).sum() for m, v in zip(masses, v0))
        o.step(60)
        p1 = sum(m * o.get_particles(k)["vx"].sum() for k, m in enumerate(masses))
        drift[scheme] = abs(p1 - p0) / scale
    assert drift[oracle.MC2] <= 1e-11, drift
    assert drift[oracle.EC2] > 1e-6, drift


def test_mc2_heats_less_than_mc_ec2_not_at_all():
    mc = _energy_error(oracle.MC, 0.1, 250.0, 1, dx_lambda=8.0, ppc=64, N=128, quiet=True)
    mc2 = _energy_error(oracle.MC2, 0.1, 250.0, 1, dx_lambda=8.0, ppc=64, N=128, quiet=True)
    ec2 = _energy_error(oracle.EC2, 0.1, 250.0, 1, dx_lambda=8.0, ppc=64, N=128, quiet=True)
    assert mc > mc2 > 100 * ec2, (mc, mc2, ec2)
    assert mc2 > 5e-3, mc2
