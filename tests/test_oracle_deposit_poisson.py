"""Pins for the oracle's deposit (Eq. 2-3), Poisson solve (Eq. 4) and field
(Eq. 5 and the centred MC field) against closed forms and exact identities."""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I

EPS0 = 8.8541878128e-12


def grids():
    rng = np.random.default_rng(3)
    yield "uniform", I.uniform_edges(64, 0.3)
    yield "doubling", oracle.doubling_grid(256, 0.3, 0.05, 1, 8)
    yield "tanh", I.tanh_edges(90, 0.3, 0.3 / 1024 * 4)
    w = rng.uniform(0.5, 2.0, 77)
    e = np.concatenate([[0.0], np.cumsum(w)])
    yield "random", e * (0.3 / e[-1])


# ------------------------------------------------------------------ deposit
def test_fixed_deposit_total_is_exact():
    rng = np.random.default_rng(0)
    N, n = 100, 50000
    cell = rng.integers(0, N, n).astype(np.int32)
    xi = rng.random(n).astype(np.float32)
    S = oracle.deposit_fixed(N, cell, xi)
    assert int(S.sum(dtype=np.uint64)) == n * 2 ** 32


def test_fixed_deposit_single_particle_shares():
    S = oracle.deposit_fixed(4, [2], np.array([0.25], np.float32))
    assert S.tolist() == [0, 0, 3 * 2 ** 30, 2 ** 30, 0]
    S = oracle.deposit_fixed(4, [0], np.array([0.0], np.float32))
    assert S.tolist() == [2 ** 32, 0, 0, 0, 0]
    # the largest float below 1 keeps 2^8 units on the left node
    S = oracle.deposit_fixed(4, [3], np.array([np.float32(1) - np.float32(2 ** -24)]))
    assert S.tolist() == [0, 0, 0, 2 ** 8, 2 ** 32 - 2 ** 8]
    # below 2^-9 the product xi*2^32 has a fraction: floor
    tiny = np.float32(3.0 * 2 ** -40)
    S = oracle.deposit_fixed(4, [1], np.array([tiny]))
    assert S.tolist() == [0, 2 ** 32, 0, 0, 0]


def test_fixed_deposit_matches_fp64_cic_within_quantum():
    """The FP64 deposit of a run (Q = q w D) and the fixed-point rule agree to
    at most one 2^-32 quantum per contributing particle."""
    rng = np.random.default_rng(1)
    N, n = 32, 4000
    e = I.uniform_edges(N, 0.1)
    o = oracle.OracleRun()
    o.set_grid(e, oracle.DIRICHLET)
    o.add_species(1.0, 1.0, 1.0, n)
    o.init(0, 1e-9, [0], [0.0])
    cell = rng.integers(0, N, n).astype(np.int32)
    xi = rng.random(n).astype(np.float32)
    z = np.zeros(n, np.float32)
    o.set_particles_cell(0, cell, xi, z, z, z, np.arange(n, dtype=np.uint64))
    D = o.fields()["Q"]
    S = oracle.deposit_fixed(N, cell, xi).astype(np.float64) * 2.0 ** -32
    cnt = np.bincount(cell, minlength=N + 1) + np.bincount(cell + 1, minlength=N + 1)
    assert np.all(np.abs(D - S) <= cnt * 2.0 ** -32 + 1e-12)


def test_deposit_lattice_is_exact():
    """Two particles per cell at xi = 1/4, 3/4: every interior node collects
    exactly 2 (Eq. 2-3 with S_1 the linear hat)."""
    N = 16
    cell = np.repeat(np.arange(N, dtype=np.int32), 2)
    xi = np.tile(np.array([0.25, 0.75], np.float32), N)
    S = oracle.deposit_fixed(N, cell, xi)
    assert np.all(S[1:N] == 2 * 2 ** 32)
    assert S[0] == 2 ** 32 and S[N] == 2 ** 32


# ------------------------------------------------------------------ Poisson
@pytest.mark.parametrize("name,x", list(grids()))
def test_poisson_uniform_slab_parabola(name, x):
    """Uniform charge density rho0, phi = 0 at both walls: phi = rho0 x (L-x)/(2 eps0).
    The finite-volume 3-point stencil is exact on quadratics on any grid."""
    rho0 = 1e-6
    N = x.size - 1
    L = x[-1]
    V = np.zeros(N + 1)
    dx = np.diff(x)
    V[1:N] = 0.5 * (dx[:-1] + dx[1:])
    phi = oracle.poisson_thomas(x, rho0 * V, 0.0, 0.0)
    exact = rho0 * x * (L - x) / (2 * EPS0)
    assert np.max(np.abs(phi - exact)) <= 1e-11 * np.max(np.abs(exact))


@pytest.mark.parametrize("name,x", list(grids()))
def test_poisson_point_charge_green_function(name, x):
    """A sheet charge Q at node m between grounded walls: the continuum Green's
    function, piecewise linear with a kink -Q/eps0 at x_m; exact on the stencil."""
    N = x.size - 1
    L = x[-1]
    for m in (1, N // 3, N - 1):
        Q = np.zeros(N + 1)
        Q[m] = 2.5e-9
        phi = oracle.poisson_thomas(x, Q, 0.0, 0.0)
        xm = x[m]
        exact = np.where(x <= xm, Q[m] / EPS0 * x * (L - xm) / L,
                         Q[m] / EPS0 * xm * (L - x) / L)
        assert np.max(np.abs(phi - exact)) <= 1e-11 * np.max(np.abs(exact))


@pytest.mark.parametrize("name,x", list(grids()))
def test_poisson_vacuum_is_linear(name, x):
    V0 = 317.0
    phi = oracle.poisson_thomas(x, np.zeros_like(x), V0, 0.0)
    assert np.allclose(phi, V0 * (1 - x / x[-1]), rtol=0, atol=1e-11 * V0)


@pytest.mark.parametrize("name,x", list(grids()))
def test_thomas_equals_dense_elimination(name, x):
    rng = np.random.default_rng(5)
    Q = rng.normal(0, 1e-9, x.size)
    a = oracle.poisson_thomas(x, Q, 12.0, -3.0)
    b = oracle.poisson_dense(x, Q, 12.0, -3.0)
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))


# ------------------------------------------------------------------ field
@pytest.mark.parametrize("name,x", list(grids()))
def test_ec_field_gauss_law(name, x):
    """Eq. 4-5 together: E_j - E_{j-1} = Q_j / eps0 at every interior node."""
    rng = np.random.default_rng(6)
    Q = rng.normal(0, 1e-9, x.size)
    phi = oracle.poisson_thomas(x, Q, 50.0, 0.0)
    E = oracle.field(x, phi, oracle.DIRICHLET, oracle.EC)
    assert E.size == x.size - 1
    lhs = (E[1:] - E[:-1]) * EPS0
    assert np.max(np.abs(lhs - Q[1:-1])) <= 1e-7 * np.max(np.abs(Q))


def test_mc_field_is_mean_of_face_fields_on_uniform_grid():
    x = I.uniform_edges(40, 0.2)
    rng = np.random.default_rng(7)
    phi = rng.normal(0, 10, x.size)
    Eec = oracle.field(x, phi, oracle.DIRICHLET, oracle.EC)
    Emc = oracle.field(x, phi, oracle.DIRICHLET, oracle.MC)
    assert np.allclose(Emc[1:-1], 0.5 * (Eec[:-1] + Eec[1:]), rtol=1e-12, atol=0)
    assert Emc[0] == Eec[0] and Emc[-1] == Eec[-1]
    phi[-1] = phi[0]
    Ep = oracle.field(x, phi, oracle.PERIODIC, oracle.MC)
    Ee = oracle.field(x, phi, oracle.PERIODIC, oracle.EC)
    assert np.isclose(Ep[0], 0.5 * (Ee[0] + Ee[-1]), rtol=1e-12) and Ep[0] == Ep[-1]


def test_ec_field_is_minus_gradient_of_cic_potential():
    """EC property (Sec. 1, Sec. 2a note after Eq. 9): the particle field is
    minus the derivative of the CIC-interpolated potential."""
    x = oracle.doubling_grid(64, 0.1, 0.01, 1, 4)
    rng = np.random.default_rng(8)
    phi = rng.normal(0, 10, x.size)
    E = oracle.field(x, phi, oracle.DIRICHLET, oracle.EC)
    for j in range(x.size - 1):
        for xi in (0.1, 0.5, 0.9):
            h = 1e-7 * (x[j + 1] - x[j])
            X = x[j] + xi * (x[j + 1] - x[j])

            def pcic(Y):
                t = (Y - x[j]) / (x[j + 1] - x[j])
                return (1 - t) * phi[j] + t * phi[j + 1]
            d = (pcic(X + h) - pcic(X - h)) / (2 * h)
            assert np.isclose(-d, E[j], rtol=1e-6, atol=1e-9 * np.abs(phi).max())
