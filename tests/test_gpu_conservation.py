"""Conservation properties of the GPU path (Sec. 1, App. B), on collisionless
periodic Maxwellians (uniform neutralising background):

* MC (and MC2) on a uniform periodic grid conserves total momentum (the
  gather is the transpose of the deposit), to FP32 rounding; EC does not.
* The EC total energy error falls about 4x when dt halves (0.2 -> 0.1/w_pe),
  as the oracle's does (second order), and stays close to the oracle's value
  on the same seed; likewise for the higher-order EC2 scheme.
* At dx = 8 lambda_De the MC scheme heats while EC does not (App. B)."""
import numpy as np
import pytest

from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _momentum(g, masses):
    tot, scale = 0.0, 0.0
    for s, m in enumerate(masses):
        v = g.get_particles(s)["vx"].astype(np.float64)
        tot += m * v.sum()
        scale += m * np.abs(v).sum()
    return tot, scale


def test_mc_momentum_conserved_ec_not():
    masses = [I.ME, I.M_ION]
    drift = {}
    for scheme in (I.MC, I.EC, I.MC2):
        cfg = I.periodic_plasma(N=32, dx_lambda=3.0, ppc=64, dt_wpe=0.2, seed=4, scheme=scheme,
                                ions=True)
        g = gpu_from_config(cfg)
        p0, sc = _momentum(g, masses)
        g.step(60)
        p1, _ = _momentum(g, masses)
        drift[scheme] = abs(p1 - p0) / sc
        g.close()
    assert drift[I.MC] <= 2e-6 and drift[I.MC2] <= 2e-6, drift
    assert drift[I.EC] > 20 * drift[I.MC] and drift[I.EC] > 1e-5, drift


def _gpu_energy_error(scheme, dt_wpe, T_wpe, seed, dx_lambda=4.0, ppc=512, N=64):
    cfg = I.periodic_plasma(N=N, dx_lambda=dx_lambda, ppc=ppc, dt_wpe=dt_wpe, seed=seed,
                            scheme=scheme)
    cfg.sample_every = 1
    g = gpu_from_config(cfg)
    W = []
    for _ in range(int(round(T_wpe / dt_wpe))):
        g.step(1)
        d = g.diagnostics(profiles=False)
        W.append(float(d["ke"].sum()) + float(d["fe"]))
    g.close()
    W = np.array(W)
    return float(np.max(np.abs(W - W[0])) / W[0])


def _oracle_energy_error(scheme, dt_wpe, T_wpe, seed, dx_lambda=4.0, ppc=512, N=64):
    from helpers import oracle_from_config
    cfg = I.periodic_plasma(N=N, dx_lambda=dx_lambda, ppc=ppc, dt_wpe=dt_wpe, seed=seed,
                            scheme=scheme)
    o = oracle_from_config(cfg)
    W = []
    for _ in range(int(round(T_wpe / dt_wpe))):
        o.step(1)
        ke, fe = o.energy()
        W.append(ke.sum() + fe)
    o.close()
    W = np.array(W)
    return float(np.max(np.abs(W - W[0])) / W[0])


def test_ec_energy_second_order_in_dt():
    ratios = []
    for seed in (5, 6):
        a = _gpu_energy_error(I.EC, 0.2, 50.0, seed)
        b = _gpu_energy_error(I.EC, 0.1, 50.0, seed)
        ratios.append(a / b)
        assert b < 1e-4, (seed, a, b)
        # same seed, same initial state: the oracle's error is of the same size
        ob = _oracle_energy_error(I.EC, 0.1, 50.0, seed)
        assert 0.5 * ob <= b <= 2.0 * ob, (seed, b, ob)
    assert np.mean(ratios) >= 3.0, ratios


def test_ec2_energy_second_order_in_dt():
    ratios = []
    for seed in (5, 6):
        a = _gpu_energy_error(I.EC2, 0.2, 50.0, seed)
        b = _gpu_energy_error(I.EC2, 0.1, 50.0, seed)
        ratios.append(a / b)
        assert b < 1e-4, (seed, a, b)
        ob = _oracle_energy_error(I.EC2, 0.1, 50.0, seed)
        assert 0.5 * ob <= b <= 2.0 * ob, (seed, b, ob)
    assert np.mean(ratios) >= 3.0, ratios


def test_mc_heats_where_ec_does_not():
    ec = _gpu_energy_error(I.EC, 0.1, 1000.0, 1, dx_lambda=8.0, ppc=64)
    mc = _gpu_energy_error(I.MC, 0.1, 1000.0, 1, dx_lambda=8.0, ppc=64)
    assert mc > 0.05, (mc, ec)
    assert mc > 8 * ec, (mc, ec)
