"""Pins for the oracle's loader (uniform density, Maxwellian, Sec. 2b) and
sanity of a short RF-CCP run of the small 128-cell discharge; Table 1's
stated resolution figures against the plasma formulas."""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I
from helpers import oracle_from_config


def test_loader_uniform_maxwellian():
    cfg = I.config_small()
    o = oracle_from_config(cfg)
    for s, sp in enumerate(cfg.species):
        p = o.get_particles(s)
        n = p["X"].size
        assert n == sp.n0
        assert np.array_equal(p["id"], np.arange(n, dtype=np.uint64))
        # positions: uniform on [0, L) (Kolmogorov-Smirnov distance)
        x = np.sort(p["X"]) / cfg.edges[-1]
        ks = np.max(np.abs(x - (np.arange(1, n + 1) - 0.5) / n))
        assert ks < 1.63 / np.sqrt(n)
        sd = np.sqrt(I.QE * sp.T_eV / sp.m)
        for c in ("vx", "vy", "vz"):
            assert abs(p[c].mean()) < 5 * sd / np.sqrt(n)
            assert abs(p[c].std() / sd - 1) < 5 / np.sqrt(2 * n)


def test_loader_uses_philox_stream():
    """X = u L with u = r0 * 2^-32 from Philox(counter = (i, 0, 0xFFFFFFFF,
    (s << 8) | 0x80))."""
    cfg = I.config_small(seed=1234)
    o = oracle_from_config(cfg)
    p = o.get_particles(1)
    for i in (0, 1, 500, 8191):
        r = oracle.philox4x32_10((i, 0, 0xFFFFFFFF, (1 << 8) | 0x80), (1234, 0))
        assert p["X"][i] == r[0] * 2.0 ** -32 * cfg.edges[-1]


def test_initial_charge_and_rf_boundary():
    cfg = I.config_small()
    o = oracle_from_config(cfg)
    f = o.fields()
    tot = sum(s.q * s.w * s.n0 for s in cfg.species)
    assert abs(f["Q"].sum() - tot) <= 1e-12 * sum(abs(s.q * s.w * s.n0) for s in cfg.species)
    assert f["phi"][0] == 0.0 and f["phi"][-1] == 0.0  # sin(0) = 0
    o.step(50)
    f = o.fields()
    t = 50 * cfg.dt
    assert np.isclose(f["phi"][0], cfg.v0 * np.sin(2 * np.pi * cfg.freq * t), rtol=1e-12)


def test_short_ccp_run_sanity():
    """200 steps of the 128-cell discharge: particle bookkeeping closes and the
    electrons that leave are mostly the fast ones lost to the walls."""
    cfg = I.config_small()
    o = oracle_from_config(cfg)
    o.reset_averages(10)
    o.step(200)
    c = o.counters()
    assert c["step"] == 200
    for s, sp in enumerate(cfg.species):
        cs = c["species"][s]
        born = c["species"][0]["births"]
        assert cs["n"] == sp.n0 + born - cs["absorbed_left"] - cs["absorbed_right"] - cs["lost"]
        assert cs["lost"] == 0
    e = c["species"][0]
    assert e["absorbed_left"] + e["absorbed_right"] > 0
    assert sum(e["collisions"]) > 0
    a = o.averages()
    assert a["n_samples"] == 20
    assert np.all(np.isfinite(a["density"])) and np.all(a["density"] >= 0)
    assert np.all(np.isfinite(a["Tx"]))
    bulk = slice(40, 90)
    # 300 V on a weakly screened 5e13 m^-3 plasma heats electrons ohmically
    assert a["Tx"][0][bulk].mean() > 2.0
    assert a["Tx"][1][bulk].mean() < 0.5           # ions stay cold


def test_no_drive_keeps_temperature():
    """Without RF the collisional plasma only loses energy: the bulk electron
    temperature stays near its 2 eV start; without RF and collisions it keeps
    it to a few percent."""
    for coll in (True, False):
        cfg = I.ccp("flat", N=128, n0=5e13, dt=1 / (200 * I.F_RF), ppc=64, v0=0.0,
                    p_mtorr=30.0, n_steps=0, collisions=coll)
        o = oracle_from_config(cfg)
        o.step(100)
        o.reset_averages(10)
        o.step(200)
        Te = o.averages()["Tx"][0][40:90].mean()
        assert 1.6 < Te < 2.4


def test_table1_resolution_figures():
    """Table 1 parameters give lambda_De ~ 0.975 dx_ref and w_pe dt ~ 0.087,
    consistent with the 1.11 dx_ref and 0.085 stated at steady state (Sec. 3a)."""
    n0, Te = 7e15, 2.585
    lam = np.sqrt(I.EPS0 * Te / (n0 * I.QE))
    wpe = np.sqrt(n0 * I.QE ** 2 / (I.EPS0 * I.ME))
    dx_ref = 0.3 / 2048
    dt = 1 / (4000 * 13.56e6)
    assert abs(lam / dx_ref - 0.975) < 0.005
    assert abs(wpe * dt - 0.087) < 0.001
    assert abs(dx_ref - 1.465e-4) < 1e-7
    assert 5100 * 4000 == 20_400_000 and 100 * 4000 == 400_000 and 4000 // 10 == 400


def test_quiet_start_positions_velocities_and_zero_field():
    """Quiet start: X_i = (i + 1/2) L / n exactly; velocities are the random
    loader's (same Philox block); an evenly spaced load with whole particles
    per cell on a uniform periodic grid deposits the same charge on every
    node, so the initial field and field energy vanish."""
    cfg = I.periodic_plasma(N=32, dx_lambda=4.0, ppc=16, dt_wpe=0.1, seed=7)
    rnd = oracle_from_config(cfg)
    cfg.quiet = True
    q = oracle_from_config(cfg)
    pr, pq = rnd.get_particles(0), q.get_particles(0)
    n = pq["X"].size
    L = cfg.edges[-1]
    assert np.array_equal(pq["X"], (np.arange(n) + 0.5) / n * L)
    for k in ("vx", "vy", "vz", "id"):
        assert np.array_equal(pq[k], pr[k]), k
    ke, fe = q.energy()
    f = q.fields()
    assert np.max(np.abs(f["E"])) < 1e-9 * np.max(np.abs(rnd.fields()["E"]))
    assert fe <= 1e-20 * (0.5 * I.ME * cfg.species[0].w * np.sum(pq["vx"] ** 2))
    with pytest.raises(RuntimeError):
        q.set_quiet_start(False)  # only before init


def test_quiet_start_app_b_mc_heats_ec_conserves():
    """App. B on the oracle with a quiet start: at dx = 8 lambda_De the MC
    scheme's total energy grows by tens of per cent in 2500 steps (grid
    heating) while EC's stays within 0.2 %; at dx = lambda_De both stay small."""
    out = {}
    for r in (1.0, 8.0):
        for sch in (I.EC, I.MC):
            c = I.periodic_plasma(N=128, dx_lambda=r, ppc=64, dt_wpe=0.1, seed=3, scheme=sch,
                                  n0=7e15, Te=2.585, quiet=True)
            o = oracle_from_config(c)
            o.step(1)
            ke, fe = o.energy()
            w0 = ke.sum() + fe
            o.step(2500)
            ke, fe = o.energy()
            out[(r, sch)] = (ke.sum() + fe) / w0 - 1.0
            o.close()
    assert abs(out[(8.0, I.EC)]) < 2e-3, out
    assert out[(8.0, I.MC)] > 0.1, out
    assert abs(out[(1.0, I.EC)]) < 2e-3 and abs(out[(1.0, I.MC)]) < 5e-3, out


def test_set_step_continues_a_state_from_its_own_level():
    """A colliding RF discharge stepped to level 7, its particles copied into a
    fresh run moved to level 7: one more step gives the same particles bit for
    bit (the RF bias and the random stream follow the level); left at level 0
    the copy diverges."""
    cfg = I.config_small(seed=4)
    a = oracle_from_config(cfg)
    a.step(7)
    st = [a.get_particles(s) for s in range(2)]

    def copy(level):
        b = oracle_from_config(cfg)
        if level:
            b.set_step(level)
        for s in range(2):
            p = st[s]
            b.set_particles(s, p["X"], p["vx"], p["vy"], p["vz"], p["id"])
        b.step(1)
        return b

    a.step(1)
    b, c = copy(7), copy(0)
    assert b.counters()["step"] == 8
    for s in range(2):
        pa, pb, pc = a.get_particles(s), b.get_particles(s), c.get_particles(s)
        ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
        for k in ("X", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[k][ia], pb[k][ib]), (s, k)
        ic = np.argsort(pc["id"])
        if pc["id"].size == pa["id"].size and np.array_equal(pc["id"][ic], pa["id"][ia]):
            assert not np.array_equal(pa["vx"][ia], pc["vx"][ic])
