"""GPU particle rebalancing (Sec. 3d proposes it; the merge/split rule is this
library's design, written first in the oracle) against the oracle, through
the C ABI.

* One rebalancing from an identical state (random weights, over- and
  under-full cells, uniform and doubling grids, EC and MC): the same particle
  ids survive and appear on both sides; per id the cell and the weight
  multiplier are exact, the offset and the velocities are the FP64 results
  rounded to FP32 (offset within 2^-23 of a cell, velocities within 1e-6 of
  the group's velocity scale); the merge and split counters are equal; the
  node charges (CIC shares times weights) of both particle sets agree to the
  offsets' FP32 rounding.
* The step after it, collisional: one-step parity as for the plain runs
  (cells exact away from faces, positions and velocities to 1e-5, collision
  candidates exactly equal).
* A 114-cell doubling-grid discharge rebalancing every 20 steps: the GPU on
  the oracle's seeds against the oracle (time-averaged profiles paired, no
  farther apart than two independent GPU seeds), identical counters over the
  first steps, and the particles per cell brought toward the target.
"""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I
from helpers import gpu_from_config, oracle_from_config, rel_l2, require_gpu
from test_gpu_parity import _compare, _counters_match

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _cfg(edges=None, scheme=I.EC, collisions=False, seed=3, every=0, target=24, lo=12, hi=36, m0=8):
    c = I.ccp("rb", N=32, n0=5e13, dt=1.0 / (400 * I.F_RF), ppc=0, v0=200.0, p_mtorr=60.0,
              n_steps=1, seed=seed, scheme=scheme, edges=edges, L=0.04, collisions=collisions,
              n_per_species=1000)
    c.rebalance = dict(every=every, target=target, lo=lo, hi=hi, m0=m0)
    I.with_headroom(c, 4.0)
    return c


def _state(cfg, rng, counts):
    """A state with the given particles per cell (both species), random
    offsets, Maxwellian velocities and weights 1..16."""
    out = []
    for s, sp in enumerate(cfg.species):
        cell = np.repeat(np.arange(cfg.N), counts).astype(np.int32)
        n = cell.size
        xi = rng.random(n).astype(np.float32)
        vth = np.sqrt(I.QE * (3.0 if s == 0 else 0.2) / sp.m)
        v = rng.normal(0, vth, (3, n)).astype(np.float32)
        ids = (np.uint64(10 ** 6 * s + 7) + rng.permutation(n).astype(np.uint64) * np.uint64(3))
        k = rng.integers(1, 17, n).astype(np.uint32)
        out.append(dict(cell=cell, xi=xi, vx=v[0], vy=v[1], vz=v[2], id=ids, k=k))
    return out


def _set(g, o, st):
    for s, p in enumerate(st):
        g.set_particles(s, p["cell"], p["xi"], p["vx"], p["vy"], p["vz"], p["id"])
        g.set_weights(s, p["k"])
        o.set_particles_cell(s, p["cell"], p["xi"], p["vx"], p["vy"], p["vz"], p["id"])
        o.set_weights(s, p["k"])


def _node_charges(edges, cell, xi, k):
    D = np.zeros(edges.size)
    np.add.at(D, cell, k * (1.0 - xi))
    np.add.at(D, cell + 1, k * xi)
    return D


@pytest.mark.parametrize("scheme,grid,bc", [(I.EC, "uniform", I.DIRICHLET), (I.MC, "uniform", I.DIRICHLET),
                                            (I.EC, "doubling", I.DIRICHLET), (I.MC, "doubling", I.PERIODIC)])
def test_one_rebalancing_matches_oracle(scheme, grid, bc):
    edges = None if grid == "uniform" else oracle.doubling_grid(64, 0.04, 0.008, 1, 4)
    cfg = _cfg(edges=edges, scheme=scheme)
    cfg.bc = bc
    rng = np.random.default_rng(7)
    N = cfg.N
    counts = rng.integers(0, 90, N)  # target 24: over-full (> 36) and under-full (< 12) cells
    counts[: N // 4] = rng.integers(0, 12, N // 4)
    st = _state(cfg, rng, counts)
    g, o = gpu_from_config(cfg), oracle_from_config(cfg)
    _set(g, o, st)
    g.rebalance_now()
    o.rebalance_now()
    dg = g.diagnostics(profiles=False)["species"]
    rbo = o.rebalance_counters()
    e = cfg.edges
    for s in range(2):
        assert dg[s]["rb_merged"] == rbo[s]["merged"] > 0, (s, dg[s]["rb_merged"], rbo[s])
        assert dg[s]["rb_split"] == rbo[s]["split"] > 0, (s, dg[s]["rb_split"], rbo[s])
        gp, op = g.get_particles(s), o.get_particles(s)
        gk, ok = g.get_weights(s), o.get_weights(s)
        oc, oxi = o.get_particles_cell(s)
        assert gp["id"].size == op["id"].size
        gi, oi = np.argsort(gp["id"]), np.argsort(op["id"])
        assert np.array_equal(gp["id"][gi], op["id"][oi])
        assert np.array_equal(gk[gi], ok[oi])
        assert np.array_equal(gp["cell"][gi], oc[oi])
        assert np.all(np.abs(gp["xi"][gi].astype(np.float64) - oxi[oi]) <= 2.0 ** -23)
        vs = np.sqrt(I.QE * 3.0 / cfg.species[s].m)
        for comp in ("vx", "vy", "vz"):
            d = np.abs(gp[comp][gi].astype(np.float64) - op[comp][oi])
            assert np.all(d <= 1e-6 * (np.abs(op[comp][oi]) + vs)), comp
        # node charges of both particle sets, and of the state before
        Dg = _node_charges(e, gp["cell"], gp["xi"].astype(np.float64), gk.astype(np.float64))
        Do = _node_charges(e, oc, oxi, ok.astype(np.float64))
        D0 = _node_charges(e, st[s]["cell"], st[s]["xi"].astype(np.float64), st[s]["k"].astype(np.float64))
        scale = D0.max()
        assert np.max(np.abs(Dg - Do)) <= 1e-6 * scale
        assert np.max(np.abs(Do - D0)) <= 1e-9 * scale
        assert int(gk.astype(np.int64).sum()) == int(st[s]["k"].astype(np.int64).sum())
    g.close()
    o.close()


def test_step_after_rebalancing_matches_oracle():
    cfg = _cfg(collisions=True, seed=4)
    rng = np.random.default_rng(8)
    counts = rng.integers(0, 90, cfg.N)
    st = _state(cfg, rng, counts)
    g, o = gpu_from_config(cfg), oracle_from_config(cfg)
    _set(g, o, st)
    g.rebalance_now()
    o.rebalance_now()
    before = [dict(id=g.get_particles(s)["id"], **{c: g.get_particles(s)[c] for c in ("vx", "vy", "vz")})
              for s in range(2)]
    g.step(1)
    g.sync()
    o.step(1)
    rep = _compare(cfg, g, o, before)
    for s in range(2):
        assert rep[s]["only"] == 0 and rep[s]["bad"] <= 2, rep
    _counters_match(g, o)


def _doubling_run(seed, every=20, steps=600):
    edges = oracle.doubling_grid(1024, I.L_GAP, 0.05, 4, 32)
    c = I.config_nonuniform(edges, seed=seed)
    c.sample_every = 15
    c.n_steps = steps
    c.rebalance = dict(every=every, target=256, lo=128, hi=384, m0=16)
    I.with_headroom(c, 3.0)
    return c


def test_rebalanced_discharge_paired_with_oracle():
    """114-cell doubling grid, 58k particles, rebalancing every 20 steps for
    600 steps: the GPU on two oracle seeds against the oracle runs of those
    seeds (profiles no farther apart than two independent GPU seeds); the
    rebalancing counters agree exactly over the first 40 steps; the spread
    of particles per cell shrinks toward the target."""
    from paper_2308_13092_gb300 import ecpic
    seeds = list(range(500, 516))
    oseeds = [600, 601]
    eng = ecpic.Engine(max_slots=len(seeds) + len(oseeds), max_cells=256)
    tk = {s: eng.submit(_doubling_run(s)) for s in seeds + oseeds}
    while True:
        r, q = eng.pump(600)
        if r == 0 and q == 0:
            break
    gpu = {}
    for s, t in tk.items():
        res = eng.poll(t, diagnostics=True, profiles=True)
        assert res["state"] == 2, (s, res["state"])
        gpu[s] = res["diag"]
    eng.close()
    keys = (("ne", lambda d: d["density"][0]), ("ni", lambda d: d["density"][1]),
            ("phi", lambda d: d["phi"]), ("Te", lambda d: d["Tx"][0]))
    ora = {}
    for s in oseeds:
        o = oracle_from_config(_doubling_run(s))
        o.step(600, allow_capacity=True)
        ora[s] = o.averages()
        o.close()
    for name, get in keys:
        G = [get(gpu[s]) for s in seeds]
        spread = np.mean([rel_l2(G[i], G[j]) for i in range(len(G)) for j in range(i + 1, len(G))])
        og = {"ne": lambda a: a["density"][0], "ni": lambda a: a["density"][1],
              "phi": lambda a: a["phi"], "Te": lambda a: a["Tx"][0]}[name]
        paired = np.mean([rel_l2(get(gpu[s]), og(ora[s])) for s in oseeds])
        print(f"rebalanced doubling-114 {name}: paired {paired:.4f} seed spread {spread:.4f}")
        assert paired <= spread, (name, paired, spread)
    for s in seeds:
        sp = gpu[s]["species"]
        assert sp[0]["rb_merged"] > 0 and sp[0]["rb_split"] > 0


def test_rebalancing_counters_follow_the_oracle_and_even_out_the_cells():
    cfg = _doubling_run(600, steps=40)
    g, o = gpu_from_config(cfg), oracle_from_config(cfg)
    counts0 = np.bincount(g.get_particles(0)["cell"], minlength=cfg.N)
    g.step(40)
    g.sync()
    o.step(40, allow_capacity=True)
    dg = g.diagnostics(profiles=False)["species"]
    rbo = o.rebalance_counters()
    for s in range(2):
        assert (dg[s]["rb_merged"], dg[s]["rb_split"]) == (rbo[s]["merged"], rbo[s]["split"]), s
        assert dg[s]["n"] == o.counters()["species"][s]["n"]
    counts1 = np.bincount(g.get_particles(0)["cell"], minlength=cfg.N)
    dev0 = np.mean(np.abs(counts0 - 256))
    dev1 = np.mean(np.abs(counts1 - 256))
    assert dev1 < 0.5 * dev0, (dev0, dev1)


def _key(d):
    return [(s["n"], s["births"], s["candidates"], tuple(s["collisions"]), s["rb_merged"],
             s["rb_split"]) for s in d["species"]]


def _small_rb(seed, every, capacity_extra=None):
    c = I.config_small(seed=seed)
    c.sample_every = 10
    c.n_steps = 240
    c.rebalance = dict(every=every, target=64, lo=55, hi=70, m0=16)
    if capacity_extra is not None:
        for sp in c.species:
            sp.capacity = sp.n0 + capacity_extra
    return c


def test_rebalancing_run_alone_equals_run_in_mix():
    """Two rebalancing runs (cadences 20 and 30) and a plain one in one engine
    batch: each rebalancing run's counters, rebalancing counts, particles,
    weights and density equal the same run stepped alone (the rebalancing is
    per run and per cell; the deposit is an integer sum)."""
    from paper_2308_13092_gb300 import ecpic
    cfgs = [_small_rb(21, 20), I.config_small(seed=22), _small_rb(23, 30)]
    cfgs[1].n_steps = 240
    cfgs[1].sample_every = 10
    eng = ecpic.Engine(max_slots=3, max_cells=256)
    tks = [eng.submit(c) for c in cfgs]
    while True:
        r, q = eng.pump(100)
        if r == 0 and q == 0:
            break
    for c, t in zip(cfgs, tks):
        if not c.rebalance:
            continue
        dm = eng.poll(t, diagnostics=True, profiles=True)["diag"]
        g = gpu_from_config(c)
        g.step(c.n_steps)
        g.sync()
        da = g.diagnostics(profiles=True)
        assert _key(dm) == _key(da)
        assert dm["species"][0]["rb_merged"] > 0 and dm["species"][0]["rb_split"] > 0
        assert np.array_equal(dm["density"], da["density"])
    eng.close()


def test_rebalancing_run_admitted_into_a_stepping_batch():
    """A plain run steps alone (the step graphs are captured for a batch with
    no weight multipliers); a rebalancing run then joins, and later leaves
    while the plain run goes on.  The batch's pass switches to the weighted
    kernel and back; both runs equal the same runs stepped alone."""
    from paper_2308_13092_gb300 import ecpic
    plain = I.config_small(seed=24)
    plain.n_steps = 400
    plain.sample_every = 10
    rb = _small_rb(25, 20)
    eng = ecpic.Engine(max_slots=2, max_cells=256)
    t0 = eng.submit(plain)
    eng.pump(60)
    t1 = eng.submit(rb)
    while True:
        r, q = eng.pump(50)
        if r == 0 and q == 0:
            break
    for c, t in ((plain, t0), (rb, t1)):
        dm = eng.poll(t, diagnostics=True, profiles=True)["diag"]
        g = gpu_from_config(c)
        g.step(c.n_steps)
        g.sync()
        da = g.diagnostics(profiles=True)
        assert _key(dm) == _key(da)
        assert np.array_equal(dm["density"], da["density"])
    eng.close()


def test_rebalancing_run_grows_like_an_ample_one():
    """A rebalancing run given its initial load plus 300 particles of capacity,
    growing automatically, follows the run given ample capacity particle for
    particle (weights carried through the reallocation)."""
    a = gpu_from_config(_small_rb(24, 20, capacity_extra=40_000))
    b = gpu_from_config(_small_rb(24, 20, capacity_extra=300))
    b.set_auto_grow(True)
    a.step(240)
    b.step(240)
    a.sync()
    b.sync()
    assert _key(a.diagnostics()) == _key(b.diagnostics())
    for s in range(2):
        pa, pb = a.get_particles(s), b.get_particles(s)
        ka, kb = a.get_weights(s), b.get_weights(s)
        ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
        for key in ("cell", "xi", "vx", "vy", "vz", "id"):
            assert np.array_equal(pa[key][ia], pb[key][ib]), (s, key)
        assert np.array_equal(ka[ia], kb[ib])
