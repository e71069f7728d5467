"""Pins for the oracle's particle rebalancing (Sec. 3d proposes rebalancing
to keep the particles per cell near a target on non-uniform grids and gives
no algorithm; the merge/split rule is this project's design).

Every check is an invariant computed here from the particles the oracle
returns (positions, velocities, weight multipliers), independently of the
rebalancing code:
* per cell, the total weight (integer) is unchanged exactly;
* the CIC node charges (sum k (1 - xi), sum k xi) are unchanged to FP64
  rounding -- a merge places its pair at the weighted centroid, a split keeps
  the position;
* per cell, the momentum sum k v and every component's sum k v_c^2 (hence
  the energy and the x temperature) are unchanged to FP64 rounding;
* the particle counts follow the rule: a merging cell loses two particles
  per merged group of four, G = min(floor(n/4), ceil((n - target)/2)); a
  splitting cell gains S = min(target - n, #{k >= 2});
* ids stay unique; split children take child_id(parent, level, 3);
* the fixed-point weighted deposit rule sums to 2^32 sum k exactly;
* a run with rebalancing: collisionless periodic plasma on a doubling grid
  keeps its total energy like one without (the rebalancing itself changes
  it by rounding only), and a loaded multiplier m0 with base weight w/m0
  gives the same fields as the plain load.
"""
import numpy as np
import pytest

import oracle
from paper_2308_13092_gb300 import inputs as I

QE, ME = I.QE, I.ME


def _run(edges, bc=I.PERIODIC, w=1e-6, cap=20000, every=0, target=8, lo=4, hi=12, m0=1, ns=1):
    o = oracle.OracleRun()
    o.set_grid(edges, bc, 0.0, 0.0, 0.0, 0.0)
    o.set_scheme(I.EC)
    for s in range(ns):
        o.add_species(-QE if s == 0 else QE, ME if s == 0 else I.M_ION, w, cap)
    o.set_gas(0.0, 300.0, I.M_ION)
    o.set_rebalance(every, target, lo, hi, m0)
    o.init(1, 1e-11, [0] * ns, [0.0] * ns)
    return o


def _cells(edges, X):
    N = edges.size - 1
    j = np.clip(np.searchsorted(edges, X, side="right") - 1, 0, N - 1)
    return j, (X - edges[j]) / (edges[j + 1] - edges[j])


def _cell_sums(o, s=0):
    e = o.edges
    p = o.get_particles(s)
    k = o.get_weights(s).astype(np.float64)
    j, xi = _cells(e, p["X"])
    N = e.size - 1
    out = dict(n=np.bincount(j, minlength=N), W=np.bincount(j, weights=k, minlength=N))
    D = np.zeros(N + 1)
    np.add.at(D, j, k * (1 - xi))
    np.add.at(D, j + 1, k * xi)
    out["D"] = D
    for c in ("vx", "vy", "vz"):
        out["P" + c] = np.bincount(j, weights=k * p[c], minlength=N)
        out["E" + c] = np.bincount(j, weights=k * p[c] ** 2, minlength=N)
    out["ids"] = p["id"]
    out["k"] = o.get_weights(s)
    return out


def _load(o, edges, counts, rng, k=None, s=0, vscale=1e6):
    """counts[j] particles at random offsets of cell j, random velocities."""
    cell = np.repeat(np.arange(edges.size - 1), counts)
    xi = rng.random(cell.size)
    X = edges[cell] + xi * np.diff(edges)[cell]
    v = rng.normal(0.0, vscale, (3, cell.size))
    ids = rng.permutation(cell.size).astype(np.uint64) * np.uint64(7) + np.uint64(5)
    o.set_particles(s, X, v[0], v[1], v[2], ids)
    if k is not None:
        o.set_weights(s, k)
    return cell


def _assert_invariants(a, b):
    assert np.array_equal(a["W"], b["W"])  # integer weights per cell
    assert np.allclose(b["D"], a["D"], rtol=1e-12, atol=1e-12 * a["D"].max())
    for c in ("vx", "vy", "vz"):
        sc = np.abs(a["P" + c]).max() + 1e-300
        assert np.allclose(b["P" + c], a["P" + c], rtol=1e-12, atol=1e-12 * sc), c
        assert np.allclose(b["E" + c], a["E" + c], rtol=1e-12), c
    assert np.unique(b["ids"]).size == b["ids"].size


@pytest.mark.parametrize("weighted", [False, True])
def test_merge_counts_and_invariants(weighted):
    rng = np.random.default_rng(1)
    edges = I.uniform_edges(6, 0.06)
    counts = np.array([3, 13, 40, 12, 25, 100])  # target 8, lo 4, hi 12
    o = _run(edges)
    cell = _load(o, edges, counts, rng)
    if weighted:
        # unequal weights: the centroid, the mean and the spreads are weighted
        o.set_weights(0, rng.integers(1, 9, cell.size).astype(np.uint32))
    a = _cell_sums(o)
    o.rebalance_now()
    b = _cell_sums(o)
    _assert_invariants(a, b)
    T = 8
    expect = []
    for n in counts:
        if n > 12:
            G = min(n // 4, -(-(n - T) // 2))
            expect.append(n - 2 * G)
        elif weighted and n < 4:
            expect.append(n + min(8 - n, int((a["k"][cell == 0] >= 2).sum())))
        else:
            expect.append(n)  # 3 < lo but no particle has k >= 2: nothing to split
    assert np.array_equal(b["n"], np.array(expect)), (b["n"], expect)
    rb = o.rebalance_counters()[0]
    assert rb["merged"] == sum((n - e) // 2 for n, e in zip(counts, expect) if n > 12)
    assert rb["skipped"] == 0
    if not weighted:
        # merged particles carry the group's weights 2 + 2 (four of weight 1)
        assert rb["split"] == 0
        assert set(np.unique(b["k"])) <= {1, 2}
        assert int((b["k"] == 2).sum()) == 2 * rb["merged"]


def test_merge_pairs_sit_at_the_centroid_with_mean_and_spread():
    """One cell of 16 particles, target 12: G = min(4, 2) = 2 groups merged,
    the two nearest the middle of the (vx, id) order (groups 1 and 2); each
    becomes a pair at the group's centroid with velocities u +- d."""
    rng = np.random.default_rng(5)
    edges = I.uniform_edges(3, 0.03)
    o = _run(edges, target=12, lo=4, hi=13)
    cell = _load(o, edges, [0, 16, 0], rng)
    p0 = o.get_particles(0)
    order = np.lexsort((p0["id"], p0["vx"]))
    o.rebalance_now()
    p1 = o.get_particles(0)
    k1 = o.get_weights(0)
    assert p1["X"].size == 12
    for g in (1, 2):
        sel = order[4 * g: 4 * g + 4]
        ids = np.sort(p0["id"][sel])[:2]
        pair = np.isin(p1["id"], ids)
        assert pair.sum() == 2 and np.all(k1[pair] == 2)
        assert np.allclose(p1["X"][pair], p0["X"][sel].mean(), rtol=1e-14)
        for c in ("vx", "vy", "vz"):
            u = p0[c][sel].mean()
            sd = p0[c][sel].std()
            assert np.allclose(np.sort(np.abs(p1[c][pair] - u)), sd, rtol=1e-9), c
    # the other eight are untouched
    rest = np.setdiff1d(np.arange(16), order[4:12])
    for i in rest:
        j = np.nonzero(p1["id"] == p0["id"][i])[0]
        assert j.size == 1 and p1["vx"][j[0]] == p0["vx"][i] and p1["X"][j[0]] == p0["X"][i]
    del cell


def test_split_counts_weights_ids_and_invariants():
    rng = np.random.default_rng(2)
    edges = I.uniform_edges(5, 0.05)
    counts = np.array([2, 3, 5, 1, 0])  # target 8, lo 4: cells 0, 1, 3 split
    o = _run(edges)
    cell = _load(o, edges, counts, rng)
    k = rng.integers(1, 9, cell.size).astype(np.uint32)
    o.set_weights(0, k)
    a = _cell_sums(o)
    p0 = o.get_particles(0)
    o.rebalance_now()
    b = _cell_sums(o)
    _assert_invariants(a, b)
    for j, n in enumerate(counts):
        if 0 < n < 4:
            heavy = int((k[cell == j] >= 2).sum())
            assert b["n"][j] == n + min(8 - n, heavy)
        else:
            assert b["n"][j] == n
    # every split: parent keeps ceil(k/2) and its id, child floor(k/2) and child_id(id, level, 3)
    p1 = o.get_particles(0)
    k1 = o.get_weights(0)
    for i in np.nonzero((cell != 2) & (k >= 2))[0]:
        pid = int(p0["id"][i])
        me = np.nonzero(p1["id"] == pid)[0]
        assert me.size == 1 and k1[me[0]] == (k[i] + 1) // 2
        cid = oracle.child_id(pid, 0, 3)
        ch = np.nonzero(p1["id"] == np.uint64(cid))[0]
        assert ch.size == 1 and k1[ch[0]] == k[i] // 2
        assert p1["X"][ch[0]] == p0["X"][i] and p1["vx"][ch[0]] == p0["vx"][i]


def test_split_takes_the_heaviest_first():
    rng = np.random.default_rng(3)
    edges = I.uniform_edges(2, 0.02)
    o = _run(edges, target=5, lo=4, hi=9)
    _load(o, edges, [3, 0], rng)
    o.set_weights(0, np.array([2, 9, 3], np.uint32))
    p0 = o.get_particles(0)
    o.rebalance_now()  # S = min(5 - 3, 3) = 2: the weights 9 and 3 split
    k1 = np.sort(o.get_weights(0))
    assert np.array_equal(k1, np.array([1, 2, 2, 4, 5], np.uint32)), k1
    assert o.get_particles(0)["X"].size == 5
    del p0


def test_weighted_fixed_point_rule_sums_exactly():
    rng = np.random.default_rng(4)
    N, n = 50, 5000
    cell = rng.integers(0, N, n).astype(np.int32)
    xi = rng.random(n).astype(np.float32)
    k = rng.integers(1, 65537, n).astype(np.uint32)
    S = oracle.deposit_fixed_w(N, cell, xi, k)
    assert int(S.sum(dtype=np.uint64)) == int(k.astype(np.uint64).sum()) * 2 ** 32
    # weight 1 everywhere is the plain rule
    assert np.array_equal(oracle.deposit_fixed_w(N, cell, xi, np.ones(n, np.uint32)),
                          oracle.deposit_fixed(N, cell, xi))
    # a particle of weight k deposits as k particles at its place
    rep = np.repeat(np.arange(200), k[:200] % 7 + 1)
    assert np.array_equal(oracle.deposit_fixed_w(N, cell[:200], xi[:200], k[:200] % 7 + 1),
                          oracle.deposit_fixed(N, cell[rep], xi[rep]))


def test_cells_above_the_limit_are_skipped():
    rng = np.random.default_rng(6)
    edges = I.uniform_edges(2, 0.02)
    o = _run(edges, cap=10000)
    _load(o, edges, [5000, 20], rng)
    o.rebalance_now()
    b = _cell_sums(o)
    assert b["n"][0] == 5000 and b["n"][1] < 20
    assert o.rebalance_counters()[0]["skipped"] == 1


def test_loaded_multiplier_gives_the_plain_fields():
    """Loading with multiplier m0 and base weight w/m0 describes the same
    plasma: identical charge, field and energies at level 0."""
    cfg = I.periodic_plasma(N=32, dx_lambda=2.0, ppc=32, seed=3, ions=True)
    from helpers import oracle_from_config
    a = oracle_from_config(cfg)
    b = oracle_from_config(cfg, init=False)
    b.set_rebalance(0, 8, 4, 16, 64)
    b.init(cfg.seed, cfg.dt, [s.n0 for s in cfg.species], [s.T_eV for s in cfg.species])
    fa, fb = a.fields(), b.fields()
    assert np.allclose(fa["Q"], fb["Q"], rtol=1e-13, atol=1e-13 * np.abs(fa["Q"]).max())
    assert np.allclose(fa["E"], fb["E"], rtol=1e-12, atol=1e-12 * np.abs(fa["E"]).max())
    a.step(2)
    b.step(2)
    assert np.allclose(a.energy()[0], b.energy()[0], rtol=1e-12)
    assert np.all(b.get_weights(0) == 64)


def test_rebalanced_periodic_run_keeps_energy_like_the_plain_run():
    """Collisionless periodic electrons (immobile background) on a doubling
    grid, loaded uniformly: coarse cells merge, fine cells split every 20
    steps; the total energy drift over 400 steps stays within 2x of the plain
    run's (the rebalancing changes the energy by rounding only), and the
    particles per cell move toward the target."""
    n_ref, ppc = 128, 16
    edges = oracle.doubling_grid(n_ref, 0.02, 0.004, 1, 8)
    lam = 0.02 / n_ref / 2.0
    n0 = I.EPS0 * 2.0 / (lam * lam * QE)
    wpe = np.sqrt(n0 * QE ** 2 / (I.EPS0 * ME))
    out = {}
    for every in (0, 20):
        o = oracle.OracleRun()
        o.set_grid(edges, I.PERIODIC, 0, 0, 0, 0)
        o.set_scheme(I.EC)
        n = ppc * n_ref
        o.add_species(-QE, ME, n0 * 0.02 / n, 4 * n)
        o.set_gas(0.0, 300.0, I.M_ION)
        o.set_rebalance(every, 4 * ppc, 2 * ppc, 6 * ppc, 16)
        o.set_quiet_start(True)
        o.init(5, 0.1 / wpe, [n], [2.0])
        o.step(1)
        ke, fe = o.energy()
        w0 = ke.sum() + fe
        o.step(400)
        ke, fe = o.energy()
        out[every] = ((ke.sum() + fe) / w0 - 1.0, _cell_sums(o), o.rebalance_counters()[0])
    d0, d1 = abs(out[0][0]), abs(out[20][0])
    assert d1 < 2.0 * d0 + 2e-4, (d0, d1)
    rb = out[20][2]
    assert rb["merged"] > 0 and rb["split"] > 0
    cnt0, cnt1 = out[0][1]["n"], out[20][1]["n"]
    target = 4 * ppc
    assert np.mean(np.abs(cnt1 - target)) < 0.7 * np.mean(np.abs(cnt0 - target)), (cnt0, cnt1)
