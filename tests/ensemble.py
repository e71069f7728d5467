"""Ensemble comparison of full runs, GPU against the oracle (test glue).

A run's trajectory depends on FP32 vs FP64 rounding, so the GPU and the
oracle decorrelate after some hundreds of steps even from one seed, and
whole runs are compared as ensembles.  The seed-to-seed spread of a
discharge can be far from normal (the under-resolved discharges' ionisation
counts are heavy-tailed: at dx = 8 lambda_De the births over 3000 steps range
from 111 to 3961 across 64 seeds, median 672), so two statistics are used:

* a two-sample permutation test of the ensemble means: the GPU population
  (many seeds; cheap) and the oracle runs (few; costly) are pooled, and the
  observed relative L2 distance between the two means must not be extreme
  among random relabellings of the pool into groups of the same sizes
  (p >= P_MIN with a fixed permutation stream);
* a paired comparison: the GPU runs on the oracle's own seeds start from the
  same load (bit-identical cells, offsets within 2^-24) and share its early
  history, so each GPU-oracle pair must lie no farther apart than two
  independent GPU runs do on average.
"""
from __future__ import annotations

import itertools

import numpy as np

from helpers import rel_l2

P_MIN = 1e-3
N_PERM = 4000


def permutation_p(G, O, n_perm=N_PERM, seed=12345):
    """p-value of relL2(mean(O), mean(G)) under random relabelling of the
    pooled runs (rows of G and O); (1 + #{T* >= T}) / (1 + n_perm)."""
    G = np.asarray(G, float)
    O = np.asarray(O, float)
    t_obs = rel_l2(O.mean(0), G.mean(0))
    pool = np.concatenate([G, O])
    n_o = O.shape[0]
    rng = np.random.default_rng(seed)
    hits = 0
    for _ in range(n_perm):
        idx = rng.permutation(pool.shape[0])
        a, b = pool[idx[:n_o]], pool[idx[n_o:]]
        if rel_l2(a.mean(0), b.mean(0)) >= t_obs:
            hits += 1
    return (1 + hits) / (1 + n_perm), t_obs


def spread(runs, max_pairs=400):
    """Mean relative L2 distance between two independent runs (the seed
    spread), over at most max_pairs pairs."""
    runs = list(runs)
    pairs = list(itertools.combinations(range(len(runs)), 2))[:max_pairs]
    return float(np.mean([rel_l2(runs[i], runs[j]) for i, j in pairs]))


def paired(Gp, O):
    """Mean relative L2 distance of the GPU runs on the oracle's seeds to
    their oracle partners."""
    return float(np.mean([rel_l2(g, o) for g, o in zip(Gp, O)]))


def compare(G, Gp, O, name):
    """Both statistics for one profile (or rate vector); returns a report
    line and asserts: p >= P_MIN and paired <= seed spread."""
    p, t = permutation_p(G, O)
    sg = spread(G)
    so = spread(O)
    pd = paired(Gp, O)
    line = (f"{name}: relL2(means) {t:.4f} perm p {p:.4f} | paired {pd:.4f} "
            f"seed spread GPU {sg:.4f} oracle {so:.4f} | paired/spread {pd / sg:.2f}")
    assert p >= P_MIN, line
    assert pd <= sg, line
    return line
