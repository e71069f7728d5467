"""Host-side logic without a GPU: the benchmark's choice of sort cadences
(the timed window must hold whole sort cycles), the threaded oracle timing
(every thread's runs stepped, particle-steps counted), and the ensemble
statistics used by the full-run parity tests (permutation p-values under the
null and under a shift, the paired distance)."""
import numpy as np
import pytest

import bench
import ensemble
from paper_2308_13092_gb300 import inputs as I


@pytest.mark.parametrize("steps", [1, 3, 7, 20, 64, 100, 400, 4000, 4001])
def test_sort_cadences_divide_the_window(steps):
    ks = bench.sort_cadences(steps)
    assert 1 <= len(ks) <= 4 and ks == sorted(set(ks))
    for k in ks:
        assert 1 <= k <= 4096
        if steps >= 4 and any(steps % d == 0 for d in range(4, min(64, steps) + 1)):
            assert steps % k == 0 and 4 <= k <= 64, (steps, ks)


def test_sort_cadences_examples():
    assert bench.sort_cadences(20) == [10, 20]
    assert bench.sort_cadences(4000) == [8, 16, 32, 50]
    assert bench.sort_cadences(64) == [8, 16, 32, 64]


def test_autotune_step_count_matches_the_trials():
    # two trials per (K, grid) pair; per trial: K steps to start the cadence
    # and max(per_trial, 2K) rounded up to whole cycles of the sort and of the
    # sample (every 40 steps); five grids
    assert bench.autotune_steps(64, Ks=(10, 20)) == 2 * 5 * ((10 + 80) + (20 + 80))
    # K = 50: lcm(50, 40) = 200 <= 8 x 100
    assert bench.autotune_steps(64, Ks=(50,)) == 2 * 5 * (50 + 200)
    # without sampling: whole sort cycles only
    assert bench.autotune_steps(64, Ks=(10, 20), sample_every=0) == 2 * 5 * ((10 + 70) + (20 + 80))
    # a common multiple above 8x the trial falls back to the sort cycle
    assert bench.autotune_steps(64, Ks=(63,), sample_every=40) == 2 * 5 * (63 + 126)


def test_threaded_oracle_timing_counts_every_runs_particle_steps():
    cfgs = I.batched_manifest(6, seed=3, steps=10, scale=0.01)
    v, ps, done, used, warm = bench.oracle_parallel(cfgs, 3, 1, 4, budget_s=60.0)
    assert used == 6 and done == 4 and warm == 1
    assert v > 0
    # particle-steps: live particles at the start of each timed step, summed
    lo = sum(c.n_particles for c in cfgs) * 4 * 0.5
    hi = sum(c.n_particles for c in cfgs) * 4 * 2.0
    assert lo <= ps <= hi


def test_permutation_p_is_not_small_under_the_null():
    rng = np.random.default_rng(0)
    ps = []
    for t in range(20):
        G = rng.normal(1.0, 0.1, (64, 40))
        O = rng.normal(1.0, 0.1, (4, 40))
        ps.append(ensemble.permutation_p(G, O, n_perm=400, seed=t)[0])
    assert min(ps) > 0.005 and np.mean(ps) > 0.3


def test_permutation_p_catches_a_shift_and_heavy_tails_do_not_fool_it():
    rng = np.random.default_rng(1)
    G = rng.normal(1.0, 0.1, (64, 40))
    O = rng.normal(1.0, 0.1, (4, 40)) * 1.06
    assert ensemble.permutation_p(G, O, n_perm=2000)[0] < 1e-3
    # a heavy-tailed spread (lognormal scale per run) from one distribution
    Gh = rng.lognormal(0.0, 0.8, (64, 1)) * np.ones((1, 40))
    Oh = rng.lognormal(0.0, 0.8, (4, 1)) * np.ones((1, 40))
    assert ensemble.permutation_p(Gh, Oh, n_perm=2000)[0] > 1e-3


def test_paired_and_spread():
    rng = np.random.default_rng(2)
    G = rng.normal(1.0, 0.1, (16, 30))
    O = rng.normal(1.0, 0.1, (4, 30))
    Gp = O * (1.0 + rng.normal(0.0, 0.01, O.shape))
    assert ensemble.paired(Gp, O) < 0.2 * ensemble.spread(G)
    line = ensemble.compare(G, Gp, O, "synthetic")
    assert "paired" in line
    with pytest.raises(AssertionError):
        ensemble.compare(G, Gp * 1.5, O * 1.5, "shifted")


def test_traffic_pin_ignores_comments_but_not_code():
    a = "int x = 1; // one\n/* a block\n comment */ int y;"
    b = "int x = 1;\n\n   int y;   // another comment"
    assert bench.kernel_code(a) == bench.kernel_code(b)
    assert bench.kernel_code("int x = 1;") != bench.kernel_code("int x = 2;")
    assert len(bench.kernel_sources_sha256()) == 64


def test_sample_steps_in_a_window():
    # the push of level k samples when (k + 1) % 40 == 0: levels 39, 79, ...
    assert bench.sample_steps(0, 39) == 0
    assert bench.sample_steps(0, 40) == 1
    assert bench.sample_steps(39, 1) == 1
    assert bench.sample_steps(40, 39) == 0
    assert bench.sample_steps(1000, 4000) == 100
    assert bench.sample_steps(7, 20, every=0) == 0
    # a 20-step window holds one sample step for half of its start levels
    assert sum(bench.sample_steps(k, 20) for k in range(40)) == 20
