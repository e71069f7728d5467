"""Pins for the oracle's doubling grid generator (Sec. 3c rules 1-4) against
the cell counts printed in Table 2 and the estimate of Eq. 11-12."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_cells.txt")


def table2():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            a, b, c = (int(v) for v in line.split())
            rows.append((a, b, c))
    return rows


def test_golden_has_all_rows():
    assert len(table2()) == 15


@pytest.mark.parametrize("dmin,dmax,cells", table2())
def test_doubling_grid_reproduces_table2(dmin, dmax, cells):
    e = oracle.doubling_grid(2048, 0.3, 0.05, dmin, dmax)
    assert e.size - 1 == cells


@pytest.mark.parametrize("dmin,dmax,cells", table2())
def test_doubling_grid_rules(dmin, dmax, cells):
    L = 0.3
    e = oracle.doubling_grid(2048, L, 0.05, dmin, dmax)
    dx_ref = L / 2048
    dx = np.diff(e) / dx_ref
    k = np.round(dx).astype(int)
    assert np.allclose(dx, k, atol=1e-6)
    # sizes are dx_min times a power of two, within [dx_min, dx_max] (rules 2-3)
    assert k.min() >= dmin and k.max() <= dmax
    assert all(((v // dmin) & (v // dmin - 1)) == 0 and v % dmin == 0 for v in k)
    # neighbours differ by at most a factor 2 (rule 4)
    r = k[1:] / k[:-1]
    assert np.all((r >= 0.5) & (r <= 2.0))
    # buffer of dx_min cells from each electrode (rule 1), mirror symmetric
    nb = int(np.ceil(0.05 / (dmin * dx_ref) - 1e-9))
    assert np.all(k[:nb] == dmin) and np.all(k[-nb:] == dmin)
    assert np.array_equal(k, k[::-1])
    assert e[0] == 0.0 and e[-1] == L


@pytest.mark.parametrize("dmin,dmax,cells", table2())
def test_cell_count_estimate_eq11(dmin, dmax, cells):
    """Eq. 11 ignores the transition cells; the generator stays within them."""
    L, Lb, dx_ref = 0.3, 0.05, 0.3 / 2048
    est = (L - 2 * Lb) / (dmax * dx_ref) + 2 * Lb / (dmin * dx_ref)
    R = dmax / dmin
    CR = 2 * (1 - 1 / R) * Lb / L + 1 / R
    assert np.isclose(est / (L / (dmin * dx_ref)), CR, rtol=1e-12)   # Eq. 12 from Eq. 11
    n_trans = 2 * int(np.log2(R)) + 2
    assert abs(cells - est) <= n_trans * 1.0 + 1


def test_figure6_example_sizes():
    """Fig. 6: N_ref = 128, L_buff = 10 dx_ref, sizes 1, 2, 4, 8 dx_ref."""
    L = 1.0
    e = oracle.doubling_grid(128, L, 10 * L / 128, 1, 8)
    k = np.round(np.diff(e) / (L / 128)).astype(int)
    assert set(k.tolist()) == {1, 2, 4, 8}
    assert k.sum() == 128


def test_speedup_numbers_sec3d():
    """9.4x fewer cells (Table 2 last row) and its 2D/3D powers (Sec. 3d)."""
    cr = 2048 / (oracle.doubling_grid(2048, 0.3, 0.05, 4, 32).size - 1)
    assert round(cr, 1) == 9.4
    assert round(cr ** 2) == 88
    assert abs(cr ** 3 - 830) < 5
