"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every function include/ecpic.h declares; the host-side grid generator of the
library reproduces Table 2.  No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2308_13092_gb300 import build as B
from paper_2308_13092_gb300 import ecpic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ecpic.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ecpic_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ecpic_create", "ecpic_set_grid", "ecpic_add_species", "ecpic_set_gas",
              "ecpic_add_process", "ecpic_init", "ecpic_step", "ecpic_diagnostics"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    path = B.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the binding marshals exactly the declared functions
    assert set(ecpic.SIGNATURES) == set(declared_functions())


def test_library_is_built_for_sm103a():
    path = B.build()
    blob = open(path, "rb").read()
    assert b"sm_103a" in blob or b"sm_103" in blob


def _table2():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "table2_cells.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("dmin,dmax,cells", _table2())
def test_library_doubling_grid_table2(dmin, dmax, cells):
    e = ecpic.ecpic_doubling_grid(2048, 0.3, 0.05, dmin, dmax)
    assert e.size - 1 == cells
    assert e[0] == 0.0 and e[-1] == 0.3 and np.all(np.diff(e) > 0)


def test_library_doubling_grid_cfg3_case():
    e = ecpic.ecpic_doubling_grid(1024, 0.3, 0.05, 4, 32)
    assert e.size - 1 == 114
