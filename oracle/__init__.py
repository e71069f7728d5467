"""FP64 CPU oracle for the EC-PIC 1D3V hot path (arXiv 2308.13092).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The GPU product never imports it.
"""
from .oracle import (  # noqa: F401
    OracleRun, build, lib, philox4x32_10, child_id, deposit_fixed, deposit_fixed2, deposit_fixed_w,
    poisson_thomas, poisson_dense, field, doubling_grid,
    ELASTIC, EXCITATION, IONIZATION, ION_ELASTIC, CX,
    DIRICHLET, PERIODIC, EC, MC, EC2, MC2,
)
