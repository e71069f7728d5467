"""Test glue: build oracle runs (and GPU runs) from the shared input recipes."""
from __future__ import annotations

import numpy as np

from paper_2308_13092_gb300 import inputs as I


def oracle_from_config(cfg: I.RunConfig, init: bool = True):
    from oracle import OracleRun
    o = OracleRun()
    o.set_grid(cfg.edges, cfg.bc, cfg.v0, cfg.freq, cfg.phase, cfg.vdc)
    o.set_scheme(cfg.scheme)
    for s in cfg.species:
        o.add_species(s.q, s.m, s.w, s.capacity)
    o.set_gas(cfg.n_gas, cfg.T_gas, cfg.m_gas)
    for p in cfg.processes:
        o.add_process(p.species, p.kind, p.threshold, p.dE, p.sigma, p.product)
    if cfg.sample_every:
        o.reset_averages(cfg.sample_every)
    if getattr(cfg, "quiet", False):
        o.set_quiet_start(True)
    if getattr(cfg, "tallies", None):
        o.set_tallies(**cfg.tallies)
    if getattr(cfg, "rebalance", None):
        o.set_rebalance(**cfg.rebalance)
    if init:
        o.init(cfg.seed, cfg.dt, [s.n0 for s in cfg.species], [s.T_eV for s in cfg.species])
    return o


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_from_config(cfg: I.RunConfig, **kw):
    from paper_2308_13092_gb300 import ecpic
    return ecpic.Run.from_config(cfg, **kw)


def require_gpu():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
