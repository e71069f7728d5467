"""Allocation-free deposit entry point (ecpic_deposit_device_noalloc) through
the C ABI.  On the same seeded (cell, xi) input it must give the sums of
ecpic_deposit_device and of the oracle's fixed-point rule (Eq. 2-3 in units of
2^-32 particle); the sums are integers, so the tolerance is zero.  Checked on
two calls in a row, with the device's free memory not shrinking across them.
The file name puts it last in the suite, so it runs both alone and after the
other tests."""
import gc

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

E_MAX_CELLS = 2048  # ECPIC_NOALLOC_MAX_CELLS


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_13092_gb300 import ecpic
    ecpic.lib()
    return ecpic


def _inputs(seed, N, n):
    rng = np.random.default_rng(seed)
    cell = rng.integers(-1, N, n).astype(np.int32)  # -1: absorbed, skipped
    cell[: n // 2].sort()  # half in cell order, half random
    xi = rng.random(n).astype(np.float32)
    xi[:7] = 0.0
    xi[7:14] = np.float32(1) - np.float32(2 ** -24)
    return (torch.from_numpy(cell).cuda(), torch.from_numpy(xi).cuda())


def _reference(E, N, cell, xi):
    S = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    E.ecpic_deposit_device(N, cell.numel(), cell.data_ptr(), xi.data_ptr(), S.data_ptr())
    return S


def test_noalloc_deposit_equals_deposit_device_two_calls(E):
    cases = [(11, 1024, 300001), (12, 2048, (1 << 20) + 3)]
    inputs = [_inputs(seed, N, n) for seed, N, n in cases]
    refs = [_reference(E, N, c, x) for (_, N, _), (c, x) in zip(cases, inputs)]
    outs = [torch.zeros(N + 1, dtype=torch.int64, device="cuda") for _, N, _ in cases]
    warm = torch.zeros(cases[0][1] + 1, dtype=torch.int64, device="cuda")
    # first call: one-time set-up (scratch address lookup, module load)
    c0, x0 = inputs[0]
    E.ecpic_deposit_device_noalloc(cases[0][1], c0.numel(), c0.data_ptr(), x0.data_ptr(), warm.data_ptr())
    torch.cuda.synchronize()
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        free_before = torch.cuda.mem_get_info()[0]
        for (_, N, n), (c, x), S in zip(cases, inputs, outs):  # two calls in a row
            E.ecpic_deposit_device_noalloc(N, n, c.data_ptr(), x.data_ptr(), S.data_ptr())
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
    finally:
        gc.enable()
    assert free_after >= free_before
    assert torch.equal(warm, refs[0])
    for (_, N, n), (c, x), S, R in zip(cases, inputs, outs, refs):
        assert torch.equal(S, R)
        live = int((c >= 0).sum())
        assert int(S.sum()) == live * 2 ** 32
        # the oracle's fixed-point rule on the same input (absorbed skipped)
        ch, xh = c.cpu().numpy(), x.cpu().numpy()
        keep = ch >= 0
        So = oracle.deposit_fixed(N, ch[keep], xh[keep])
        assert np.array_equal(S.cpu().numpy().view(np.uint64), So)


def test_noalloc_deposit_accumulates_and_limits(E):
    N, n = 300, 40000
    c, x = _inputs(5, N, n)
    R = _reference(E, N, c, x)
    S = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        E.ecpic_deposit_device_noalloc(N, n, c.data_ptr(), x.data_ptr(), S.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(S, 2 * R)
    E.ecpic_deposit_device_noalloc(N, 0, 0, 0, S.data_ptr())  # nothing to add
    torch.cuda.synchronize()
    assert torch.equal(S, 2 * R)
    with pytest.raises(E.EcpicError) as err:
        E.ecpic_deposit_device_noalloc(E_MAX_CELLS + 1, n, c.data_ptr(), x.data_ptr(), S.data_ptr())
    assert err.value.code == E.ECPIC_ERR_CAPACITY
