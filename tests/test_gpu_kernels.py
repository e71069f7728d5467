"""GPU parity of the kernel-level entry points against the oracle, through the
C ABI: Philox4x32-10 bit for bit, and the warp-aggregated fixed-point CIC
deposit bit for bit on identical (cell, xi) input (Eq. 2-3)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_13092_gb300 import ecpic
    ecpic.lib()
    return ecpic


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_philox_device_matches_oracle(E):
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = 0
    ctr[16:32, 3] = 0xFFFFFFFF
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    dc, dk = _dev(ctr.view(np.int32)), _dev(key.view(np.int32))
    out = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    E.ecpic_philox_device(n, dc.data_ptr(), dk.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    for i in list(range(64)) + list(rng.choice(n, 200, replace=False)):
        assert oracle.philox4x32_10(ctr[i], key[i]) == [int(v) for v in got[i]]


def _deposit_case(E, N, cell, xi):
    S = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    dc, dx = _dev(cell.astype(np.int32)), _dev(xi.astype(np.float32))
    E.ecpic_deposit_device(N, cell.size, dc.data_ptr(), dx.data_ptr(), S.data_ptr())
    torch.cuda.synchronize()
    got = S.cpu().numpy().view(np.uint64)
    keep = cell >= 0
    want = oracle.deposit_fixed(N, cell[keep], xi[keep])
    return got, want


@pytest.mark.parametrize("N,n,order", [(1, 5, "random"), (7, 1000, "random"), (128, 33, "sorted"),
                                       (1024, 300001, "sorted"), (1024, 300001, "random"),
                                       (2048, 1 << 20, "sorted"), (64, 2 ** 22 + 17, "clustered")])
def test_deposit_device_bit_exact(E, N, n, order):
    rng = np.random.default_rng(N * 7 + n)
    if order == "clustered":
        cell = rng.integers(N // 2 - 1, N // 2 + 1, n).astype(np.int32)
    else:
        cell = rng.integers(0, N, n).astype(np.int32)
    if order == "sorted":
        cell.sort()
    xi = rng.random(n).astype(np.float32)
    # faces and extreme shares
    k = min(n, 64)
    xi[:k // 3] = 0.0
    xi[k // 3: 2 * k // 3] = np.float32(1) - np.float32(2 ** -24)
    xi[2 * k // 3: k] = np.float32(2 ** -30)
    got, want = _deposit_case(E, N, cell, xi)
    assert np.array_equal(got, want)
    assert int(got.sum(dtype=np.uint64)) == n * 2 ** 32


@pytest.mark.parametrize("N,order", [(2048, "random"), (96, "clustered")])
def test_deposit_device_many_flushes(E, N, order):
    # 2^25 + 5 particles over at most 304 blocks: each block adds more than
    # 65,536 particles, so its shared sums are flushed to S mid-way
    n = (1 << 25) + 5
    rng = np.random.default_rng(N)
    if order == "clustered":
        cell = rng.integers(N // 2 - 2, N // 2 + 2, n).astype(np.int32)
    else:
        cell = rng.integers(0, N, n).astype(np.int32)
    xi = rng.random(n, dtype=np.float32)
    xi[:1000] = np.float32(1) - np.float32(2 ** -24)
    got, want = _deposit_case(E, N, cell, xi)
    assert np.array_equal(got, want)
    assert int(got.sum(dtype=np.uint64)) == n * 2 ** 32


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("N,n,order", [(8, 3000, "random"), (256, 200001, "sorted"),
                                       (1024, 500003, "random")])
def test_deposit2_device_bit_exact(E, bc, N, n, order):
    # EC2 quadratic-spline shares: the same integers as the oracle routine,
    # folds at Dirichlet walls and periodic wrap included
    rng = np.random.default_rng(N + n + bc)
    cell = rng.integers(0, N, n).astype(np.int32)
    if order == "sorted":
        cell.sort()
    xi = rng.random(n).astype(np.float32)
    edge = np.array([0.0, 0.5, np.nextafter(np.float32(0.5), np.float32(0)), 1 - 2.0 ** -24,
                     2.0 ** -30, 0.25], np.float32)
    xi[:edge.size] = edge
    cell[:edge.size] = [0, N - 1, 0, N - 1, N // 2, 0]
    S = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    dc, dx = _dev(cell), _dev(xi)
    E.ecpic_deposit_device2(N, bc, n, dc.data_ptr(), dx.data_ptr(), S.data_ptr())
    torch.cuda.synchronize()
    got = S.cpu().numpy().view(np.uint64)
    want = oracle.deposit_fixed2(N, bc, cell, xi)
    assert np.array_equal(got, want)


def test_deposit_device_skips_dead_and_empty(E):
    rng = np.random.default_rng(1)
    N, n = 100, 5000
    cell = rng.integers(-1, N, n).astype(np.int32)
    xi = rng.random(n).astype(np.float32)
    got, want = _deposit_case(E, N, cell, xi)
    assert np.array_equal(got, want)
    S = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    E.ecpic_deposit_device(N, 0, 0, 0, S.data_ptr())
    torch.cuda.synchronize()
    assert int(S.abs().sum()) == 0
