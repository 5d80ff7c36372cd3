"""Device random numbers through the C ABI: the library's Philox4x32-10
against cuRAND's Philox4_32_10 (an independent implementation run on the
GPU) and against the oracle, and the normal transform against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    oracle.build()
    return torch, pdd, oracle


def _blocks(torch, pdd, ctr, key, fn):
    c = torch.from_numpy(ctr.view(np.int32)).cuda()
    k = torch.from_numpy(key.view(np.int32)).cuda()
    out = torch.zeros(ctr.size, dtype=torch.int32, device="cuda")
    fn(c.data_ptr(), k.data_ptr(), out.data_ptr(), ctr.size // 4)
    return out.cpu().numpy().view(np.uint32).reshape(-1, 4)


def test_philox_matches_curand_and_oracle(env):
    torch, pdd, oracle = env
    rng = np.random.default_rng(11)
    n = 4096
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    # cuRAND takes the block index as an offset of 4 * block 32-bit outputs in a
    # 64-bit count: keep 4 * (ctr0 | ctr1 << 32) below 2^64
    ctr[:, 1] = 0
    ctr[: n // 2, 1] = rng.integers(0, 2**30, size=n // 2).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ours = _blocks(torch, pdd, ctr.reshape(-1).copy(), key.reshape(-1).copy(), pdd.pdd_debug_philox)
    ref = _blocks(torch, pdd, ctr.reshape(-1).copy(), key.reshape(-1).copy(),
                  pdd.pdd_debug_philox_curand)
    assert np.array_equal(ours, ref)
    for i in range(0, n, 97):
        assert np.array_equal(ours[i], oracle.philox4x32_10(ctr[i], key[i]))


@pytest.mark.parametrize("precision", [0, 1])
def test_normals_match_oracle(env, precision):
    torch, pdd, oracle = env
    count = 4000
    seed, tag, node, path = (77 << 32) + 5, 3, 12, 345
    dt = torch.float32 if precision == 0 else torch.float64
    out = torch.zeros(count, dtype=dt, device="cuda")
    ptr = out.data_ptr()
    pdd.pdd_debug_normals(seed, tag, node, path, 10, count, precision,
                          ptr if precision == 0 else None, ptr if precision == 1 else None)
    got = out.cpu().numpy().astype(np.float64)
    ref = oracle.normals(seed, tag, node, path, count, first=10)
    err = np.abs(got - ref)
    if precision == 1:
        assert err.max() < 1e-12
    else:
        # SFU log / sincos: ~1e-6 typical; the error grows where r = |n| is tiny
        assert np.mean(err < 2e-6) > 0.995
        assert err.max() < 1e-4
