"""GPU parity of the window-3 two-comparison filter (Section 3) against the
oracle's restatement of the same scheme: values bit for bit, and the GPU's
comparison count equal to the oracle's count summed over the GPU's chunks of
16 outputs (each chunk starts its own pair)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

CHUNK = 16


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _expected_count(a):
    m = a.size - 2
    total = 0
    for j0 in range(0, m, CHUNK):
        _, _, c = oracle.w3(a[j0:min(j0 + CHUNK, m) + 2])
        total += c
    return total


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int16, np.uint8])
@pytest.mark.parametrize("n", [3, 4, 17, 18, 19, 530, 4099, 100_003])
def test_w3_matches_oracle(mmf, dtype, n):
    a = synth.random_walk(n, seed=n, dtype=dtype)
    x = torch.from_numpy(a).cuda()
    mx, mn, cnt = mmf.filter1d_w3(x, count=True)
    torch.cuda.synchronize()
    emx, emn, _ = oracle.w3(a)
    assert np.array_equal(mx.cpu().numpy(), emx) and np.array_equal(mn.cpu().numpy(), emn)
    m = n - 2
    assert int(cnt.item()) == -(-m // CHUNK) + 2 * m == _expected_count(a)


@pytest.mark.parametrize("off", [1, 2, 3, 5])
def test_w3_views_and_ties(mmf, off):
    """Misaligned views take the scalar path; ties and plateaus give the same
    values as the oracle (and as the window-3 definition)."""
    for a in (synth.random_walk(10_007, seed=off, dtype=np.float32),
              (synth.uniform(10_007, seed=off, dtype=np.uint8) // 100).astype(np.uint8),
              np.repeat(synth.random_walk(2000, seed=off, dtype=np.int16), 5)):
        x = torch.from_numpy(a).cuda()[off:]
        mx, mn = mmf.filter1d_w3(x)
        torch.cuda.synchronize()
        emx, emn, _ = oracle.w3(a[off:])
        bmx, bmn = oracle.bf1d(a[off:], 3)
        assert np.array_equal(mx.cpu().numpy(), emx) and np.array_equal(mn.cpu().numpy(), emn)
        assert np.array_equal(emx, bmx) and np.array_equal(emn, bmn)


def test_w3_full_size_against_default_kernel(mmf):
    """n = 2^28 f32: the two-comparison kernel equals the library's default
    w = 3 filter (the register slide) at every output, and the count is
    ceil((n-2)/16) + 2(n-2)."""
    n = 1 << 28
    x = synth.torch_by_name("uniform", n, 7, torch.device("cuda"))
    mx, mn, cnt = mmf.filter1d_w3(x, count=True)
    dmx, dmn = mmf.filter1d(x, 3)
    torch.cuda.synchronize()
    assert torch.equal(mx, dmx) and torch.equal(mn, dmn)
    m = n - 2
    assert int(cnt.item()) == -(-m // CHUNK) + 2 * m
    idx = np.random.default_rng(3).integers(0, m, 200)
    xs = x.cpu().numpy()
    for j in idx:
        assert mx[j].item() == xs[j:j + 3].max() and mn[j].item() == xs[j:j + 3].min()
    del x, mx, mn, dmx, dmn
    torch.cuda.empty_cache()


def test_w3_small_and_null_outputs(mmf):
    x = torch.arange(2, dtype=torch.float32, device="cuda")
    mx, mn = mmf.filter1d_w3(x)
    assert mx.numel() == 0
    assert mmf.device_status() == 0
