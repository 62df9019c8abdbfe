"""GPU parity of the separable 2D filter against the oracle's literal
rectangle max/min (no separation on the oracle side); bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

WINDOWS = [(1, 1), (3, 3), (1, 7), (7, 1), (2, 5), (9, 9), (10, 10), (15, 15), (17, 4), (4, 33),
           (63, 63), (64, 3), (3, 64), (255, 1), (1, 255), (100, 13)]


@pytest.fixture(scope="module")
def mmf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_cs_0610046_gb300 as m
    return m


def _expect(img, wy, wx):
    return oracle.bf2d(img, wy, wx)


@pytest.mark.parametrize("dtype", [np.float32, np.uint8, np.float64, np.int16])
@pytest.mark.parametrize("wy,wx", WINDOWS)
def test_2d_windows(mmf, dtype, wy, wx):
    imgs = synth.blobs2d(2, 300, 262, seed=wy * 7 + wx, dtype=dtype, nblobs=20)
    if dtype == np.int16:
        imgs = (imgs.astype(np.int32) - 16000).astype(np.int16)
    x = torch.from_numpy(imgs).cuda()
    mx, mn = mmf.filter2d(x, wy, wx)
    torch.cuda.synchronize()
    for k in range(imgs.shape[0]):
        em, en = _expect(imgs[k], wy, wx)
        assert np.array_equal(mx[k].cpu().numpy(), em), f"max image {k}"
        assert np.array_equal(mn[k].cpu().numpy(), en), f"min image {k}"


def test_2d_pitched_rows_and_ragged(mmf):
    """Rows padded to a larger pitch, sizes not multiples of any tile."""
    full = synth.blobs2d(3, 131, 517, seed=3, dtype=np.float32, nblobs=9)
    base = torch.from_numpy(full).cuda()
    x = base[:, :, :501]  # pitch 517, width 501
    for wy, wx in ((5, 6), (40, 1), (1, 40), (33, 71)):
        mx, mn = mmf.filter2d(x, wy, wx)
        torch.cuda.synchronize()
        for k in range(3):
            em, en = _expect(full[k, :, :501], wy, wx)
            assert np.array_equal(mx[k].cpu().numpy(), em) and np.array_equal(mn[k].cpu().numpy(), en)


def test_2d_window_larger_than_image(mmf):
    x = torch.rand(2, 10, 12, device="cuda")
    mx, mn = mmf.filter2d(x, 11, 3)
    assert mx.numel() == 0 and mn.numel() == 0
    mx, mn = mmf.filter2d(x, 10, 12)
    assert torch.equal(mx.reshape(-1), x.amax(dim=(1, 2))) and torch.equal(mn.reshape(-1), x.amin(dim=(1, 2)))


def test_2d_fused_request_is_refused(mmf):
    x = torch.rand(1, 64, 64, device="cuda")
    with pytest.raises(mmf.MMFError):
        mmf.filter2d(x, 3, 3, fuse=1)


def test_2d_full_size_sampled(mmf):
    """A 4096 x 4096 image (the 2D workload's image size), sampled pixels
    against the literal rectangle."""
    img = synth.blobs2d(1, 4096, 4096, seed=41, dtype=np.uint8, nblobs=200)
    x = torch.from_numpy(img).cuda()
    rng = np.random.default_rng(4)
    for wy, wx in ((3, 3), (15, 15), (63, 63), (255, 1), (1, 255)):
        mx, mn = mmf.filter2d(x, wy, wx)
        torch.cuda.synchronize()
        ys = rng.integers(0, 4096 - wy + 1, 2000)
        xs = rng.integers(0, 4096 - wx + 1, 2000)
        em, en = oracle.bf2d_at(img[0], wy, wx, ys, xs)
        gm = mx[0].cpu().numpy()[ys, xs]
        gn = mn[0].cpu().numpy()[ys, xs]
        assert np.array_equal(gm, em) and np.array_equal(gn, en)
    assert mmf.device_status() == 0
