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


@pytest.mark.parametrize("fuse", [0, 1, -1])
@pytest.mark.parametrize("dtype", [np.float32, np.uint8, np.float64, np.int16])
@pytest.mark.parametrize("wy,wx", WINDOWS)
def test_2d_windows(mmf, dtype, wy, wx, fuse):
    """Unfused (row pass to a workspace, then columns), fused (the shared
    memory tile kernel up to 31 x 31, else row maxima computed inside the
    column pass) and the automatic choice against the literal rectangle."""
    imgs = synth.blobs2d(2, 300, 262, seed=wy * 7 + wx, dtype=dtype, nblobs=20)
    if dtype == np.int16:
        imgs = (imgs.astype(np.int32) - 16000).astype(np.int16)
    x = torch.from_numpy(imgs).cuda()
    if fuse == 1 and wx > 64 and wy > 1:
        with pytest.raises(mmf.MMFError):
            mmf.filter2d(x, wy, wx, fuse=1)
        return
    mx, mn = mmf.filter2d(x, wy, wx, fuse=fuse)
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
    for wy, wx, fuse in ((5, 6, 0), (5, 6, 1), (40, 1, -1), (1, 40, -1), (33, 71, 0), (33, 17, 1), (12, 3, 1),
                         (31, 31, -1), (2, 30, 1), (31, 2, 1), (16, 16, -1)):
        mx, mn = mmf.filter2d(x, wy, wx, fuse=fuse)
        torch.cuda.synchronize()
        for k in range(3):
            em, en = _expect(full[k, :, :501], wy, wx)
            assert np.array_equal(mx[k].cpu().numpy(), em) and np.array_equal(mn[k].cpu().numpy(), en)


def test_2d_row_pass_as_one_series(mmf):
    """The two-pass form with a workspace large enough for the row pass to
    filter every row of every image as one series: over padded rows (the
    windows that straddle a row's padding are computed and never read) and
    dense ones, against the literal rectangle; then the same pitched images
    with the queried workspace, which takes the rows one by one."""
    full = synth.blobs2d(3, 131, 517, seed=5, dtype=np.float32, nblobs=9)
    base = torch.from_numpy(full).cuda()
    big = torch.empty(2 * 3 * 131 * 528 * 4, dtype=torch.uint8, device="cuda")
    for x, width in ((base[:, :, :501], 501), (base, 517)):
        for wy, wx in ((5, 6), (33, 71), (2, 2), (40, 200), (3, 501 if width == 501 else 517)):
            for ws in (big, None):
                mx, mn = mmf.filter2d(x, wy, wx, fuse=0, workspace=ws)
                torch.cuda.synchronize()
                for k in range(3):
                    em, en = _expect(full[k, :, :width], wy, wx)
                    assert np.array_equal(mx[k].cpu().numpy(), em), (width, wy, wx, ws is None, k)
                    assert np.array_equal(mn[k].cpu().numpy(), en), (width, wy, wx, ws is None, k)
    for dtype in (np.uint8, np.int16, np.float64):
        imgs = synth.blobs2d(2, 70, 150, seed=6, dtype=dtype, nblobs=4)
        x = torch.from_numpy(imgs).cuda()
        for wy, wx in ((4, 11), (20, 3)):
            mx, mn = mmf.filter2d(x, wy, wx, fuse=0)
            torch.cuda.synchronize()
            for k in range(2):
                em, en = _expect(imgs[k], wy, wx)
                assert np.array_equal(mx[k].cpu().numpy(), em) and np.array_equal(mn[k].cpu().numpy(), en)
    assert mmf.device_status() == 0


@pytest.mark.parametrize("dtype", [np.uint8, np.int16])
def test_2d_fused_odd_width_unpaired(mmf, dtype):
    """Odd output widths and offset views take the one-column-per-thread
    forms of the fused kernel."""
    full = synth.blobs2d(2, 77, 300, seed=8, dtype=dtype, nblobs=5)
    base = torch.from_numpy(full).cuda()
    for off, wx in ((0, 4), (1, 3), (3, 8)):
        x = base[:, :, off:off + 251]
        mx, mn = mmf.filter2d(x, 6, wx, fuse=1)
        torch.cuda.synchronize()
        for k in range(2):
            em, en = _expect(full[k, :, off:off + 251], 6, wx)
            assert np.array_equal(mx[k].cpu().numpy(), em) and np.array_equal(mn[k].cpu().numpy(), en)


@pytest.mark.parametrize("dtype", [np.uint8, np.int16, np.float32])
def test_2d_packed_every_window(mmf, dtype):
    """The register-streaming kernel (fuse = 2): every window up to 9 x 9
    (9 x 5 for i16); output widths of every residue modulo the word (rows of
    the dense outputs start at every byte misalignment), several warp chunks
    per row, bands of 64 rows with a ragged last one, against the literal
    rectangle."""
    imgs = synth.blobs2d(2, 150, 300, seed=5, dtype=dtype, nblobs=12)
    if dtype == np.int16:
        imgs = (imgs.astype(np.int32) - 16000).astype(np.int16)
    if dtype == np.float32:
        imgs = (imgs - np.float32(0.5)).astype(np.float32)
    x = torch.from_numpy(imgs).cuda()
    maxwx = 5 if dtype == np.int16 else 9
    for wy in range(1, 10):
        for wx in range(1, maxwx + 1):
            mx, mn = mmf.filter2d(x, wy, wx, fuse=2)
            torch.cuda.synchronize()
            for k in range(2):
                em, en = _expect(imgs[k], wy, wx)
                assert np.array_equal(mx[k].cpu().numpy(), em), (wy, wx, k)
                assert np.array_equal(mn[k].cpu().numpy(), en), (wy, wx, k)
    assert mmf.device_status() == 0


@pytest.mark.parametrize("dtype", [np.uint8, np.int16, np.float32])
def test_2d_packed_pitch_offsets_and_refusals(mmf, dtype):
    """Pitched input rows, output buffers starting at every misalignment, a
    single output column, an image narrower than one word; misaligned input
    rows are refused by the forced packed kernel and take another kernel in
    the automatic choice (f32 rows are always word-aligned)."""
    full = synth.blobs2d(3, 90, 308, seed=6, dtype=dtype, nblobs=7)
    base = torch.from_numpy(full).cuda()
    x = base[:, :, :300]  # pitch 308 elements
    n, H = 3, 90
    for wy, wx, off in ((3, 3, 1), (5, 2, 2), (9, 5, 3), (2, 4, 0), (1, 5, 1), (4, 1, 3)):
        Ho, Wo = H - wy + 1, 300 - wx + 1
        bm = torch.empty(n * Ho * Wo + 8, dtype=x.dtype, device="cuda")
        bn = torch.empty(n * Ho * Wo + 8, dtype=x.dtype, device="cuda")
        om = bm[off:off + n * Ho * Wo].view(n, Ho, Wo)
        on = bn[(off + 1) % 4:(off + 1) % 4 + n * Ho * Wo].view(n, Ho, Wo)
        mmf.filter2d(x, wy, wx, fuse=2, out_max=om, out_min=on)
        torch.cuda.synchronize()
        for k in range(n):
            em, en = _expect(full[k, :, :300], wy, wx)
            assert np.array_equal(om[k].cpu().numpy(), em) and np.array_equal(on[k].cpu().numpy(), en), (wy, wx)
    maxwx = 5 if dtype == np.int16 else 9
    for W, wx in ((maxwx, maxwx), (3, 2), (2, 1)):
        xs = base[:, :, :W]
        mx, mn = mmf.filter2d(xs, 3, wx, fuse=2)
        torch.cuda.synchronize()
        for k in range(n):
            em, en = _expect(full[k, :, :W], 3, wx)
            assert np.array_equal(mx[k].cpu().numpy(), em) and np.array_equal(mn[k].cpu().numpy(), en), (W, wx)
    xo = base[:, :, 1:301]  # rows start one element off a 4-byte boundary (not for f32)
    if dtype != np.float32:
        with pytest.raises(mmf.MMFError) as e:
            mmf.filter2d(xo, 3, 3, fuse=2)
        assert e.value.status == 7
    mx, mn = mmf.filter2d(xo, 3, 3, fuse=2 if dtype == np.float32 else -1)
    torch.cuda.synchronize()
    for k in range(n):
        em, en = _expect(full[k, :, 1:301], 3, 3)
        assert np.array_equal(mx[k].cpu().numpy(), em) and np.array_equal(mn[k].cpu().numpy(), en)
    with pytest.raises(mmf.MMFError) as e:
        mmf.filter2d(x, 10, 3, fuse=2)
    assert e.value.status == 7
    with pytest.raises(mmf.MMFError) as e:
        mmf.filter2d(x.double(), 3, 3, fuse=2)
    assert e.value.status == 7
    with pytest.raises(mmf.MMFError) as e:
        mmf.filter2d(x, 3, 3, fuse=3)
    assert e.value.status == 1
    assert mmf.device_status() == 0


def test_2d_window_larger_than_image(mmf):
    x = torch.rand(2, 10, 12, device="cuda")
    mx, mn = mmf.filter2d(x, 11, 3)
    assert mx.numel() == 0 and mn.numel() == 0
    mx, mn = mmf.filter2d(x, 10, 12)
    assert torch.equal(mx.reshape(-1), x.amax(dim=(1, 2))) and torch.equal(mn.reshape(-1), x.amin(dim=(1, 2)))


def test_2d_fused_limits(mmf):
    """A forced fused request beyond the fused kernel's row window is refused;
    within it no workspace is needed."""
    x = torch.rand(1, 128, 128, device="cuda")
    with pytest.raises(mmf.MMFError):
        mmf.filter2d(x, 3, 65, fuse=1)
    lib = mmf.load()
    import ctypes
    need = ctypes.c_size_t(1)
    assert lib.mmf_filter2d_workspace(1, 128, 128, 3, 3, 0, 1, ctypes.byref(need)) == 0 and need.value == 0
    assert lib.mmf_filter2d_workspace(1, 128, 128, 3, 3, 0, 0, ctypes.byref(need)) == 0 and need.value > 0


def test_2d_full_size_sampled(mmf):
    """A 4096 x 4096 image (the 2D workload's image size), sampled pixels
    against the literal rectangle."""
    img = synth.blobs2d(1, 4096, 4096, seed=41, dtype=np.uint8, nblobs=200)
    x = torch.from_numpy(img).cuda()
    rng = np.random.default_rng(4)
    for wy, wx, fuse in ((3, 3, 0), (3, 3, 1), (3, 3, 2), (7, 9, 2), (15, 15, 0), (15, 15, 1), (63, 63, -1),
                         (255, 1, -1), (1, 255, -1)):
        mx, mn = mmf.filter2d(x, wy, wx, fuse=fuse)
        torch.cuda.synchronize()
        ys = rng.integers(0, 4096 - wy + 1, 2000)
        xs = rng.integers(0, 4096 - wx + 1, 2000)
        em, en = oracle.bf2d_at(img[0], wy, wx, ys, xs)
        gm = mx[0].cpu().numpy()[ys, xs]
        gn = mn[0].cpu().numpy()[ys, xs]
        assert np.array_equal(gm, em) and np.array_equal(gn, en)
    assert mmf.device_status() == 0
