"""CPU model of the register-streaming 2D kernel: packed for 1- and 2-byte
elements (windows up to 9 x 9 for u8, 9 x 5 for i16), one column per word
for f32 (up to 9 x 9), checked against the oracle's literal rectangle
maximum and minimum.

Each thread holds one 32-bit word of 4 (u8) or 2 (i16) output columns and
streams a band of output rows; a warp covers 31 words of a row and its lane
31 computes the next warp's first word as well (a halo, for the stores); for
f32 a warp covers 33 - wx words, the window's next columns coming from the
next lanes (the last wx - 1 lanes a halo whose outputs are not stored).  Row pass: the input words at the thread's
columns and the next two, the window's elements taken as byte-shifted words
(funnel shifts of two neighbouring words) and combined per element (SIMD
max/min of packed lanes).  Column pass: per tile of 8 output rows, the row
results of rows y .. y+15 combined by doubling (Table 1's naive windows
shared between neighbours, as in the other 2D kernels).  Stores: output rows
are dense (width Wo), so a row's words are generally not 4-byte aligned; with
a = the byte misalignment of a warp's first word, lanes 0 .. 30 store the
aligned word made of their bytes [4-a, 4) and the next lane's bytes [0, 4-a)
(one shuffle; lane 30's next is the halo), lane 31 stores nothing, and the
first warp of a row stores its lane 0's bytes [0, 4-a) (the row's start);
only columns below Wo are stored, whole words where all are, element by
element otherwise.  This model runs those steps on
bytes and checks that every output byte is written exactly once with the
rectangle's value, for several widths (every misalignment), band and tile
edges, windows and element sizes, and that a planted ownership mistake is
caught (and a funnel shift of 32 bits, which wraps to 0)."""
import numpy as np
import pytest

import oracle
import synth

BAND, TILE = 64, 8


def _words(row_bytes, j):
    """Word j of a row (little-endian), zero past the row's end."""
    b = row_bytes[4 * j:4 * j + 4]
    b = np.concatenate([b, np.zeros(4 - len(b), np.uint8)]) if len(b) < 4 else b
    return int.from_bytes(b.tobytes(), "little")


def _elems(word, sz):
    return [(word >> (8 * sz * i)) & ((1 << (8 * sz)) - 1) for i in range(4 // sz)]


def _pack(vals, sz):
    w = 0
    for i, v in enumerate(vals):
        w |= (int(v) & ((1 << (8 * sz)) - 1)) << (8 * sz * i)
    return w


def _funnel(lo, hi, shift):
    """The 32 low bits of hi:lo shifted right by shift mod 32 (funnel shift)."""
    return ((hi << 32 | lo) >> (shift & 31)) & 0xFFFFFFFF


def _model(img, wy, wx, mistake=None):
    H, W = img.shape
    sz = img.dtype.itemsize
    L = 4 // sz
    signed = img.dtype == np.int16
    f32 = img.dtype == np.float32
    Ho, Wo = H - wy + 1, W - wx + 1
    nwc = -(-Wo // L)
    chunk_w = 33 - wx if f32 else 31  # f32: the last wx-1 lanes are a halo
    nchunks = -(-nwc // chunk_w)
    out = {"max": np.zeros(Ho * Wo * sz, np.uint8), "min": np.zeros(Ho * Wo * sz, np.uint8)}
    written = {k: np.zeros(Ho * Wo * sz, np.int32) for k in out}
    raw = img.view(np.uint8).reshape(H, W * sz)

    def as_val(e):
        if f32:
            return float(np.array([e], np.uint32).view(np.float32)[0])
        return e - (1 << 16) if signed and e >= 1 << 15 else e

    def as_bits(v):
        return int(np.array([v], np.float32).view(np.uint32)[0]) if f32 else v

    def row_result(y, j):
        """(max word, min word) of the window row pass at word column j."""
        if y >= H:
            return 0, 0
        w0, w1, w2 = (_words(raw[y], j + i) for i in range(3))
        m = n = None
        for k in range(wx):
            if f32:  # word j + k: the next lanes' words, taken by shuffles
                ev = [as_val(_words(raw[y], j + k))]
                m = ev if m is None else [max(a, b) for a, b in zip(m, ev)]
                n = ev if n is None else [min(a, b) for a, b in zip(n, ev)]
                continue
            b = k * sz  # the kernel's word choice; a funnel shift takes its count modulo 32
            if b < 4:
                s = _funnel(w0, w1, 8 * b)
            elif b < 8 or mistake == "funnel_wrap":
                s = _funnel(w1, w2, 8 * (b - 4))
            else:
                s = w2
            ev = [as_val(e) for e in _elems(s, sz)]
            m = ev if m is None else [max(a, b) for a, b in zip(m, ev)]
            n = ev if n is None else [min(a, b) for a, b in zip(n, ev)]
        return _pack([as_bits(v) for v in m], sz), _pack([as_bits(v) for v in n], sz)

    def col_op(words, opf):
        return _pack([as_bits(opf(vs)) for vs in zip(*[[as_val(e) for e in _elems(w, sz)] for w in words])], sz)

    for band in range(-(-Ho // BAND)):
        y0, y1 = band * BAND, min(band * BAND + BAND, Ho)
        for chunk in range(nchunks):
            for y in range(y0, y1):
                rm = {}
                for lane in range(32):
                    j = chunk * chunk_w + lane
                    rows = [row_result(y + i, j) for i in range(wy)]
                    rm[lane] = (col_op([r[0] for r in rows], max), col_op([r[1] for r in rows], min))
                ob0 = (y * Wo + chunk * chunk_w * L) * sz  # byte offset of lane 0's first column
                a = ob0 % 4  # the kernel takes it from the address; the output base is 4-aligned here
                for side, si in (("max", 0), ("min", 1)):
                    def put(byte_off, col, val):
                        if col < Wo:
                            out[side][byte_off:byte_off + sz] = np.frombuffer(int(val).to_bytes(sz, "little"),
                                                                              np.uint8)
                            written[side][byte_off:byte_off + sz] += 1
                    for lane in range(32):
                        v = rm[lane][si]
                        x0 = (chunk * chunk_w + lane) * L
                        ob = ob0 + lane * 4
                        if lane >= chunk_w and mistake != "halo_stores":
                            continue  # the halo: the next warp's first words
                        if a == 0:
                            for e in range(L):
                                put(ob + e * sz, x0 + e, _elems(v, sz)[e])
                            continue
                        nxt = rm[lane + 1][si] if lane < 31 else v
                        aw = ((nxt << 32 | v) >> (8 * (4 - a))) & 0xFFFFFFFF
                        for e in range(L):
                            put(ob + (4 - a) + e * sz, x0 + (4 - a) // sz + e, _elems(aw, sz)[e])
                        if lane == 0 and chunk == 0 and mistake != "no_head":
                            for e in range((4 - a) // sz):
                                put(ob + e * sz, x0 + e, _elems(v, sz)[e])
    for side in out:
        assert (written[side] == 1).all(), f"{side}: bytes written {np.unique(written[side])} times"
    return (out["max"].view(img.dtype).reshape(Ho, Wo), out["min"].view(img.dtype).reshape(Ho, Wo))


@pytest.mark.parametrize("dtype", [np.uint8, np.int16, np.float32])
@pytest.mark.parametrize("W", [131, 132, 133, 134, 261])
def test_packed_model_against_rectangle(dtype, W):
    if dtype == np.float32 and W not in (133, 261):
        pytest.skip("f32 words are always aligned: two widths suffice")
    rng = np.random.default_rng(W)
    img = synth.blobs2d(1, 75, W, seed=W, dtype=dtype, nblobs=6)[0]
    if dtype == np.int16:
        img = (img.astype(np.int32) - 16000).astype(np.int16)
    if dtype == np.float32:
        img = (img - np.float32(0.5)).astype(np.float32)  # negative values too
    maxwx = 5 if dtype == np.int16 else 9
    for wy, wx in ((3, 3), (1, 1), (9, maxwx), (2, 1), (1, 4), (int(rng.integers(1, 10)), int(rng.integers(1, maxwx + 1)))):
        gm, gn = _model(img, wy, wx)
        em, en = oracle.bf2d(img, wy, wx)
        assert np.array_equal(gm, em) and np.array_equal(gn, en), (wy, wx)


def test_packed_model_planted_mistakes():
    img = synth.blobs2d(1, 10, 133, seed=1, dtype=np.uint8, nblobs=3)[0]  # Wo = 131: every misalignment
    with pytest.raises(AssertionError, match="written"):
        _model(img, 2, 3, mistake="no_head")
    with pytest.raises(AssertionError, match="written"):
        img2 = synth.blobs2d(1, 10, 300, seed=1, dtype=np.uint8, nblobs=3)[0]  # three chunks per row
        _model(img2, 2, 3, mistake="halo_stores")
    # Byte offset 8 (u8 windows of 9, i16 of 5) taken as a shift of 32 wraps
    # to the middle word; f32 halo lanes that store overwrite the next warp's
    # words with wrong values.
    gm, gn = _model(img, 1, 9, mistake="funnel_wrap")
    em, en = oracle.bf2d(img, 1, 9)
    assert not (np.array_equal(gm, em) and np.array_equal(gn, en))
    imf = synth.blobs2d(1, 10, 80, seed=2, dtype=np.float32, nblobs=3)[0]
    with pytest.raises(AssertionError, match="written"):
        _model(imf, 2, 5, mistake="halo_stores")
