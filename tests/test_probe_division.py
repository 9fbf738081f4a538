"""The forest's probe offsets divide by the pixel's depth with multiply-high instructions instead
of an integer division (the kernels' DepthDivisor forms in csrc/forest.cu).  These tests check
both forms exhaustively against truncating integer division, trunc(delta * 1000 / d), which is the
reading of the depth-adaptive offset (Sec. 3.3: each agent's relocaliser is a regression forest;
its split features are the library's integer reading of the published depth-adaptive pixel-pair
differences).  Host arithmetic only: 32-bit multiply-high emulated with 64-bit integers."""
import numpy as np


def _trunc_div(n, d):
    q = np.abs(n) // d
    return np.where(n < 0, -q, q)


def _mulhi(a, b):
    """High word of the signed 32 x 32-bit product (an arithmetic shift of the 64-bit product)."""
    return (a.astype(np.int64) * b.astype(np.int64)) >> 32


def test_shifted_offset_form_is_exact_for_every_depth_and_offset():
    """Offsets with |delta| <= 255 stored times 128, d in [16, 65535]:
    trunc(delta * 1000 / d) = mulhi(128 delta, floor(2^25 * 1000 / d) + 1) + [delta < 0]."""
    delta = np.arange(-255, 256, dtype=np.int64)
    for d0 in range(16, 65536, 4096):
        d = np.arange(d0, min(d0 + 4096, 65536), dtype=np.int64)[:, None]
        m7 = (1000 << 25) // d + 1
        assert (m7 < 2 ** 31).all()                       # a positive signed 32-bit multiplier
        raw = 128 * delta[None, :]
        got = _mulhi(raw, m7) + (raw < 0)
        assert np.array_equal(got, _trunc_div(delta[None, :] * 1000, d)), d0


def test_shift_form_is_exact_for_depths_from_65():
    """Any int16 offset, d in [65, 65535]: with l = ceil(log2 d), M = floor(2^(25 + l) / d) + 1,
    trunc(n / d) = (mulhi(n, M) >> (25 + l - 32)) + [n < 0] for n = 1000 delta.  Every d, all
    offsets up to 300 in magnitude and a seeded sample of the rest of the int16 range."""
    rng = np.random.default_rng(3)
    delta = np.unique(np.concatenate([np.arange(-300, 301), rng.integers(-32768, 32768, 600),
                                      [-32768, 32767]])).astype(np.int64)
    n = delta * 1000
    for d0 in range(65, 65536, 2048):
        d = np.arange(d0, min(d0 + 2048, 65536), dtype=np.int64)[:, None]
        l = np.ceil(np.log2(d)).astype(np.int64)
        l = np.where((1 << l) < d, l + 1, l)              # exact ceil(log2 d)
        l = np.where((1 << (l - 1)) >= d, l - 1, l)
        shift = 25 + l
        assert (shift >= 32).all()
        m = (np.int64(1) << shift) // d + 1
        assert (m < 2 ** 31).all()
        got = (_mulhi(n[None, :], m) >> (shift - 32)) + (n[None, :] < 0)
        assert np.array_equal(got, _trunc_div(n[None, :], d)), d0


def test_the_shifted_form_fails_without_its_bounds():
    """The bounds matter: at d = 15 the multiplier no longer fits a signed word, and an offset of
    300 breaks the exactness bound |delta| d < 2^25 at the largest depths."""
    assert (1000 << 25) // 15 + 1 >= 2 ** 31
    d = np.arange(60000, 65536, dtype=np.int64)[:, None]
    delta = np.arange(256, 600, dtype=np.int64)[None, :]
    m7 = (1000 << 25) // d + 1
    got = _mulhi(128 * delta, m7)
    assert not np.array_equal(got, _trunc_div(delta * 1000, d))
