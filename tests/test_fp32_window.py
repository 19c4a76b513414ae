"""The FP32C walk's opening criterion (Sec. 3 Eq. 5 in FP32) and the window in
which it takes the decision again in FP64.

The walk forms R = x_hi - c_hi from the target and centroid rounded to float,
d2 = R.R with fused multiply-adds, and compares with rcrit2 rounded to float.
Whenever |d2 - rcrit2| <= wa d2 + wb (wa = 4e-6 + b/2, wb = b/2, b = 5e-7 X_t,
X_t the target's largest coordinate) it re-decides in FP64.  These tests check,
with the kernel's float arithmetic emulated in numpy, that every case whose
FP32 decision differs from the FP64 one lies inside that window, and that the
error bound behind it holds on random near-threshold cases."""
import numpy as np


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _fma32(a, b, c):
    # a, b, c are floats; a*b is exact in double, one double add, one rounding to
    # float (differs from a single rounding only in double-rounding ties, which
    # the window's margin covers)
    return _f32(a * b + c)


def _fp32_dm(x, c, rc2):
    xh, ch = _f32(x), _f32(c)
    R = _f32(xh - ch)
    d2 = _fma32(R[:, 0], R[:, 0], _fma32(R[:, 1], R[:, 1], _f32(R[:, 2] * R[:, 2])))
    return _f32(d2 - _f32(rc2)), d2, xh


def _window(xh, d2):
    b = _f32(5e-7 * np.abs(xh).max(axis=1))
    wa = _f32(0.5 * b + 4e-6)
    return _f32(wa * d2 + _f32(0.5 * b))


def _cases(n, scale, seed, dmin=1e-3, rel=1e-4):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-scale, scale, (n, 3))
    d = np.exp(rng.uniform(np.log(dmin), np.log(2 * scale), n))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    c = x - d[:, None] * u
    # rcrit^2 close to the exact d^2: within rel of it
    d2 = ((x - c) ** 2).sum(axis=1)
    rc2 = d2 * (1.0 + rng.uniform(-rel, rel, n))
    return x, c, rc2


def test_decisions_outside_the_window_match_fp64():
    for scale, seed in ((1.0, 1), (40.0, 2), (1000.0, 3)):
        x, c, rc2 = _cases(200000, scale, seed)
        dm32, d2, xh = _fp32_dm(x, c, rc2)
        exact = ((x - c) ** 2).sum(axis=1) - rc2
        outside = np.abs(dm32) > _window(xh, d2)
        assert outside.sum() > 1000
        assert np.array_equal(dm32[outside] > 0, exact[outside] > 0)
        # the FP32 decision does go wrong in some of these cases: the window is needed
        x, c, rc2 = _cases(200000, scale, seed, rel=3e-7)
        dm32, d2, xh = _fp32_dm(x, c, rc2)
        exact = ((x - c) ** 2).sum(axis=1) - rc2
        wrong = (dm32 > 0) != (exact > 0)
        assert wrong.any()
        assert (np.abs(dm32[wrong]) <= _window(xh[wrong], d2[wrong])).all()


def test_error_bound_holds():
    # |dm32 - dm64| <= 2^-22 sqrt(3) X_t d + 2^-21 d2 (+ the squared R error)
    for scale, seed in ((1.0, 4), (40.0, 5), (1000.0, 6)):
        x, c, rc2 = _cases(200000, scale, seed)
        dm32, d2, xh = _fp32_dm(x, c, rc2)
        exact = ((x - c) ** 2).sum(axis=1) - rc2
        dd = np.sqrt(((x - c) ** 2).sum(axis=1))
        X = np.abs(x).max(axis=1)
        e = 2.0 ** -23 * (np.sqrt(3) * X + dd)
        bound = 2.0 ** -22 * np.sqrt(3) * X * dd + 2.0 ** -21 * dd ** 2 + e ** 2
        assert (np.abs(dm32 - exact) <= bound).all()
        # and the window contains the bound (d <= (d2 + 1) / 2)
        assert (bound <= _window(xh, d2) * (1 + 1e-6)).all()


def test_window_is_narrow():
    # the re-decision stays rare: for boxes at distances of 1 and beyond in a
    # cloud of coordinates up to 40 it fires only within 5e-5 of the threshold
    x, c, _ = _cases(100000, 40.0, 7, dmin=1.0)
    d2 = ((x - c) ** 2).sum(axis=1)
    for f in (0.99995, 1.00005):
        dm32, d2_32, xh = _fp32_dm(x, c, d2 * f)
        assert (np.abs(dm32) > _window(xh, d2_32)).all()
