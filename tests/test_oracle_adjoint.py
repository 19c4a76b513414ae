"""Pins of the oracle's adjoint (the reverse-mode derivative of the tree force and
of the split-step push), against finite differences of the oracle's own forward
computation and against translation invariance."""
import numpy as np
import pytest

from paper_0709_3331_gb300.inputs import gaussian_cloud


def _accel(orc, x, c, theta, eps, leaf_cap, direct):
    if direct:
        E, _ = orc.direct(x, c.species, c.q, eps)
        return E * (c.q[c.species] / c.m[c.species])[:, None], None
    T = orc.Tree(x, c.species, c.q, leaf_cap=leaf_cap)
    E, _, npp, nmp = T.force(theta, eps, counts=True)
    return E * (c.q[c.species] / c.m[c.species])[:, None], (npp, nmp, T.export()["begin"].shape)


@pytest.mark.parametrize("direct,theta,leaf_cap", [(True, 0.5, 1), (False, 0.5, 4),
                                                   (False, 0.8, 8), (False, 0.0, 4)])
def test_force_adjoint_directional_derivative(orc, direct, theta, leaf_cap):
    c = gaussian_cloud(256, 1.0, 3)
    eps = 0.05
    rng = np.random.default_rng(1)
    lam = rng.normal(size=(c.n, 3))
    mu = orc.force_adjoint(c.pos, c.species, c.q, c.m, lam, theta, eps, leaf_cap=leaf_cap,
                           direct_sum=direct)
    checked = 0
    for trial in range(6):
        d = rng.normal(size=(c.n, 3))
        h = 1e-6
        ap, kp = _accel(orc, c.pos + h * d, c, theta, eps, leaf_cap, direct)
        am, km = _accel(orc, c.pos - h * d, c, theta, eps, leaf_cap, direct)
        if not direct:   # the frozen-tree derivative only where the tree did not change
            _, k0 = _accel(orc, c.pos, c, theta, eps, leaf_cap, direct)
            if not all(np.array_equal(a, b) for a, b in zip(kp[:2] + km[:2], k0[:2] + k0[:2])):
                continue
        fd = (lam * (ap - am)).sum() / (2 * h)
        ad = (mu * d).sum()
        assert abs(fd - ad) <= 1e-6 * (abs(fd) + np.abs(lam).sum() * 1e-3), (fd, ad)
        checked += 1
    assert checked >= 3


@pytest.mark.parametrize("direct,theta", [(True, 0.5), (False, 0.6), (False, 0.3)])
def test_force_adjoint_translation_invariance(orc, direct, theta):
    # a(x) does not change when every particle moves together, so sum_s mu_s = 0;
    # a missing centre term of the expansion's source side breaks this
    c = gaussian_cloud(512, 1.0, 8)
    lam = np.random.default_rng(2).normal(size=(c.n, 3))
    mu = orc.force_adjoint(c.pos, c.species, c.q, c.m, lam, theta, 0.02, leaf_cap=4,
                           direct_sum=direct)
    assert np.abs(mu.sum(0)).max() <= 1e-10 * np.abs(mu).sum()


@pytest.mark.parametrize("direct,k", [(True, 1), (True, 4), (False, 4)])
def test_run_adjoint_vs_finite_differences(orc, direct, k):
    c = gaussian_cloud(128, 1.0, 12)
    dt, nb, theta, eps, lc = 2e-3, 2, 0.5, 0.05, 4
    L, gx, gv = orc.run_adjoint_ke_e(c.pos, c.vel, c.species, c.q, c.m, dt, k, nb, theta, eps,
                                     leaf_cap=lc, direct_sum=direct)

    def loss(p, v):
        _, vv, _ = orc.run(p, v, c.species, c.q, c.m, dt, k, nb, theta, eps, leaf_cap=lc,
                           direct_sum=direct)
        e = c.species == 1
        return 0.5 * c.m[1] * (vv[e] ** 2).sum()

    assert L == pytest.approx(loss(c.pos, c.vel), rel=1e-14)
    rng = np.random.default_rng(5)
    h = 1e-6
    good = 0
    coords = [(rng.integers(c.n), rng.integers(3)) for _ in range(16)]
    for i, a in coords:
        for which, g in (("x", gx), ("v", gv)):
            p, v = c.pos.copy(), c.vel.copy()
            arr = p if which == "x" else v
            arr[i, a] += h
            lp = loss(p, v)
            arr[i, a] -= 2 * h
            lm = loss(p, v)
            fd = (lp - lm) / (2 * h)
            if abs(fd - g[i, a]) <= 1e-5 * (abs(fd) + 1e-3 * abs(L)):
                good += 1
    # the tree may reorganise under a perturbation (a box boundary or an opening
    # decision crossed): allow a few such coordinates there, none for the direct sum
    assert good >= (32 if direct else 29), good
