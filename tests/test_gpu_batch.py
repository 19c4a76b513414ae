"""Ensembles of independent clouds in one context (ucp_create_batch): every cloud
must give what it gives alone -- bit for bit against a solo GPU context (same
tree, same warps, same order of sums) and within the parity tolerances against
the FP64 oracle run on that cloud alone."""
import math

import numpy as np
import pytest

from paper_0709_3331_gb300.inputs import batched_sizes, gaussian_cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0709_3331_gb300 import build as b
    b.build()
    import paper_0709_3331_gb300 as P
    return P


def _ensemble(sizes, seed0=4000):
    clouds = [gaussian_cloud(n, (n / 2048.0) ** (1.0 / 3.0), seed0 + i) for i, n in enumerate(sizes)]
    pos = np.concatenate([c.pos for c in clouds])
    vel = np.concatenate([c.vel for c in clouds])
    sp = np.concatenate([c.species for c in clouds])
    return clouds, pos, vel, sp


def rel_rms(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


SIZES = [2048, 6002, 512, 4096, 1000, 34]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_force_equals_solo(U, prec):
    clouds, pos, vel, sp = _ensemble(SIZES)
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=16, precision=prec, sizes=SIZES) as ctx:
        ctx.set_state(pos, vel, sp)
        acc, phi = ctx.tree_force(0.5, 0.01)
        cubes = ctx.get_cubes()
        p2p, m2p = ctx.get_counts()
    off = 0
    for i, c in enumerate(clouds):
        with U.Context(c.n, c.q, c.m, leaf_cap=16, precision=prec) as solo:
            solo.set_state(c.pos, c.vel, c.species)
            a1, p1 = solo.tree_force(0.5, 0.01)
            cube1 = solo.get_cube()
            q1, m1 = solo.get_counts()
        sl = slice(off, off + c.n)
        assert np.array_equal(acc[sl], a1) and np.array_equal(phi[sl], p1)
        assert np.array_equal(cubes[i], cube1)
        assert np.array_equal(p2p[sl], q1) and np.array_equal(m2p[sl], m1)
        off += c.n


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-4)])
def test_batch_force_vs_oracle(U, orc, prec, tol):
    clouds, pos, vel, sp = _ensemble(SIZES, seed0=77)
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=16, precision=prec, sizes=SIZES) as ctx:
        ctx.set_state(pos, vel, sp)
        acc, phi = ctx.tree_force(0.5, 0.01)
    off = 0
    for c in clouds:
        E, ph = orc.Tree(c.pos, c.species, c.q, leaf_cap=16).force(0.5, 0.01, nthreads=4)
        a_ref = E * (c.q[c.species] / c.m[c.species])[:, None]
        sl = slice(off, off + c.n)
        assert rel_rms(acc[sl], a_ref) <= tol
        assert rel_rms(phi[sl], ph) <= tol
        off += c.n


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_step_equals_solo(U, prec):
    sizes = [1024, 3000, 256]
    clouds, pos, vel, sp = _ensemble(sizes, seed0=11)
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=8, precision=prec, sizes=sizes) as ctx:
        ctx.set_state(pos, vel, sp)
        ctx.step(1e-3, 5, 10, 0.5, 0.01)
        p, v = ctx.get_state()
        en = ctx.energy_clouds(0.5, 0.01)
        tot = ctx.energy(0.5, 0.01)
    off = 0
    for i, c in enumerate(clouds):
        with U.Context(c.n, c.q, c.m, leaf_cap=8, precision=prec) as solo:
            solo.set_state(c.pos, c.vel, c.species)
            solo.step(1e-3, 5, 10, 0.5, 0.01)
            p1, v1 = solo.get_state()
            e1 = solo.energy(0.5, 0.01)
        sl = slice(off, off + c.n)
        assert np.array_equal(p[sl], p1) and np.array_equal(v[sl], v1)
        np.testing.assert_allclose(en[i, :4], e1[:4], rtol=1e-12)
        assert en[i, 5] == 10
        off += c.n
    np.testing.assert_allclose(tot[:4], en[:, :4].sum(0), rtol=1e-12)


def test_batch_standard_size_mix_vs_oracle(U, orc):
    # the size distribution of the 64-cloud ensemble (log-uniform 4096..65536),
    # first 6 clouds, FP32C with FP64 state, one tree force each
    ns, _ = batched_sizes()
    sizes = ns[:6]
    clouds, pos, vel, sp = _ensemble(sizes)
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=16, precision=1, sizes=sizes) as ctx:
        ctx.set_state(pos, vel, sp)
        acc, _ = ctx.tree_force(0.5, 0.01)
    off = 0
    rng = np.random.default_rng(0)
    for c in clouds:
        tl = np.sort(rng.choice(c.n, 256, replace=False))
        E, _ = orc.Tree(c.pos, c.species, c.q, leaf_cap=16).force(0.5, 0.01, targets=tl,
                                                                   nthreads=4)
        a_ref = E * (c.q[c.species[tl]] / c.m[c.species[tl]])[:, None]
        assert rel_rms(acc[off + tl], a_ref) <= 1e-4
        off += c.n


def test_batch_rejects_bad_sizes(U):
    with pytest.raises(U.UcpError):
        U.Context(10, sizes=[5, 0, 5])
    with pytest.raises(U.UcpError):
        U.Context(11, sizes=[5, 5])
    with pytest.raises(U.UcpError):
        U.Context(300, sizes=[1] * 300)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_kelbg_equals_solo(U, prec):
    """The Kelbg electron-ion law in an ensemble: every cloud as alone, and the
    same when the blocks replay captured graphs."""
    sizes = [2000, 700, 3000]
    clouds, pos, vel, sp = _ensemble(sizes, seed0=31)
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=16, precision=prec, sizes=sizes,
                   kelbg_lambda=0.05) as ctx:
        ctx.set_graphs(True)
        ctx.set_state(pos, vel, sp)
        acc, phi = ctx.tree_force(0.5, 0.01)
        ctx.step(1e-3, 5, 10, 0.5, 0.01)
        p, v = ctx.get_state()
    off = 0
    for c in clouds:
        with U.Context(c.n, c.q, c.m, leaf_cap=16, precision=prec, kelbg_lambda=0.05) as solo:
            solo.set_state(c.pos, c.vel, c.species)
            a1, p1 = solo.tree_force(0.5, 0.01)
            solo.step(1e-3, 5, 10, 0.5, 0.01)
            q1, w1 = solo.get_state()
        sl = slice(off, off + c.n)
        assert np.array_equal(acc[sl], a1) and np.array_equal(phi[sl], p1)
        assert np.array_equal(p[sl], q1) and np.array_equal(v[sl], w1)
        off += c.n


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_accel_vjp_equals_solo(U, prec, tol):
    """The frozen-tree adjoint walk on an ensemble gives each cloud's own
    vector-Jacobian product (the source-side atomic sums may differ in the last
    bits, so within rounding)."""
    sizes = [1500, 400, 2600]
    clouds, pos, vel, sp = _ensemble(sizes, seed0=41)
    lam = np.random.default_rng(2).standard_normal((len(sp), 3))
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=16, precision=prec, sizes=sizes) as ctx:
        ctx.set_state(pos, vel, sp)
        mu = ctx.accel_vjp(0.5, 0.01, lam)
    off = 0
    for c in clouds:
        sl = slice(off, off + c.n)
        with U.Context(c.n, c.q, c.m, leaf_cap=16, precision=prec) as solo:
            solo.set_state(c.pos, c.vel, c.species)
            m1 = solo.accel_vjp(0.5, 0.01, lam[sl].copy())
        assert rel_rms(mu[sl], m1) <= tol
        off += c.n


def test_batch_gradient_equals_solo(U):
    """ucp_grad_ke_electrons on an ensemble: the loss is the sum of the clouds'
    losses and each cloud's gradient is its own (within the atomic-sum rounding)."""
    sizes = [1200, 900]
    clouds, pos, vel, sp = _ensemble(sizes, seed0=51)
    c0 = clouds[0]
    with U.Context(len(sp), c0.q, c0.m, leaf_cap=16, precision=1, sizes=sizes) as ctx:
        ctx.set_state(pos, vel, sp)
        L, gx, gv = ctx.grad_ke_electrons(1e-3, 2, 6, 0.5, 0.01, 2)
    off, Ls = 0, 0.0
    for c in clouds:
        sl = slice(off, off + c.n)
        with U.Context(c.n, c.q, c.m, leaf_cap=16, precision=1) as solo:
            solo.set_state(c.pos, c.vel, c.species)
            L1, gx1, gv1 = solo.grad_ke_electrons(1e-3, 2, 6, 0.5, 0.01, 2)
        Ls += L1
        assert rel_rms(gx[sl], gx1) <= 1e-6 and rel_rms(gv[sl], gv1) <= 1e-6
        off += c.n
    assert L == pytest.approx(Ls, rel=1e-12)
