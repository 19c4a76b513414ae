"""Launch shapes of the FP32C walk (threads per block x resident blocks per SM)
change only how the persistent grid schedules its 32-target chunks: every shape,
and the one ucp_autotune picks, must give the same forces, potentials and
interaction counts bit for bit, alone and on an ensemble of clouds."""
import numpy as np
import pytest

from paper_0709_3331_gb300.inputs import gaussian_cloud

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


def _walk(ctx, theta, eps):
    acc, phi = ctx.tree_force(theta, eps)
    p2p, m2p = ctx.get_counts()
    return acc, phi, p2p, m2p


@pytest.mark.parametrize("sizes,lam", [(None, None), ([3000, 517, 20000, 33], None),
                                       (None, 0.05)])
def test_every_shape_same_forces(U, sizes, lam):
    from paper_0709_3331_gb300.ucp import UCP_WALK_SHAPES
    n = 20000 if sizes is None else sum(sizes)
    c = gaussian_cloud(n, 3.0, 41)
    with U.Context(n, c.q, c.m, leaf_cap=16, precision=1, sizes=sizes,
                   kelbg_lambda=lam) as ctx:
        ctx.set_state(c.pos, c.vel, c.species)
        ref = _walk(ctx, 0.5, 0.01)
        for sh in range(1, UCP_WALK_SHAPES):
            ctx.set_walk_shape(sh)
            got = _walk(ctx, 0.5, 0.01)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), sh
        best, ms = ctx.autotune(0.5, 0.01)
        assert 0 <= best < UCP_WALK_SHAPES and ms > 0
        got = _walk(ctx, 0.5, 0.01)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        with pytest.raises(U.UcpError):
            ctx.set_walk_shape(UCP_WALK_SHAPES)


def test_autotune_keeps_trajectory(U):
    c = gaussian_cloud(4096, 1.3, 9)
    out = []
    for tune in (False, True):
        with U.Context(c.n, c.q, c.m, leaf_cap=16, precision=1) as ctx:
            ctx.set_state(c.pos, c.vel, c.species)
            ctx.step(1e-3, 5, 10, 0.5, 0.01)
            if tune:
                ctx.autotune(0.7, 0.02)   # other theta/eps: forces must be recomputed
            ctx.step(1e-3, 5, 10, 0.5, 0.01)
            out.append(ctx.get_state())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("case", ["leaf_cap_32", "fat_leaf"])
def test_staged_sources_edge_sizes(U, orc, case):
    """Leaves at the staging buffer's size (32 sources, with odd first index: 17
    pairs, read from global memory) and a depth-21 box of 100 coincident particles
    give the same bits in every shape, and match the oracle."""
    from paper_0709_3331_gb300.ucp import UCP_WALK_SHAPES
    c = gaussian_cloud(6000, 2.0, 17)
    pos = c.pos.copy()
    leaf_cap = 32
    if case == "fat_leaf":
        pos[:100] = pos[0]
        leaf_cap = 16
    with U.Context(c.n, c.q, c.m, leaf_cap=leaf_cap, precision=1) as ctx:
        ctx.set_state(pos, c.vel, c.species)
        ref = _walk(ctx, 0.5, 0.05)
        for sh in range(1, UCP_WALK_SHAPES):
            ctx.set_walk_shape(sh)
            got = _walk(ctx, 0.5, 0.05)
            for x, y in zip(got, ref):
                assert np.array_equal(x, y), sh
        if case == "fat_leaf":
            assert ctx.get_tree()["depth"].max() == 21
    E, _ = orc.Tree(pos, c.species, c.q, leaf_cap=leaf_cap).force(0.5, 0.05, nthreads=4)
    a_ref = E * (c.q[c.species] / c.m[c.species])[:, None]
    err = np.sqrt(((ref[0] - a_ref) ** 2).sum() / (a_ref ** 2).sum())
    assert err <= 1e-4
