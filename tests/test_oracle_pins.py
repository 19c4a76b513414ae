"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks and the mistakes it would catch.  No
expected value here comes from the CUDA path.
"""
import math

import numpy as np
import pytest

from paper_0709_3331_gb300.inputs import gaussian_cloud

Q = np.array([1.0, -1.0])
M = np.array([1000.0, 1.0])


# --------------------------------------------------------------------------
# P1  Sec. 2.1 Eq. 1-2: two charges, closed form (attractive e-i, repulsive
#     like charges; softened law; no self term at r = 0).
@pytest.mark.parametrize("sp", [(1, 0), (1, 1), (0, 0)])
@pytest.mark.parametrize("eps", [0.0, 0.01, 0.3])
def test_two_body_closed_form(orc, sp, eps):
    xe = np.array([0.3, -0.2, 0.5])
    xi = np.array([-0.1, 0.4, 0.05])
    pos = np.vstack([xe, xi])
    species = np.array(sp, dtype=np.int8)
    r = xe - xi
    s = (r @ r + eps * eps) ** -0.5
    q0, q1 = Q[species[0]], Q[species[1]]
    F0 = q0 * q1 * r * s**3          # force on particle 0
    phi0 = q1 * s
    for E, phi in (orc.direct(pos, species, Q, eps),
                   orc.Tree(pos, species, Q, leaf_cap=1).force(0.5, eps),
                   orc.Tree(pos, species, Q, leaf_cap=1).force(0.0, eps)):
        np.testing.assert_allclose(q0 * E[0], F0, rtol=1e-14, atol=0)
        np.testing.assert_allclose(Q[species[1]] * E[1], -F0, rtol=1e-14, atol=0)
        assert abs(phi[0] - phi0) <= 1e-14 * abs(phi0)
    if sp == (1, 0):   # electron pulled towards the ion
        assert np.dot(F0, xi - xe) > 0


def test_coincident_pair(orc):
    x = np.array([[0.25, 0.5, -1.0], [0.25, 0.5, -1.0]])
    species = np.array([1, 0], dtype=np.int8)
    for eps in (0.01, 0.5):
        E, phi = orc.direct(x, species, Q, eps)
        assert np.all(E == 0.0)
        np.testing.assert_allclose(phi, [Q[0] / eps, Q[1] / eps], rtol=1e-15)
        T = orc.Tree(x, species, Q, leaf_cap=1)
        t = T.export()
        assert t["depth"].max() == 21 and t["is_leaf"][-1]  # depth cap -> fat leaf
        Et, pt = T.force(0.5, eps)
        assert np.all(Et == 0.0)
        np.testing.assert_allclose(pt, phi, rtol=1e-15)


# --------------------------------------------------------------------------
# P2  Newton's third law: direct forces sum to zero; the tree's net force is
#     small and shrinks as theta -> 0.
def test_newton_third_law(orc):
    c = gaussian_cloud(512, 1.0, seed=11)
    E, _ = orc.direct(c.pos, c.species, c.q, 0.01)
    F = E * c.q[c.species][:, None]
    scale = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() <= 1e-13 * scale
    prev = None
    T = orc.Tree(c.pos, c.species, c.q, leaf_cap=4)
    for theta in (0.8, 0.4, 0.1):
        Et, _ = T.force(theta, 0.01)
        net = np.abs((Et * c.q[c.species][:, None]).sum(0)).max() / scale
        if prev is not None:
            assert net < prev
        prev = net
    assert prev < 1e-6


# --------------------------------------------------------------------------
# P3  theta -> 0 (never accept) and leaf_cap >= N both reduce the tree to the
#     direct sum; small theta converges to it.
@pytest.mark.parametrize("leaf_cap", [1, 8, 64])
def test_tree_reduces_to_direct(orc, leaf_cap):
    c = gaussian_cloud(1024, 1.0, seed=3)
    E, phi = orc.direct(c.pos, c.species, c.q, 0.01)
    T = orc.Tree(c.pos, c.species, c.q, leaf_cap=leaf_cap)
    Et, pt, npp, nmp = T.force(0.0, 0.01, counts=True)
    np.testing.assert_allclose(Et, E, rtol=0, atol=1e-12 * np.abs(E).max())
    np.testing.assert_allclose(pt, phi, rtol=0, atol=1e-12 * np.abs(phi).max())
    assert np.all(npp == c.n - 1) and np.all(nmp == 0)
    Eb, _ = orc.Tree(c.pos, c.species, c.q, leaf_cap=c.n).force(0.7, 0.01)
    np.testing.assert_allclose(Eb, E, rtol=0, atol=1e-12 * np.abs(E).max())
    errs = []
    for theta in (0.9, 0.6, 0.3, 0.15):
        Et, _ = T.force(theta, 0.01)
        errs.append(math.sqrt(((Et - E) ** 2).sum() / (E**2).sum()))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5


# --------------------------------------------------------------------------
# P4  The expansion of a box about its centroid through quadrupole order:
#     the absolute error against the exact sum falls as d^-5 (octupole
#     remainder) for charged and for neutral boxes, softened or not.  A dropped
#     or wrong term leaves a d^-2, d^-3 or d^-4 error and fails the slope.
def _slope(orc, pos, species, eps, mask=7):
    rng = np.random.default_rng(7)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ds = np.array([8.0, 16.0, 32.0, 64.0])
    errs = []
    for d in ds:
        xt = d * u
        E, phi = orc.cluster_multipole(pos, species, Q, eps, xt, term_mask=mask)
        allp = np.vstack([pos, xt])
        sp = np.concatenate([species, [0]]).astype(np.int8)
        Ed, pd = orc.direct(allp, sp, Q, eps, targets=[pos.shape[0]])
        errs.append(np.linalg.norm(E - Ed[0]))
    return np.polyfit(np.log(ds), np.log(errs), 1)[0]


@pytest.mark.parametrize("neutral", [False, True])
@pytest.mark.parametrize("eps", [0.0, 0.01, 0.5])
def test_multipole_convergence_order(orc, neutral, eps):
    rng = np.random.default_rng(5)
    pos = rng.uniform(-0.5, 0.5, size=(6, 3))
    species = np.array([0, 1, 0, 1, 0, 1] if neutral else [0, 0, 1, 0, 0, 1], dtype=np.int8)
    assert abs(_slope(orc, pos, species, eps) + 5.0) < 0.3


def test_multipole_pin_catches_dropped_terms(orc):
    """Plants the mistakes in the oracle (term mask) and shows the pin fails."""
    rng = np.random.default_rng(5)
    pos = rng.uniform(-0.5, 0.5, size=(6, 3))
    neutral = np.array([0, 1, 0, 1, 0, 1], dtype=np.int8)
    charged = np.array([0, 0, 1, 0, 0, 1], dtype=np.int8)
    assert abs(_slope(orc, pos, neutral, 0.01, mask=0b101) + 3.0) < 0.3   # no dipole
    assert abs(_slope(orc, pos, neutral, 0.01, mask=0b011) + 4.0) < 0.3   # no quadrupole
    assert abs(_slope(orc, pos, charged, 0.01, mask=0b110) + 2.0) < 0.3   # no monopole


def test_multipole_potential_exact_for_single_charge(orc):
    pos = np.array([[0.1, 0.2, -0.3]])
    for sp in (0, 1):
        species = np.array([sp], dtype=np.int8)
        xt = np.array([2.0, -1.0, 0.5])
        E, phi = orc.cluster_multipole(pos, species, Q, 0.01, xt)
        Ed, pd = orc.direct(np.vstack([pos, xt]), np.array([sp, 0], np.int8), Q, 0.01,
                            targets=[1])
        np.testing.assert_allclose(E, Ed[0], rtol=1e-14)
        np.testing.assert_allclose(phi, pd[0], rtol=1e-14)


# --------------------------------------------------------------------------
# P5  Brute force on tiny inputs: the node set, the leaf rule and every
#     target's interaction list rebuilt in plain Python from the definitions
#     (boxes = particle groups sharing the top d bits of their cell
#     coordinates; Eq. 5 decides; a box is visited only if all its ancestors
#     were opened).  Counts and field must agree with the oracle.
def _brute_tree(kc, leaf_cap):
    n = kc.shape[0]
    nodes = {}

    def rec(d, members):
        key = (d, tuple(int(v) >> (21 - d) for v in kc[members[0]]))
        nodes[key] = list(members)
        if len(members) <= leaf_cap or d == 21:
            return
        groups = {}
        for j in members:
            cell = tuple(int(v) >> (21 - d - 1) for v in kc[j])
            groups.setdefault(cell, []).append(j)
        for cell in groups:
            rec(d + 1, groups[cell])

    rec(0, list(range(n)))
    return nodes


@pytest.mark.parametrize("n,leaf_cap,theta", [(12, 1, 0.5), (40, 3, 0.4), (64, 2, 0.9),
                                              (64, 1, 0.0)])
def test_brute_force_tiny(orc, n, leaf_cap, theta):
    c = gaussian_cloud(n, 1.0, seed=100 + n)
    cube = orc.root_cube(c.pos)
    kc = orc.int_coords(c.pos, cube)
    nodes = _brute_tree(kc, leaf_cap)
    T = orc.Tree(c.pos, c.species, c.q, leaf_cap=leaf_cap)
    t = T.export()
    assert T.nnodes == len(nodes)
    got = {(int(t["depth"][i]), tuple(int(v) for v in t["cell"][i])):
           sorted(t["slot"][t["begin"][i]:t["end"][i]].tolist()) for i in range(T.nnodes)}
    assert got == {k: sorted(v) for k, v in nodes.items()}
    L = cube[3]
    eps = 0.01
    E_exp = np.zeros((n, 3))
    np_exp = np.zeros(n, dtype=int)
    nm_exp = np.zeros(n, dtype=int)
    for tt in range(n):
        x = c.pos[tt]

        def visit(key):
            d, cell = key
            mem = nodes[key]
            qs = c.q[c.species[mem]]
            w = np.abs(qs)
            cen = (w[:, None] * c.pos[mem]).sum(0) / w.sum()
            side = L / 2**d
            centre = cube[:3] - L / 2 + (np.array(cell) + 0.5) * side
            delta = np.linalg.norm(cen - centre)
            if theta > 0 and side / theta + delta < np.linalg.norm(x - cen):
                nm_exp[tt] += 1
                y = c.pos[mem] - cen
                Dv = (qs[:, None] * y).sum(0)
                Qm = np.einsum("j,ja,jb->ab", qs, y, y)
                R = x - cen
                g = 1.0 / math.sqrt(R @ R + eps * eps)
                E_exp[tt] += (qs.sum() * R * g**3 - Dv * g**3 + 3 * (Dv @ R) * R * g**5
                              - 3 * (Qm @ R) * g**5 + 7.5 * (R @ Qm @ R) * R * g**7
                              - 1.5 * np.trace(Qm) * R * g**5)
                return
            children = [k for k in nodes if k[0] == d + 1
                        and all((a >> 1) == b for a, b in zip(k[1], cell))]
            if not children:
                for j in mem:
                    if j == tt:
                        continue
                    r = x - c.pos[j]
                    E_exp[tt] += c.q[c.species[j]] * r / (r @ r + eps * eps) ** 1.5
                    np_exp[tt] += 1
                return
            for k in children:
                visit(k)

        visit((0, (0, 0, 0)))
    E, _, npp, nmp = T.force(theta, eps, counts=True)
    np.testing.assert_array_equal(npp, np_exp)
    np.testing.assert_array_equal(nmp, nm_exp)
    np.testing.assert_allclose(E, E_exp, rtol=1e-10, atol=1e-12 * np.abs(E_exp).max())


# --------------------------------------------------------------------------
# P6  Smooth-field closed form: a Gaussian cloud of N_s like charges has the
#     radial field (N_s q / r^2)[erf(r/(sqrt2 s)) - sqrt(2/pi)(r/s) exp(-r^2/2s^2)];
#     zero-charge probes read the tree field up to shot noise.
def test_gaussian_cloud_field(orc):
    rng = np.random.default_rng(21)
    ns, sig = 20000, 1.0
    src = rng.normal(0, sig, size=(ns, 3))
    radii = np.array([1.0, 1.5, 2.0, 3.0, 4.0])
    dirs = rng.normal(size=(len(radii), 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    probes = radii[:, None] * dirs
    pos = np.vstack([src, probes])
    species = np.concatenate([np.zeros(ns), np.ones(len(radii))]).astype(np.int8)
    q = np.array([1.0, 0.0])
    T = orc.Tree(pos, species, q, leaf_cap=8)
    E, _ = T.force(0.5, 0.01, targets=np.arange(ns, ns + len(radii)))
    Er = (E * dirs).sum(1)
    r = radii
    closed = ns / r**2 * (np.vectorize(math.erf)(r / (math.sqrt(2) * sig))
                          - math.sqrt(2 / math.pi) * (r / sig) * np.exp(-r**2 / (2 * sig**2)))
    np.testing.assert_allclose(Er, closed, rtol=0.03)


# --------------------------------------------------------------------------
# P7  Invariances: flipping every charge negates the field exactly (forces
#     unchanged); scaling positions and eps by 2 scales E by 1/4 and phi by 1/2
#     exactly (every term of the expansion must have the right power of g);
#     relabelling particles does not change any particle's field.
def test_charge_conjugation_exact(orc):
    c = gaussian_cloud(2048, 1.0, seed=1)
    T1 = orc.Tree(c.pos, c.species, c.q, leaf_cap=8)
    T2 = orc.Tree(c.pos, c.species, -c.q, leaf_cap=8)
    E1, p1 = T1.force(0.5, 0.01)
    E2, p2 = T2.force(0.5, 0.01)
    assert np.array_equal(E1, -E2) and np.array_equal(p1, -p2)


def test_power_of_two_scaling_exact(orc):
    c = gaussian_cloud(2048, 1.0, seed=1)
    E1, p1 = orc.Tree(c.pos, c.species, c.q, leaf_cap=8).force(0.5, 0.01)
    E2, p2 = orc.Tree(c.pos * 2.0, c.species, c.q, leaf_cap=8).force(0.5, 0.02)
    assert np.array_equal(E2 * 4.0, E1) and np.array_equal(p2 * 2.0, p1)


def test_relabel_invariance(orc):
    c = gaussian_cloud(1024, 1.0, seed=4)
    perm = np.random.default_rng(0).permutation(c.n)
    E1, p1 = orc.Tree(c.pos, c.species, c.q, leaf_cap=4).force(0.5, 0.01)
    E2, p2 = orc.Tree(c.pos[perm], c.species[perm], c.q, leaf_cap=4).force(0.5, 0.01)
    np.testing.assert_allclose(E2, E1[perm], rtol=0, atol=1e-12 * np.abs(E1).max())


# --------------------------------------------------------------------------
# Keys and sort (Sec. 3 boxes as integer coordinates).
def test_interleave_known_values(orc):
    assert orc.interleave(1, 0, 0) == 1
    assert orc.interleave(0, 1, 0) == 2
    assert orc.interleave(0, 0, 1) == 4
    assert orc.interleave(1, 1, 1) == 7
    assert orc.interleave(2, 0, 0) == 8
    assert orc.interleave(0, 0, 2) == 32
    full = (1 << 21) - 1
    assert orc.interleave(full, full, full) == (1 << 63) - 1
    assert orc.interleave(full, 0, 0) == int("001" * 21, 2)


def test_root_cube_and_coords(orc):
    c = gaussian_cloud(4096, 2.0, seed=9)
    cube = orc.root_cube(c.pos)
    lo, hi = c.pos.min(0), c.pos.max(0)
    np.testing.assert_array_equal(cube[:3], (lo + hi) / 2)
    assert cube[3] == (hi - lo).max() * (1 + 2.0**-20)
    k = orc.int_coords(c.pos, cube)
    assert k.max() < 2**21
    # along the widest axis the extreme particles sit in the first and last cells;
    # every axis is centred, so its extreme cells are symmetric
    w = int(np.argmax(hi - lo))
    assert k[np.argmin(c.pos[:, w]), w] == 0
    assert k[np.argmax(c.pos[:, w]), w] == 2**21 - 1
    for a in range(3):
        kl, kh = int(k[np.argmin(c.pos[:, a]), a]), int(k[np.argmax(c.pos[:, a]), a])
        assert abs((kl + kh) - (2**21 - 1)) <= 2
    one = orc.root_cube(np.array([[1.0, 2.0, 3.0]]))
    np.testing.assert_array_equal(one, [1.0, 2.0, 3.0, 1.0])


def test_sort_order_stable(orc):
    keys = np.array([5, 3, 5, 1, 3, 3, 0], dtype=np.uint64)
    np.testing.assert_array_equal(orc.sort_order(keys), [6, 3, 1, 4, 5, 0, 2])


@pytest.mark.parametrize("leaf_cap", [1, 4, 16])
def test_tree_invariants(orc, leaf_cap):
    c = gaussian_cloud(2048, 1.0, seed=1)
    T = orc.Tree(c.pos, c.species, c.q, leaf_cap=leaf_cap)
    t = T.export()
    nn = T.nnodes
    k = orc.keys(c.pos, T.cube())
    order = orc.sort_order(k)
    # every box holds the same particles as the matching range of the
    # (key, index)-sorted order: the subdivision and the key sort agree
    assert set(t["slot"].tolist()) == set(range(c.n))
    assert np.all(k[order][1:] >= k[order][:-1])
    for i in range(nn):
        b, e = t["begin"][i], t["end"][i]
        assert set(t["slot"][b:e].tolist()) == set(order[b:e].tolist())
    for i in range(nn):
        b, e, nx, d = t["begin"][i], t["end"][i], t["next"][i], t["depth"][i]
        assert e > b
        if t["is_leaf"][i]:
            assert e - b <= leaf_cap or d == 21
            assert nx == i + 1
        else:
            assert e - b > leaf_cap
            ch = i + 1
            covered = b
            while ch < nx:
                assert t["depth"][ch] == d + 1 and t["begin"][ch] == covered
                covered = t["end"][ch]
                ch = t["next"][ch]
            assert covered == e and ch == nx
    # moments pinned by their definitions
    for i in np.random.default_rng(0).choice(nn, 50):
        mem = t["slot"][t["begin"][i]:t["end"][i]]
        qs = c.q[c.species[mem]]
        assert t["M"][i] == pytest.approx(qs.sum(), abs=1e-12)
        cen = c.pos[mem].mean(0)
        np.testing.assert_allclose(t["c"][i], cen, rtol=0, atol=1e-13)
        np.testing.assert_allclose(t["D"][i], (qs[:, None] * (c.pos[mem] - cen)).sum(0),
                                   atol=1e-12)
        y = c.pos[mem] - t["c"][i]
        Qm = np.einsum("j,ja,jb->ab", qs, y, y)
        np.testing.assert_allclose(t["Q"][i], Qm[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]],
                                   atol=1e-12)
        side = T.cube()[3] / 2.0 ** t["depth"][i]
        assert t["side"][i] == side
        assert np.all(np.abs(t["centre"][i] - cen) <= side / 2 + 1e-12)


# --------------------------------------------------------------------------
# P8  The split-step push: k = 1 is plain velocity Verlet; momentum is kept
#     to roundoff with direct forces at k = 1; the energy error of a softened
#     two-body orbit is second order in dt; forward-then-backward returns.
def test_k1_is_velocity_verlet(orc):
    c = gaussian_cloud(64, 1.0, seed=2)
    dt, steps = 1e-3, 5
    p, v, a = orc.run(c.pos, c.vel, c.species, c.q, c.m, dt, 1, steps, 0.5, 0.01,
                      direct_sum=True)
    x = c.pos.copy()
    u = c.vel.copy()
    acc = orc.accel(x, c.species, c.q, c.m, 0.5, 0.01, direct_sum=True)
    for _ in range(steps):
        u = u + 0.5 * dt * acc
        x = x + dt * u
        acc = orc.accel(x, c.species, c.q, c.m, 0.5, 0.01, direct_sum=True)
        u = u + 0.5 * dt * acc
    np.testing.assert_allclose(p, x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(v, u, rtol=1e-12, atol=1e-14)


def test_momentum_conserved_k1_direct(orc):
    c = gaussian_cloud(128, 1.0, seed=3)
    P0 = (c.m[c.species][:, None] * c.vel).sum(0)
    _, v, _ = orc.run(c.pos, c.vel, c.species, c.q, c.m, 1e-3, 1, 20, 0.5, 0.01, direct_sum=True)
    P1 = (c.m[c.species][:, None] * v).sum(0)
    scale = np.abs(c.m[c.species][:, None] * c.vel).sum()
    assert np.abs(P1 - P0).max() < 1e-13 * scale


def test_energy_error_second_order(orc):
    # bound e-i pair on a softened orbit; ion heavy
    pos = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    species = np.array([1, 0], dtype=np.int8)
    vel = np.array([[0.0, 0.9, 0.0], [0.0, -0.0009, 0.0]])
    errs = []
    for dt in (0.02, 0.01, 0.005):
        steps = int(round(2.0 / dt))
        e0 = orc.energy(pos, vel, species, Q, M, 0.5, 0.05, direct_sum=True)[3]
        emax = 0.0
        p, v, a = pos, vel, None
        for _ in range(steps // 10):
            p, v, a = orc.run(p, v, species, Q, M, dt, 1, 10, 0.5, 0.05, direct_sum=True, acc=a)
            emax = max(emax, abs(orc.energy(p, v, species, Q, M, 0.5, 0.05, direct_sum=True)[3]
                                 - e0))
        errs.append(emax)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs


@pytest.mark.parametrize("k", [1, 10])
@pytest.mark.parametrize("direct_sum", [True, False])
def test_time_reversible(orc, k, direct_sum):
    c = gaussian_cloud(256, 1.0, seed=8)
    p, v, a = orc.run(c.pos, c.vel, c.species, c.q, c.m, 1e-3, k, 1, 0.5, 0.01, leaf_cap=4,
                      direct_sum=direct_sum)
    p2, v2, _ = orc.run(p, -v, c.species, c.q, c.m, 1e-3, k, 1, 0.5, 0.01, leaf_cap=4,
                        direct_sum=direct_sum, acc=a)
    np.testing.assert_allclose(p2, c.pos, rtol=0, atol=1e-12)
    np.testing.assert_allclose(-v2, c.vel, rtol=0, atol=1e-9)


# --------------------------------------------------------------------------
# P9  Sec. 5.2: the tree's total energy tracks the all pair-wise run closely
#     for theta <= 0.6 over a short run; the energy of the direct run is kept.
def test_tree_energy_tracks_pairwise(orc):
    c = gaussian_cloud(512, 1.0, seed=6)
    eps, dt, k = 0.05, 1e-3, 10
    pd, vd, _ = orc.run(c.pos, c.vel, c.species, c.q, c.m, dt, k, 2, 0.5, eps, direct_sum=True)
    pt, vt, _ = orc.run(c.pos, c.vel, c.species, c.q, c.m, dt, k, 2, 0.5, eps, leaf_cap=4)
    e0 = orc.energy(c.pos, c.vel, c.species, c.q, c.m, 0.5, eps, direct_sum=True)
    ed = orc.energy(pd, vd, c.species, c.q, c.m, 0.5, eps, direct_sum=True)
    et = orc.energy(pt, vt, c.species, c.q, c.m, 0.5, eps, direct_sum=True)
    scale = e0[0] + e0[1] + abs(e0[2])
    assert abs(ed[3] - e0[3]) / scale < 1e-4
    assert abs(et[3] - ed[3]) / scale < 1e-4
    # tree potential energy converges to the pair sum
    errs = [abs(orc.energy(c.pos, c.vel, c.species, c.q, c.m, th, eps, leaf_cap=4)[2] - e0[2])
            / abs(e0[2]) for th in (0.6, 0.3, 0.1, 0.0)]
    assert errs[0] < 1e-2 and errs[1] < 1e-3 and errs[2] < 1e-5 and errs[3] < 1e-11
