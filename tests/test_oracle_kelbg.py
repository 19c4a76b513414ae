"""Pins of the oracle's Kelbg electron-ion interaction (Sec. 2.1 Eq. 3) and of the
physical-unit set-up of Sec. 5 (values in tests/golden/paper_sec5_setup.txt)."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sec5_setup.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = line.split("=")
            out[k.strip()] = float(v)
    return out


def _pair(orc, r, lam, eps=0.0, unlike=True):
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    sp = np.array([1, 0 if unlike else 1], dtype=np.int8)
    q = np.array([1.0, -1.0])
    with orc.kelbg(lam):
        E, phi = orc.direct(pos, sp, q, eps)
    return E, phi  # particle 0: electron (q=-1); particle 1: ion (+1) when unlike


@pytest.mark.parametrize("u", [1e-4, 1e-3, 1e-2])
def test_near_field_asymptote(orc, u):
    # Sec. 2.1: at r < lambda the potential tends to (C/lambda)(1 - r/(2 lambda))
    lam = 0.7
    E, phi = _pair(orc, u * lam, lam)
    expect = (1.0 / lam) * (1.0 - u / 2.0)   # potential at the electron due to the ion
    assert abs(phi[0] - expect) <= 0.2 * u * u / lam  # next term is +u^2/6
    # force on the electron along +x (towards the ion) tends to q^2 / (2 lambda^2)
    Fx = -1.0 * E[0][0]
    assert abs(Fx - 1.0 / (2 * lam * lam)) <= 1.0 * u / lam**2


@pytest.mark.parametrize("u", [30.0, 100.0])
def test_far_field_is_coulomb(orc, u):
    lam = 0.01
    r = u * lam
    E, phi = _pair(orc, r, lam)
    # relative departure from Coulomb: exp(-u) for the potential, (1 + u) exp(-u) for the force
    np.testing.assert_allclose(phi[0], 1.0 / r, rtol=2 * math.exp(-u) + 1e-14)
    np.testing.assert_allclose(-E[0][0], 1.0 / r**2, rtol=2 * (1 + u) * math.exp(-u) + 1e-14)


def test_force_is_minus_gradient(orc):
    lam = 0.3
    for r in (0.05, 0.3, 1.2):
        h = 1e-6
        _, pp = _pair(orc, r + h, lam)
        _, pm = _pair(orc, r - h, lam)
        E, _ = _pair(orc, r, lam)
        # potential at particle 0 as a function of the separation r: E_x(0) = +dphi/dr
        dphi = (pp[0] - pm[0]) / (2 * h)
        np.testing.assert_allclose(E[0][0], dphi, rtol=1e-7)


def test_like_pairs_and_coincident_pair(orc):
    E1, p1 = _pair(orc, 0.2, 0.5, eps=0.01, unlike=False)
    with orc.kelbg(0.5):
        pass
    pos = np.array([[0.0, 0.0, 0.0], [0.2, 0.0, 0.0]])
    E0, p0 = orc.direct(pos, np.array([1, 1], np.int8), [1.0, -1.0], 0.01)
    np.testing.assert_array_equal(E1, E0)
    # coincident electron-ion pair: finite potential q/lambda, no force
    E, phi = _pair(orc, 0.0, 0.5)
    assert np.all(E == 0.0) and phi[0] == pytest.approx(2.0)


def test_tree_uses_kelbg_in_pairs(orc):
    from paper_0709_3331_gb300.inputs import gaussian_cloud
    c = gaussian_cloud(1024, 1.0, 5)
    with orc.kelbg(0.02):
        Ed, pd = orc.direct(c.pos, c.species, c.q, 0.01)
        T = orc.Tree(c.pos, c.species, c.q, leaf_cap=8)
        Et, pt = T.force(0.0, 0.01)
        pe_d = orc.direct_pe(c.pos, c.species, c.q, 0.01)
        en = orc.energy(c.pos, c.vel, c.species, c.q, c.m, 0.0, 0.01, leaf_cap=8)
    np.testing.assert_allclose(Et, Ed, rtol=0, atol=1e-12 * np.abs(Ed).max())
    np.testing.assert_allclose(pt, pd, rtol=0, atol=1e-12 * np.abs(pd).max())
    assert en[2] == pytest.approx(pe_d, rel=1e-12)
    Ep, _ = orc.direct(c.pos, c.species, c.q, 0.01)   # back to Plummer outside the block
    assert np.abs(Ep - Ed).max() > 1e-3


def test_sec5_units(orc):
    from paper_0709_3331_gb300.inputs import sec5_units
    g = golden()
    u = sec5_units(g["density_per_cm3"], g["lambda_ei_angstrom"], g["t_e_kelvin"],
                   g["t_i_kelvin"], g["ion_mass_amu"], g["dt_fs"])
    # Wigner-Seitz radius of 4.32e9 cm^-3, computed here by hand
    a = (3.0 / (4.0 * math.pi * 4.32e9 * 1e6)) ** (1.0 / 3.0)
    assert u["length_m"] == pytest.approx(a, rel=1e-12)
    assert u["lambda"] == pytest.approx(1e-8 / a, rel=1e-12)
    # energy unit e^2 / (4 pi eps0 a) against k_B T_e
    e, eps0, kb = 1.602176634e-19, 8.8541878128e-12, 1.380649e-23
    assert u["t_e"] == pytest.approx(kb * 3.0 / (e * e / (4 * math.pi * eps0 * a)), rel=1e-9)
    assert u["m_i"] == pytest.approx(0.01 * 1.66053906660e-27 / 9.1093837015e-31, rel=1e-9)
    assert 0 < u["dt"] < 1
