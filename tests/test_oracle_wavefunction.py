"""Pins for drift (Eq. 2), kinetic energy and local energy (Eq. 4).

* drift = finite-difference gradient of log|Psi| (Psi from the oracle itself,
  differentiated numerically -- independent of the D^-1 identity);
* sum of Laplacians = finite-difference Laplacian of Psi (not log|Psi|);
* swapping two same-spin electrons flips the sign only;
* one electron in one Gaussian 1s (or 2p) primitive: E_L in closed form;
* Coulomb sums against brute-force Python loops.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from synth import make_walkers, tiny_system
from tests.helpers import one_atom_system


@pytest.fixture(scope="module")
def water():
    s = tiny_system("h2o_like")
    return s, Oracle(s)


def test_drift_is_gradient_of_log_psi(water):
    s, o = water
    R = make_walkers(s, 2)
    h = 1e-5
    for w in range(2):
        base = o.eval(R[w:w + 1])
        for e in range(s.n_elec):
            for l in range(3):
                Rp, Rm = R[w:w + 1].copy(), R[w:w + 1].copy()
                Rp[0, e, l] += h
                Rm[0, e, l] -= h
                fd = (o.eval(Rp)["logpsi"][0] - o.eval(Rm)["logpsi"][0]) / (2 * h)
                assert abs(fd - base["drift"][0, e, l]) < 1e-6 * (1 + abs(fd))


def test_kinetic_is_laplacian_of_psi(water):
    s, o = water
    R = make_walkers(s, 1)
    h = 1e-3
    base = o.eval(R)
    lp0 = base["logpsi"][0]
    tot = 0.0
    for e in range(s.n_elec):
        for l in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[0, e, l] += h
            Rm[0, e, l] -= h
            op, om = o.eval(Rp), o.eval(Rm)
            psi_p = op["sign"][0] * math.exp(op["logpsi"][0] - lp0)
            psi_m = om["sign"][0] * math.exp(om["logpsi"][0] - lp0)
            psi_0 = base["sign"][0]
            tot += (psi_p - 2 * psi_0 + psi_m) / (h * h) / psi_0
    T = base["e_parts"][0, 0]
    assert abs(-0.5 * tot - T) < 1e-4 * (1 + abs(T))


def test_same_spin_swap_flips_sign(water):
    s, o = water
    R = make_walkers(s, 3)
    base = o.eval(R)
    for (i, j) in ((0, 1), (s.n_up, s.n_up + 2)):
        Rs = R.copy()
        Rs[:, [i, j]] = Rs[:, [j, i]]
        sw = o.eval(Rs)
        np.testing.assert_array_equal(sw["sign"], -base["sign"])
        np.testing.assert_allclose(sw["logpsi"], base["logpsi"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(sw["e_loc"], base["e_loc"], rtol=1e-12)
        dr = base["drift"].copy()
        dr[:, [i, j]] = dr[:, [j, i]]
        np.testing.assert_allclose(sw["drift"], dr, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("Z", [1.0, 3.0])
def test_one_electron_gaussian_1s(Z):
    gam = 0.9
    s = one_atom_system(Z, [(0, [gam], [1.0])], n_up=1, n_dn=0, A_up=[[1.0]])
    o = Oracle(s)
    rng = np.random.default_rng(7)
    R = rng.normal(size=(5, 1, 3)) * 0.8
    out = o.eval(R)
    r2 = (R[:, 0] ** 2).sum(1)
    r = np.sqrt(r2)
    # T = -1/2 lap(e^{-g r^2}) / e^{-g r^2} = 3g - 2 g^2 r^2 ;  V_en = -Z/r
    np.testing.assert_allclose(out["e_parts"][:, 0], 3 * gam - 2 * gam ** 2 * r2, rtol=1e-12)
    np.testing.assert_allclose(out["e_loc"], 3 * gam - 2 * gam ** 2 * r2 - Z / r, rtol=1e-12)
    np.testing.assert_allclose(out["drift"][:, 0], -2 * gam * R[:, 0], rtol=1e-12)
    np.testing.assert_allclose(out["logpsi"], -gam * r2, atol=1e-13)


def test_one_electron_gaussian_2p():
    gam = 0.6
    # MO = the p_x component only
    s = one_atom_system(2.0, [(1, [gam], [1.0])], n_up=1, n_dn=0, A_up=[[1.0], [0.0], [0.0]])
    o = Oracle(s)
    rng = np.random.default_rng(8)
    R = rng.normal(size=(5, 1, 3))
    out = o.eval(R)
    r2 = (R[:, 0] ** 2).sum(1)
    # lap(x e^{-g r^2}) / (x e^{-g r^2}) = 4 g^2 r^2 - 10 g
    np.testing.assert_allclose(out["e_parts"][:, 0], 5 * gam - 2 * gam ** 2 * r2, rtol=1e-11)
    x = R[:, 0, 0]
    np.testing.assert_allclose(out["drift"][:, 0, 0], 1 / x - 2 * gam * x, rtol=1e-10)


def test_two_electrons_same_orbital_opposite_spin():
    gam, Z = 1.1, 2.0
    s = one_atom_system(Z, [(0, [gam], [1.0])], n_up=1, n_dn=1, A_up=[[1.0]], A_dn=[[1.0]])
    o = Oracle(s)
    rng = np.random.default_rng(9)
    R = rng.normal(size=(4, 2, 3)) * 0.7
    out = o.eval(R)
    r2 = (R ** 2).sum(2)
    r12 = np.linalg.norm(R[:, 0] - R[:, 1], axis=1)
    expect = (3 * gam - 2 * gam ** 2 * r2).sum(1) - (Z / np.sqrt(r2)).sum(1) + 1 / r12
    np.testing.assert_allclose(out["e_loc"], expect, rtol=1e-12)


def test_coulomb_sums_brute_force(water):
    s, o = water
    R = make_walkers(s, 2)
    out = o.eval(R)
    for w in range(2):
        ven = vee = 0.0
        for i in range(s.n_elec):
            for a in range(s.n_atom):
                ven -= s.Z[a] / math.dist(R[w, i], s.Q[a])
            for j in range(i + 1, s.n_elec):
                vee += 1 / math.dist(R[w, i], R[w, j])
        vnn = sum(s.Z[a] * s.Z[b] / math.dist(s.Q[a], s.Q[b])
                  for a in range(s.n_atom) for b in range(a + 1, s.n_atom))
        np.testing.assert_allclose(out["e_parts"][w, 1:], [ven, vee, vnn], rtol=1e-13)
        assert abs(out["e_loc"][w] - out["e_parts"][w].sum()) < 1e-12 * abs(out["e_loc"][w])


def test_singular_walker_is_flagged(water):
    s, o = water
    R = make_walkers(s, 2)
    # an alpha electron far from every nucleus: all its AOs are screened,
    # its column of D is exactly zero and the zero pivot is exact
    R[1, 1] = [1e3, 0.0, 0.0]
    R[0, s.n_up + 1] = [0.0, -1e3, 0.0]
    out = o.eval(R)
    assert out["status"][1] & 1 and not out["status"][1] & 2
    assert out["status"][0] & 2 and not out["status"][0] & 1
    assert out["logpsi"][1] == -np.inf and out["sign"][1] == 0
    assert np.all(np.isnan(out["drift"][1, : s.n_up]))
