"""Pins of the oracle's Jastrow factor (Sec. II.C, Psi_T = e^J Det_up Det_dn
with J = sum_{i<j} U_ee(r_ij) + sum_{i,a} U_en(r_ia); the Pade forms
U_ee = a r / (1 + b r), a = a_par or a_anti by spin pair, U_en = -a_a r /
(1 + b_a r)).

* Closed forms from symbolic differentiation (sympy) of the explicit trial
  function -- one electron with an e-n factor, two electrons of opposite spin
  in one orbital, two electrons of equal spin in an s and a p orbital (a 2x2
  determinant): log|Psi|, the drift grad Psi / Psi and E_L = -1/2 sum lap Psi /
  Psi + V, each written out without the oracle's derivative formulas;
* on a multi-atom system: drift = finite-difference gradient of log|Psi| and
  T = finite-difference Laplacian of Psi itself.
"""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import Oracle
from synth import make_walkers, tiny_system
from tests.helpers import one_atom_system

JAS = dict(a_par=0.25, a_anti=0.5, b_ee=1.3, a_en=0.8, b_en=2.1)


def _sym_check(o, R, psi, xs, Z_terms, atol=1e-11):
    """Compare the oracle with the symbolic trial function psi(xs) at points R."""
    n = len(xs) // 3
    lap = sum(sp.diff(psi, x, 2) for x in xs)
    f_psi = sp.lambdify(xs, psi, "numpy")
    f_lap = sp.lambdify(xs, lap, "numpy")
    f_grad = [sp.lambdify(xs, sp.diff(psi, x), "numpy") for x in xs]
    out = o.eval(R)
    for w in range(R.shape[0]):
        v = list(R[w].ravel())
        p = float(f_psi(*v))
        T = -0.5 * float(f_lap(*v)) / p
        pts = R[w]
        V = Z_terms(pts)
        assert abs(out["logpsi"][w] - math.log(abs(p))) < atol * (1 + abs(math.log(abs(p))))
        assert abs(out["e_parts"][w, 0] - T) < atol * (1 + abs(T))
        assert abs(out["e_loc"][w] - (T + V)) < atol * (1 + abs(T + V))
        drift = np.array([float(g(*v)) / p for g in f_grad]).reshape(n, 3)
        assert np.abs(out["drift"][w] - drift).max() < atol * (1 + np.abs(drift).max())


def test_one_electron_with_en_factor():
    gam, Z = 0.9, 1.0
    s = one_atom_system(Z, [(0, [gam], [1.0])], n_up=1, n_dn=0, A_up=[[1.0]])
    o = Oracle(s, jastrow=JAS)
    x, y, z = sp.symbols("x y z", real=True)
    r = sp.sqrt(x * x + y * y + z * z)
    psi = sp.exp(-gam * r ** 2) * sp.exp(-JAS["a_en"] * r / (1 + JAS["b_en"] * r))
    R = np.random.default_rng(3).normal(size=(4, 1, 3)) * 0.9
    _sym_check(o, R, psi, [x, y, z], lambda p: -Z / np.linalg.norm(p[0]))


def test_two_electrons_opposite_spin_one_orbital():
    gam, Z = 1.1, 2.0
    s = one_atom_system(Z, [(0, [gam], [1.0])], n_up=1, n_dn=1, A_up=[[1.0]], A_dn=[[1.0]])
    o = Oracle(s, jastrow=JAS)
    xs = sp.symbols("x1 y1 z1 x2 y2 z2", real=True)
    r1 = sp.sqrt(xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2)
    r2 = sp.sqrt(xs[3] ** 2 + xs[4] ** 2 + xs[5] ** 2)
    r12 = sp.sqrt((xs[0] - xs[3]) ** 2 + (xs[1] - xs[4]) ** 2 + (xs[2] - xs[5]) ** 2)
    U_en = lambda r: -JAS["a_en"] * r / (1 + JAS["b_en"] * r)
    J = JAS["a_anti"] * r12 / (1 + JAS["b_ee"] * r12) + U_en(r1) + U_en(r2)
    psi = sp.exp(-gam * r1 ** 2) * sp.exp(-gam * r2 ** 2) * sp.exp(J)
    R = np.random.default_rng(4).normal(size=(3, 2, 3)) * 0.7

    def V(p):
        return -Z / np.linalg.norm(p[0]) - Z / np.linalg.norm(p[1]) + 1 / np.linalg.norm(p[0] - p[1])
    _sym_check(o, R, psi, list(xs), V)


def test_two_electrons_equal_spin_determinant():
    gs, gp, Z = 0.8, 0.6, 3.0
    s = one_atom_system(Z, [(0, [gs], [1.0]), (1, [gp], [1.0])], n_up=2, n_dn=0,
                        A_up=[[1.0, 0.0], [0.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    o = Oracle(s, jastrow=JAS)
    xs = sp.symbols("x1 y1 z1 x2 y2 z2", real=True)
    r1s = xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2
    r2s = xs[3] ** 2 + xs[4] ** 2 + xs[5] ** 2
    r12 = sp.sqrt((xs[0] - xs[3]) ** 2 + (xs[1] - xs[4]) ** 2 + (xs[2] - xs[5]) ** 2)
    phi_s = lambda rs: sp.exp(-gs * rs)
    phi_p = lambda xx, rs: xx * sp.exp(-gp * rs)
    det = phi_s(r1s) * phi_p(xs[3], r2s) - phi_s(r2s) * phi_p(xs[0], r1s)
    U_en = lambda rs: -JAS["a_en"] * sp.sqrt(rs) / (1 + JAS["b_en"] * sp.sqrt(rs))
    J = JAS["a_par"] * r12 / (1 + JAS["b_ee"] * r12) + U_en(r1s) + U_en(r2s)
    psi = det * sp.exp(J)
    R = np.random.default_rng(5).normal(size=(3, 2, 3)) * 0.8

    def V(p):
        return -Z / np.linalg.norm(p[0]) - Z / np.linalg.norm(p[1]) + 1 / np.linalg.norm(p[0] - p[1])
    _sym_check(o, R, psi, list(xs), V, atol=1e-10)


@pytest.fixture(scope="module")
def water_j():
    s = tiny_system("h2o_like")
    jas = dict(JAS, a_en=np.linspace(0.3, 1.1, s.n_atom), b_en=np.linspace(1.0, 3.0, s.n_atom))
    return s, Oracle(s, jastrow=jas), Oracle(s)


def test_jastrow_drift_and_kinetic_by_finite_differences(water_j):
    s, o, o0 = water_j
    R = make_walkers(s, 1)
    base = o.eval(R)
    assert abs(base["logpsi"][0] - o0.eval(R)["logpsi"][0]) > 1e-3     # the factor is there
    h = 1e-5
    for e in range(s.n_elec):
        for l in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[0, e, l] += h
            Rm[0, e, l] -= h
            fd = (o.eval(Rp)["logpsi"][0] - o.eval(Rm)["logpsi"][0]) / (2 * h)
            assert abs(fd - base["drift"][0, e, l]) < 1e-6 * (1 + abs(fd))
    h = 1e-3
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
            tot += (psi_p - 2 * base["sign"][0] + psi_m) / (h * h) / base["sign"][0]
    T = base["e_parts"][0, 0]
    assert abs(-0.5 * tot - T) < 1e-4 * (1 + abs(T))
