"""Pins of the oracle's multi-determinant expansion (Sec. II.C, Eq. psit:
Psi = e^J sum_K c_K Det_K,up Det_K,dn):

* symbolic differentiation (sympy) of an explicit two-configuration trial
  function of two electrons, with and without a Jastrow factor;
* a single nonzero coefficient reproduces that determinant's evaluation;
* on the multi-atom test system with excited determinants: drift = finite-
  difference gradient of log|Psi|, T = finite-difference Laplacian of Psi.
"""
import math

import numpy as np
import sympy as sp

import oracle
from oracle import Oracle
from synth import excited_determinants, make_walkers, tiny_system
from tests.helpers import one_atom_system

JAS = dict(a_par=0.25, a_anti=0.5, b_ee=1.3, a_en=0.8, b_en=2.1)


def _two_config(jastrow):
    g1, g2, Z = 1.2, 0.35, 2.0
    shells = [(0, [g1], [1.0]), (0, [g2], [1.0])]
    d1 = one_atom_system(Z, shells, n_up=1, n_dn=1, A_up=[[1.0], [0.0]], A_dn=[[1.0], [0.0]])
    d2 = one_atom_system(Z, shells, n_up=1, n_dn=1, A_up=[[0.0], [1.0]], A_dn=[[0.0], [1.0]])
    c = [0.9, -0.4]
    xs = sp.symbols("x1 y1 z1 x2 y2 z2", real=True)
    r1s = xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2
    r2s = xs[3] ** 2 + xs[4] ** 2 + xs[5] ** 2
    psi = c[0] * sp.exp(-g1 * (r1s + r2s)) + c[1] * sp.exp(-g2 * (r1s + r2s))
    if jastrow:
        r12 = sp.sqrt((xs[0] - xs[3]) ** 2 + (xs[1] - xs[4]) ** 2 + (xs[2] - xs[5]) ** 2)
        U_en = lambda rs: -JAS["a_en"] * sp.sqrt(rs) / (1 + JAS["b_en"] * sp.sqrt(rs))
        psi = psi * sp.exp(JAS["a_anti"] * r12 / (1 + JAS["b_ee"] * r12) + U_en(r1s) + U_en(r2s))
    os_ = [Oracle(d, jastrow=JAS if jastrow else None) for d in (d1, d2)]
    return os_, c, psi, list(xs), Z


def test_two_configurations_symbolic():
    for jas in (False, True):
        os_, c, psi, xs, Z = _two_config(jas)
        lap = sum(sp.diff(psi, x, 2) for x in xs)
        f_psi = sp.lambdify(xs, psi, "numpy")
        f_lap = sp.lambdify(xs, lap, "numpy")
        f_grad = [sp.lambdify(xs, sp.diff(psi, x), "numpy") for x in xs]
        R = np.random.default_rng(6).normal(size=(4, 2, 3)) * 0.8
        out = oracle.multidet_eval(os_, c, R)
        for w in range(R.shape[0]):
            v = list(R[w].ravel())
            p = float(f_psi(*v))
            T = -0.5 * float(f_lap(*v)) / p
            V = -Z / np.linalg.norm(R[w, 0]) - Z / np.linalg.norm(R[w, 1]) + 1 / np.linalg.norm(R[w, 0] - R[w, 1])
            assert abs(out["logpsi"][w] - math.log(abs(p))) < 1e-11 * (1 + abs(math.log(abs(p))))
            assert out["sign"][w] == (1.0 if p > 0 else -1.0)
            assert abs(out["e_parts"][w, 0] - T) < 1e-10 * (1 + abs(T))
            assert abs(out["e_loc"][w] - (T + V)) < 1e-10 * (1 + abs(T + V))
            drift = np.array([float(g(*v)) / p for g in f_grad]).reshape(2, 3)
            assert np.abs(out["drift"][w] - drift).max() < 1e-10 * (1 + np.abs(drift).max())


def test_single_coefficient_is_that_determinant():
    s = tiny_system("mini_chain")
    dets = excited_determinants(s, 3)
    os_ = [Oracle(d) for d in dets]
    R = make_walkers(s, 3)
    ref = os_[1].eval(R)
    got = oracle.multidet_eval(os_, [0.0, 2.5, 0.0], R)
    np.testing.assert_allclose(got["logpsi"], ref["logpsi"] + math.log(2.5), rtol=1e-14)
    np.testing.assert_allclose(got["e_loc"], ref["e_loc"], rtol=1e-14)
    np.testing.assert_allclose(got["drift"], ref["drift"], rtol=1e-14)


def test_multidet_finite_differences():
    s = tiny_system("h2o_like")
    dets = excited_determinants(s, 3)
    os_ = [Oracle(d) for d in dets]
    c = [1.0, 0.3, -0.2]
    R = make_walkers(s, 1)
    base = oracle.multidet_eval(os_, c, R)
    h = 1e-5
    for e in range(s.n_elec):
        for l in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[0, e, l] += h
            Rm[0, e, l] -= h
            fd = (oracle.multidet_eval(os_, c, Rp)["logpsi"][0] - oracle.multidet_eval(os_, c, Rm)["logpsi"][0]) / (2 * h)
            assert abs(fd - base["drift"][0, e, l]) < 1e-6 * (1 + abs(fd))
    h = 1e-3
    lp0 = base["logpsi"][0]
    tot = 0.0
    for e in range(s.n_elec):
        for l in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[0, e, l] += h
            Rm[0, e, l] -= h
            op, om = oracle.multidet_eval(os_, c, Rp), oracle.multidet_eval(os_, c, Rm)
            psi_p = op["sign"][0] * math.exp(op["logpsi"][0] - lp0)
            psi_m = om["sign"][0] * math.exp(om["logpsi"][0] - lp0)
            tot += (psi_p - 2 * base["sign"][0] + psi_m) / (h * h) / base["sign"][0]
    T = base["e_parts"][0, 0]
    assert abs(-0.5 * tot - T) < 1e-4 * (1 + abs(T))
