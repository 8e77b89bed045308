"""Pins for the oracle's AO evaluation (Sec. II.C AO form; Eq. "Gaussian").

Checked against what the mathematics fixes, not against the oracle itself:
central finite differences of chi, the closed-form derivatives of a single
Cartesian Gaussian primitive, and unit norm by spherical quadrature.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from synth import config_system, tiny_system
from tests.helpers import one_atom_system


@pytest.fixture(scope="module")
def mini():
    s = tiny_system("mini_chain")
    return s, Oracle(s)


def _points_near(s, a, n, rng, spread=1.5):
    return s.Q[a] + spread * rng.normal(size=(n, 3))


def test_gradient_matches_central_fd(mini):
    s, o = mini
    rng = np.random.default_rng(1)
    h = 1e-5
    for mu in range(0, s.n_ao, 3):
        a = s.shell_atom[s.ao_shell[mu]]
        pts = _points_near(s, a, 4, rng)
        v = o.ao_points(mu, pts)
        for l in range(3):
            e = np.zeros(3); e[l] = h
            fd = (o.ao_points(mu, pts + e)[:, 0] - o.ao_points(mu, pts - e)[:, 0]) / (2 * h)
            scale = np.abs(v[:, 1:4]).max() + 1e-30
            assert np.max(np.abs(fd - v[:, 1 + l])) < 1e-6 * scale + 1e-12


def test_laplacian_matches_second_fd(mini):
    s, o = mini
    rng = np.random.default_rng(2)
    h = 1e-3
    for mu in range(1, s.n_ao, 3):
        a = s.shell_atom[s.ao_shell[mu]]
        pts = _points_near(s, a, 4, rng)
        v = o.ao_points(mu, pts)
        lap = -6.0 * v[:, 0]
        for l in range(3):
            e = np.zeros(3); e[l] = h
            lap = lap + o.ao_points(mu, pts + e)[:, 0] + o.ao_points(mu, pts - e)[:, 0]
        lap /= h * h
        scale = np.abs(v[:, 4]).max() + np.abs(v[:, 0]).max()
        assert np.max(np.abs(lap - v[:, 4])) < 2e-4 * scale


@pytest.mark.parametrize("L", [0, 1, 2])
def test_single_primitive_closed_form(L):
    gam, c = 0.73, 1.3
    n_comp = (L + 1) * (L + 2) // 2
    s = one_atom_system(1, [(L, [gam], [c])], n_up=1, n_dn=0, A_up=np.eye(n_comp)[:, :1],
                        Q=(0.3, -0.2, 0.1))
    o = Oracle(s)
    rng = np.random.default_rng(3)
    pts = np.array(s.Q[0]) + rng.uniform(0.3, 1.2, size=(6, 3)) * rng.choice([-1, 1], size=(6, 3))
    for mu in range(n_comp):
        n = s.ao_pow[mu]
        v = o.ao_points(mu, pts)
        d = pts - s.Q[0]
        r2 = (d ** 2).sum(1)
        chi = c * np.prod(d ** n, axis=1) * np.exp(-gam * r2)
        np.testing.assert_allclose(v[:, 0], chi, rtol=1e-13)
        for l in range(3):
            # d_l chi / chi = n_l / d_l - 2 gamma d_l
            np.testing.assert_allclose(v[:, 1 + l], chi * (n[l] / d[:, l] - 2 * gam * d[:, l]), rtol=1e-11)
        # lap chi / chi = sum_l n_l (n_l - 1) / d_l^2 - 2 gamma (2L + 3) + 4 gamma^2 |d|^2
        ratio = (n * (n - 1) / d ** 2).sum(1) - 2 * gam * (2 * L + 3) + 4 * gam ** 2 * r2
        np.testing.assert_allclose(v[:, 4], chi * ratio, rtol=1e-10, atol=1e-13)


def _sphere_quadrature(o, mu, centre, rmax=30.0, npanel=400, nrad=6, ncos=8, nphi=12):
    xg, wg = np.polynomial.legendre.leggauss(nrad)
    edges = rmax * (np.arange(npanel + 1) / npanel) ** 2
    a, b = edges[:-1, None], edges[1:, None]
    r = (0.5 * (b - a) * xg + 0.5 * (b + a)).ravel()
    wr = (0.5 * (b - a) * wg).ravel() * r ** 2
    ct, wct = np.polynomial.legendre.leggauss(ncos)
    ph = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(nphi))], -1)
    dirs = dirs.reshape(-1, 3)
    wang = np.outer(wct, np.full(nphi, 2 * np.pi / nphi)).ravel()
    pts = centre + (r[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
    w = (wr[:, None] * wang[None, :]).ravel()
    chi = o.ao_points(mu, pts)[:, 0]
    return float((w * chi * chi).sum())


def test_unit_norm_by_quadrature():
    s = config_system("158e")
    o = Oracle(s)
    # one heavy atom (s core with 8 primitives, s, s, p, p, d) and one H
    heavy = [mu for mu in range(s.n_ao) if s.shell_atom[s.ao_shell[mu]] == 0]
    h_atom = s.n_atom - 1
    hyd = [mu for mu in range(s.n_ao) if s.shell_atom[s.ao_shell[mu]] == h_atom]
    for mu in heavy + hyd:
        a = s.shell_atom[s.ao_shell[mu]]
        norm = _sphere_quadrature(o, mu, s.Q[a])
        assert abs(norm - 1.0) < 1e-6, (mu, norm)
