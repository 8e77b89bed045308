"""Pins for the oracle's adjoint d log|Psi| / dA (from the cofactor identity
behind the drift formula, Sec. II.C): central finite differences of the
oracle's own log|Psi| with respect to single MO coefficients, for a plain
walker average (g_w = 1/W) and an E_L-weighted one (g_w = 2(E_L,w - mean)/W).
"""
import numpy as np
import pytest

from oracle import Oracle
from synth import make_walkers, tiny_system


@pytest.mark.parametrize("weighting", ["plain", "eloc"])
def test_adjoint_matches_central_fd(weighting):
    s = tiny_system("mini_chain")
    o = Oracle(s)
    W = 3
    R = make_walkers(s, W)
    base = o.eval(R)
    if weighting == "plain":
        g = np.full(W, 1.0 / W)
    else:
        g = 2.0 * (base["e_loc"] - base["e_loc"].mean()) / W
    dA_up, dA_dn = o.logpsi_grad(R, g)
    rng = np.random.default_rng(21)
    h = 1e-6
    for which, dA in (("A_up", dA_up), ("A_dn", dA_dn)):
        for _ in range(8):
            mu = int(rng.integers(0, s.n_ao))
            j = int(rng.integers(0, dA.shape[1]))
            vals = []
            for sgn in (+1, -1):
                A = getattr(s, which).copy()
                A[mu, j] += sgn * h
                s2 = tiny_system("mini_chain")
                setattr(s2, which, A)
                vals.append(float((g * Oracle(s2).eval(R)["logpsi"]).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            scale = np.abs(dA).max()
            assert abs(fd - dA[mu, j]) < 1e-6 * scale, (which, mu, j, fd, dA[mu, j])
