"""Pins for the oracle's products (Eq. "abc") and inversion step (Sec. IV.B).

* LU + inverse against numpy's slogdet / inv and against the Leibniz formula;
* an exactly singular matrix gives log|det| = -inf and sign 0;
* the sparse product loop equals a dense matrix product with zeros for
  screened AOs (numpy einsum), and rows of D^-1 are the duals of columns of D.
"""
import itertools

import numpy as np

from oracle import Oracle, lu_inverse
from synth import make_walkers, tiny_system


def test_lu_inverse_matches_numpy():
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 40, 97):
        M = rng.normal(size=(n, n))
        la, sg, inv = lu_inverse(M)
        s_np, la_np = np.linalg.slogdet(M)
        assert sg == s_np
        assert abs(la - la_np) < 1e-12 * max(1.0, abs(la_np))
        np.testing.assert_allclose(inv, np.linalg.inv(M), rtol=1e-9, atol=1e-11)


def _leibniz(M):
    n = M.shape[0]
    tot = 0.0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        tot += (-1) ** inv * np.prod([M[i, p[i]] for i in range(n)])
    return tot


def test_lu_matches_leibniz():
    rng = np.random.default_rng(12)
    for n in (1, 2, 3, 4):
        for _ in range(5):
            M = rng.normal(size=(n, n))
            la, sg, _ = lu_inverse(M)
            d = _leibniz(M)
            assert sg == np.sign(d)
            assert abs(la - np.log(abs(d))) < 1e-12


def test_singular_matrix():
    M = np.arange(16.0).reshape(4, 4)
    M[2] = M[1]
    la, sg, inv = lu_inverse(M)
    assert la == -np.inf and sg == 0.0 and inv is None


def test_products_equal_dense_einsum_and_dual_identity():
    s = tiny_system("mini_chain")
    o = Oracle(s)
    R = make_walkers(s, 1)[0]
    d = o.eval_debug(R)
    for spin, (ns, e0, A, Cs, Dinv) in enumerate(((s.n_up, 0, s.A_up, d["C_up"], d["dinv_up"]),
                                                   (s.n_dn, s.n_up, s.A_dn, d["C_dn"], d["dinv_dn"]))):
        Bd = np.zeros((5, ns, s.n_ao))
        for i in range(ns):
            e = e0 + i
            K = d["cnt"][e]
            Bd[:, i, d["idx"][e, :K]] = d["B"][e, :, :K]
        Cref = np.einsum("lim,mj->lij", Bd, A)
        np.testing.assert_allclose(Cs, Cref, rtol=1e-12, atol=1e-14)
        # D_ji = phi_j(r_i);  D^-1 rows are electrons: sum_j Dinv[i,j] D[j,i] = 1
        D = Cs[0].T
        np.testing.assert_allclose(Dinv @ D, np.eye(ns), atol=1e-9)
        np.testing.assert_allclose(Dinv, np.linalg.inv(D), rtol=1e-8, atol=1e-10)
        sgn, la = np.linalg.slogdet(D)
        assert abs(la - d["logabs"][spin]) < 1e-10 * abs(la)
        assert sgn == d["sign"][spin]
