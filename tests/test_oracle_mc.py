"""Pins of the oracle's Monte Carlo step (Sec. II.A Eqs. 1-3, fixed node;
Sec. II.B reconfiguration), each against something other than the oracle's
own formulas:

* Philox4x64-10 against numpy's implementation of the same published
  generator (numpy.random.Philox, which increments its counter before each
  block);
* the Gaussian noise of the move against the normal distribution
  (Kolmogorov-Smirnov, moments, pair independence);
* the move against the drift-diffusion it defines: displacements of many
  walkers from one point have mean tau b and covariance tau I;
* the weight against the properties of a branching factor: 1 when E_L equals
  E_T at both ends, below 1 above E_T, symmetric in the two ends, and the
  fixed-node rule (a sign change is never accepted);
* the reconfiguration against the probabilities it must realise (chi-square
  over many generations), invariance under rescaling all weights by a power
  of two (exact integer drawing), zero weights never drawn;
* the whole step against physics: fixed-node DMC of the hydrogen atom with a
  nodeless single-Gaussian trial function projects from its variational
  energy -4/(3 pi) = -0.4244 Ha to the exact ground-state energy -1/2 Ha.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from helpers import one_atom_system


@pytest.mark.parametrize("key", [(0, 0), (5, 7), (2 ** 64 - 1, 12345), (0xDEADBEEF, 2 ** 63)])
@pytest.mark.parametrize("ctr", [(1, 0, 0, 0), (7, 3, 9, 1), (2 ** 40, 2 ** 63, 11, 2 ** 64 - 1)])
def test_philox_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array((ctr[0] - 1,) + tuple(ctr[1:]), dtype=np.uint64))
    ref = bg.random_raw(4)
    got = oracle.philox4x64(ctr, key)
    np.testing.assert_array_equal(got, ref)


def test_move_normals_are_standard_normal():
    eta = oracle.move_normals(2000, 3 * 40, seed=99, step=3)     # 240000 numbers, 30 blocks per walker
    x = eta.ravel()
    n = x.size
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # the two numbers of one Box-Muller pair and neighbouring blocks are uncorrelated
    a, b = eta[:, 0::2].ravel(), eta[:, 1::2].ravel()
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(a.size)
    # other steps, walkers and seeds give other numbers
    assert not np.array_equal(oracle.move_normals(1, 12, 99, 3), oracle.move_normals(1, 12, 99, 4))
    assert not np.array_equal(oracle.move_normals(1, 12, 99, 3), oracle.move_normals(1, 12, 98, 3))
    assert np.array_equal(oracle.move_normals(2, 12, 99, 3)[1], oracle.move_normals(1, 12, 99, 3, w0=1)[0])


def test_move_is_drift_plus_diffusion():
    """Eq. (1): from one point R with drift b, R' - R ~ N(tau b, tau I)."""
    W, N, tau = 40000, 2, 0.03
    R = np.tile(np.array([[0.3, -1.2, 2.0], [1.0, 0.5, -0.25]]), (W, 1, 1))
    b = np.tile(np.array([[1.5, -0.7, 0.2], [-3.0, 0.0, 0.9]]), (W, 1, 1))
    d = (oracle.dmc_move(R, b, tau, seed=5, step=17) - R).reshape(W, 3 * N)
    mean = d.mean(axis=0)
    se = math.sqrt(tau / W)
    assert np.all(np.abs(mean - tau * b[0].ravel()) < 5 * se), (mean, tau * b[0].ravel())
    cov = np.cov(d.T)
    assert np.allclose(np.diag(cov), tau, rtol=0.03)
    off = cov - np.diag(np.diag(cov))
    assert np.abs(off).max() < 0.03 * tau
    # the same noise with and without drift: the two moves differ by tau b (up to rounding)
    d0 = oracle.dmc_move(R, np.zeros_like(b), tau, 5, 17)
    assert np.abs(oracle.dmc_move(R, b, tau, 5, 17) - d0 - tau * b).max() < 1e-14


def test_weight_properties_and_fixed_node_rule():
    tau, eT = 0.02, -10.0
    e_old = np.array([-10.0, -9.0, -11.0, -10.5, -9.5, -10.0, -10.0])
    e_new = np.array([-10.0, -9.0, -11.0, -9.5, -10.5, -8.0, -12.0])
    s_old = np.array([1.0, 1.0, -1.0, 1.0, 1.0, 1.0, -1.0])
    s_new = np.array([1.0, 1.0, -1.0, 1.0, 1.0, -1.0, -1.0])   # walker 5 crosses a node
    st_old = np.zeros(7, np.uint32)
    st_new = np.array([0, 0, 0, 0, 0, 0, 4], np.uint32)        # walker 6: proposed state invalid
    w, acc = oracle.dmc_weight(e_old, s_old, st_old, e_new, s_new, st_new, tau, eT)
    assert w[0] == 1.0                                      # E_L = E_T at both ends
    assert w[1] < 1.0 < w[2]                                # above E_T walkers die, below they multiply
    assert w[3] == w[4]                                     # symmetric in the two ends
    assert list(acc) == [1, 1, 1, 1, 1, 0, 0]               # no node crossing, no invalid move
    # a rejected move weighs the walker at its old position at both ends
    w_rej, _ = oracle.dmc_weight(e_old[5:], s_old[5:], st_old[5:], e_old[5:], s_old[5:], st_old[5:], tau, eT)
    np.testing.assert_array_equal(w[5:], w_rej)
    # an invalid old walker carries no weight
    w_bad, acc_bad = oracle.dmc_weight(e_old[:1], s_old[:1], np.array([1], np.uint32), e_new[:1], s_new[:1],
                                       st_new[:1], tau, eT)
    assert w_bad[0] == 0.0 and acc_bad[0] == 0
    # a constant E_L above E_T by dE for n steps multiplies the weight by exp(-n tau dE)
    dE = 0.37
    wn, _ = oracle.dmc_weight(np.full(1, eT + dE), np.ones(1), np.zeros(1, np.uint32), np.full(1, eT + dE),
                              np.ones(1), np.zeros(1, np.uint32), tau, eT)
    assert abs(math.log(wn[0]) * 50 + 50 * tau * dE) < 1e-12


def test_reconfiguration_draws_with_the_weights():
    p = np.array([1.0, 2.0, 3.0, 4.0, 0.0, 2.5])
    W = p.size
    counts = np.zeros(W)
    n_gen = 4000
    for step in range(n_gen):
        idx, sw, alive, zero = oracle.srmc(p, seed=3, step=step)
        assert not zero and alive == 5 and sw == p.sum()
        counts += np.bincount(idx, minlength=W)
    assert counts[4] == 0                                   # zero weight: never drawn
    expect = n_gen * W * p / p.sum()
    live = p > 0
    chi2 = (((counts - expect) ** 2) / np.where(live, expect, 1.0))[live].sum()
    assert stats.chi2.sf(chi2, live.sum() - 1) > 1e-4, (counts, expect)


def test_reconfiguration_exact_integer_drawing():
    rng = np.random.default_rng(4)
    w = np.exp(rng.normal(size=257))
    idx, _, _, _ = oracle.srmc(w, seed=8, step=5)
    for k in (-30, -1, 1, 17):                               # weights times 2^k: the same draws
        idx2, _, _, _ = oracle.srmc(np.ldexp(w, k), seed=8, step=5)
        np.testing.assert_array_equal(idx, idx2)
    w2 = w.copy()
    w2[[3, 50]] = [np.nan, -1.0]                              # non-finite and negative: dropped
    idx3, _, alive, _ = oracle.srmc(w2, seed=8, step=5)
    assert alive == 255 and not np.isin(idx3, [3, 50]).any()
    dom = np.full(64, 1e-300)
    dom[9] = 1.0
    idx4, _, _, _ = oracle.srmc(dom, seed=8, step=5)          # below 2^-40 of the largest: never drawn
    assert (idx4 == 9).all()
    idx5, _, alive5, zero = oracle.srmc(np.zeros(10), seed=8, step=5)
    assert zero and alive5 == 0 and (idx5 == np.arange(10)).all()


def test_dmc_hydrogen_atom_projects_to_exact_energy():
    """Fixed-node DMC with constant population (Sec. II) on one electron and a
    proton, trial function one normalised s Gaussian with the variationally
    optimal exponent 8 / (9 pi): VMC gives -4 / (3 pi) = -0.4244 Ha; the
    trial function has no node, so DMC is exact up to the time step and
    population control: -0.5 Ha.  Estimator: sum_n P_n sum_k w_k E_L,k /
    sum_n P_n sum_k w_k with P_n the product of the 50 preceding generations'
    mean weights (the paper's global weight over a window)."""
    g = 8.0 / (9.0 * math.pi)
    c = (2.0 * g / math.pi) ** 0.75
    s = one_atom_system(1, [(0, [g], [c])], 1, 0, [[1.0]])
    o = oracle.Oracle(s)
    M, tau, nstep, neq, L = 1000, 0.02, 2000, 400, 50
    R = np.random.default_rng(1).normal(size=(M, 1, 3)) * 1.2
    ev = o.eval(R)
    st = {"R": R, "drift": ev["drift"], "e_loc": ev["e_loc"], "logpsi": ev["logpsi"], "sign": ev["sign"],
          "status": ev["status"]}
    eT, num, den, logw = -0.45, 0.0, 0.0, []
    for n in range(nstep):
        st, info = oracle.dmc_step(o, st, tau, eT, seed=21, step=n)
        logw.append(math.log(info["sum_w"] / M))
        P = math.exp(sum(logw[-L - 1:-1])) if n >= 1 else 1.0
        if n >= neq:
            num += P * info["sum_w_eloc"]
            den += P * info["sum_w"]
            eT = num / den
    e_dmc = num / den
    assert abs(e_dmc + 0.5) < 0.02, e_dmc
    assert e_dmc < -4.0 / (3.0 * math.pi) - 0.05
