"""Pins for the oracle's screening (Sec. III: AO dropped where g < eps,
atomic-radius early exit) and for what screening does to the products.

* the stored radius R2 of every shell is the first double at which g < eps;
* the per-electron lists equal a brute-force scan over every shell (no atomic
  early exit), away from the eps boundary where two exp implementations may
  disagree by an ulp;
* at d2 == R2 the shell is inactive, one ulp below it is active (strict <);
* screened vs unscreened products differ by at most the dropped terms.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from synth import config_system, make_walkers, tiny_system
from tests.helpers import one_atom_system


def _g(s, t, x):
    p0, n = s.shell_pstart[t], s.shell_nprim[t]
    return sum(s.prim_coef[p0 + k] * math.exp(-s.prim_gamma[p0 + k] * x) for k in range(n))


def test_radius_is_first_double_below_eps():
    s = config_system("158e")
    o = Oracle(s)
    for t in range(s.n_shell):
        r2 = o.R2[t]
        assert r2 > 0
        assert _g(s, t, r2) < s.eps
        assert _g(s, t, np.nextafter(r2, 0.0)) >= s.eps


def test_lists_match_brute_force():
    s = config_system("158e")
    o = Oracle(s)
    rng = np.random.default_rng(5)
    lo, hi = s.Q.min(0) - 4, s.Q.max(0) + 4
    pts = rng.uniform(lo, hi, size=(150, 3))
    pts = np.concatenate([pts, make_walkers(s, 1)[0][:60]])
    cnt, idx = o.screen_points(pts)
    sh_first = np.searchsorted(s.ao_shell, np.arange(s.n_shell))
    checked = 0
    for p, r in enumerate(pts):
        expect, ambiguous = [], False
        for t in range(s.n_shell):
            d = r - s.Q[s.shell_atom[t]]
            d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
            g = _g(s, t, d2)
            if abs(g - s.eps) < 1e-9 * s.eps:
                ambiguous = True
            if g >= s.eps:
                L = s.shell_L[t]
                expect.extend(range(sh_first[t], sh_first[t] + (L + 1) * (L + 2) // 2))
        if ambiguous:
            continue
        checked += 1
        assert list(idx[p, : cnt[p]]) == sorted(expect)
    assert checked > 200


def test_boundary_is_strict():
    s = one_atom_system(1, [(0, [0.8, 0.2], [0.9, 0.4]), (1, [0.5], [0.7])], n_up=1, n_dn=0,
                        A_up=np.ones((4, 1)))
    o = Oracle(s)
    for t in range(2):
        R2 = o.R2[t]
        x = math.sqrt(R2)
        # search neighbouring doubles x for x*x == R2 and for x*x just below R2
        cands = [x]
        for _ in range(8):
            cands.append(np.nextafter(cands[-1], 0.0))
        cands.append(x)
        y = x
        for _ in range(8):
            y = np.nextafter(y, np.inf)
            cands.append(y)
        below = max((c for c in cands if c * c < R2), key=lambda c: c * c)
        atleast = min((c for c in cands if c * c >= R2), key=lambda c: c * c)
        other_R2 = o.R2[1 - t]
        for c, active in ((below, True), (atleast, False)):
            cnt, idx = o.screen_points(np.array([[c, 0.0, 0.0]]))
            got = set(idx[0, : cnt[0]].tolist())
            mine = set(range(0, 1)) if t == 0 else set(range(1, 4))
            assert (mine <= got) == active
            assert len(mine & got) in (0, len(mine))
        # the other shell's decision is just its own comparison
        assert other_R2 != R2


def test_screening_error_bounded_by_dropped_terms():
    s = tiny_system("mini_chain")
    o_scr, o_full = Oracle(s), Oracle(s, unscreened=True)
    R = make_walkers(s, 2)
    for w in range(2):
        a = o_scr.eval_debug(R[w])
        b = o_full.eval_debug(R[w])
        for spin, (ns, e0, A) in enumerate(((s.n_up, 0, s.A_up), (s.n_dn, s.n_up, s.A_dn))):
            Ca, Cb = (a["C_up"], b["C_up"]) if spin == 0 else (a["C_dn"], b["C_dn"])
            for i in range(ns):
                e = e0 + i
                kept = set(a["idx"][e, : a["cnt"][e]].tolist())
                full_idx = b["idx"][e, : b["cnt"][e]]
                assert b["cnt"][e] == s.n_ao
                bound = np.zeros((5, ns))
                for k, mu in enumerate(full_idx):
                    if mu in kept:
                        continue
                    bound += np.abs(b["B"][e, :, k])[:, None] * np.abs(A[mu])[None, :]
                diff = np.abs(Ca[:, i, :] - Cb[:, i, :])
                assert np.all(diff <= bound + 1e-13 * (np.abs(Cb[:, i, :]) + 1))
        # every dropped AO is below eps in its radial part, so the effect is tiny
        assert abs(a["logabs"].sum() - b["logabs"].sum()) < 1e-4
