"""Step a1 of the mixed path (qmc_shell_masks) against the oracle's screening,
bit-exact: the mask kernel decides d2 < R2 in FP32 away from the shell radius
and falls back to the exact FP64 test inside an error band, so the decisions
must equal the FP64 ones everywhere, including electrons placed within a few
ulps of a shell radius."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu

dev = torch.device("cuda", 0)


def _oracle_masks(s, o, pts, words):
    cnt, idx = o.screen_points(pts)
    out = np.zeros((len(pts), words), dtype=np.uint32)
    for p in range(len(pts)):
        for sh in np.unique(s.ao_shell[idx[p, : cnt[p]]]):
            out[p, sh >> 5] |= np.uint32(1) << np.uint32(sh & 31)
    return out


def _gpu_masks(q, R):
    m = q.shell_masks(torch.from_numpy(R).to(dev))
    return m.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("key", ["158e", "434e", "1056e"])
def test_masks_match_oracle_on_walkers(key):
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system(key)
    o, q = Oracle(s), QmcSystem(s, 0)
    W = 3
    R = make_walkers(s, W, first=700)
    R[0, 1] = [1.0e3, -2.0e3, 5.0e2]          # far away: no active shell
    R[1, 0] = s.Q[s.n_atom // 2]               # on a nucleus
    got = _gpu_masks(q, R)
    words = got.shape[-1]
    assert words == (s.n_shell + 31) // 32
    want = _oracle_masks(s, o, R.reshape(-1, 3), words).reshape(W, s.n_elec, words)
    np.testing.assert_array_equal(got, want)
    assert not got[0, 1].any()


def test_masks_at_shell_radii():
    """Electrons a few ulps inside and outside shell radii, along each axis
    and along a diagonal, from a sample of shells of every atom type."""
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("434e")
    o, q = Oracle(s), QmcSystem(s, 0)
    rng = np.random.default_rng(11)
    shells = rng.choice(s.n_shell, size=60, replace=False)
    pts = []
    for sh in shells:
        a = s.shell_atom[sh]
        r = np.sqrt(o.R2[sh])
        for direction in (np.array([1.0, 0, 0]), np.array([0, -1.0, 0]), np.array([0, 0, 1.0]),
                          np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)):
            base = s.Q[a] + r * direction
            for k in range(-3, 4):
                p = base.copy()
                for c in range(3):
                    if direction[c] != 0:
                        step = np.spacing(abs(p[c]))
                        p[c] = p[c] + k * step * np.sign(direction[c])
                pts.append(p)
    pts = np.array(pts)
    N = s.n_elec
    n = (len(pts) + N - 1) // N
    R = np.tile(make_walkers(s, 1, first=900), (n, 1, 1))
    R.reshape(-1, 3)[: len(pts)] = pts
    got = _gpu_masks(q, R).reshape(n * N, -1)[: len(pts)]
    want = _oracle_masks(s, o, pts, got.shape[-1])
    np.testing.assert_array_equal(got, want)
    # the sample straddles the radii: both decisions occur for the sampled shells
    act = [(got[i, sh >> 5] >> (sh & 31)) & 1 for i, sh in enumerate(np.repeat(shells, 28))]
    assert 0 < sum(act) < len(act)


def test_mask_words_query():
    from paper_1209_6630_gb300 import QmcSystem
    from paper_1209_6630_gb300._lib import lib
    import ctypes as C
    s = config_system("158e")
    q = QmcSystem(s, 0)
    words = C.c_int(-1)
    assert lib().qmc_shell_masks(q.handle, 0, None, None, C.byref(words), None) == 0
    assert words.value == (s.n_shell + 31) // 32
