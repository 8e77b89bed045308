"""a4 with the panel updates on the tensor cores (a4_mode = tensor): the
Gauss-Jordan elimination of the float-float mode in panels of 32 columns,
each rank-32 update computed from exact BF16 slices of the panel and of the
pivot rows (orders 0..2 accumulated exactly, 3..5 rounded at ~2^-45 of the
update) and added to the float-pair matrix.  Against the float-float
elimination on the same C1 (no FP64 recomputation: threshold 1e30) the two
differ by the slices' rounding only; against the oracle both meet the mixed
path's bounds.  Covers a ragged last panel (79 and 217 electrons per spin),
the open-shell 866/865 system (seven row and column tiles) and singular
matrices (decided in FP64)."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


def _q(key):
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system(key)
    return s, QmcSystem(s, 0)


@pytest.mark.parametrize("key,W", [("158e", 40), ("434e", 24), ("1056e", 6), ("1731e", 3)])
def test_tensor_matches_float_float(key, W):
    s, q = _q(key)
    Rd = torch.from_numpy(make_walkers(s, W, first=510)).to(dev)
    try:
        q.set_tiles(a4_mode="float_float", a4_kappa_max=1e30)
        ff = q.eval(Rd, precision="mixed", want_dinv=True)
        q.set_tiles(a4_mode="tensor")
        tc = q.eval(Rd, precision="mixed", want_dinv=True)
    finally:
        q.set_tiles(a4_mode="float_float", a4_kappa_max=1e8)
    assert torch.equal(ff["status"], tc["status"]) and torch.equal(ff["sign"], tc["sign"])
    d_lp = (ff["logpsi"] - tc["logpsi"]).abs().max().item()
    d_inv = ((ff["dinv"] - tc["dinv"]).abs().max() / ff["dinv"].abs().max()).item()
    d_el = ((ff["e_loc"] - tc["e_loc"]).abs() / ff["e_loc"].abs()).max().item()
    print(f"{key}: |dlogpsi| {d_lp:.2e}, D^-1 normwise {d_inv:.2e}, E_L rel {d_el:.2e}")
    # the slices round the orders 3..5 at ~2^-45 of an update (float pairs: 2^-48); E_L
    # carries the D^-1 difference through the kinetic term, amplified where T and V cancel
    assert d_lp < 1e-8 and d_inv < 1e-8 and d_el < 1e-7


@pytest.mark.parametrize("key,W", [("158e", 60), ("434e", 24)])
def test_tensor_vs_oracle(key, W):
    s, q = _q(key)
    R = make_walkers(s, W, first=520)
    ref = Oracle(s).eval(R)
    q.set_tiles(a4_mode="tensor")
    try:
        g = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    finally:
        q.set_tiles(a4_mode="float_float")
    g = {k: v.cpu().numpy() for k, v in g.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["sign"], ref["sign"])
    assert np.abs(g["logpsi"] - ref["logpsi"]).max() < 1e-6
    assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5


def test_tensor_singular_decided_in_fp64():
    s, q = _q("434e")
    R = make_walkers(s, 6, first=99)
    R[2, 7] = [2e3, 0.0, 0.0]                    # alpha electron without AOs: exactly singular Det_up
    R[4, s.n_up + 3] = [0.0, 2e3, 0.0]
    q.set_tiles(a4_mode="tensor")
    try:
        o = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    finally:
        q.set_tiles(a4_mode="float_float")
    st = o["status"].cpu().numpy()
    assert st[2] == 1 and st[4] == 2 and (st[[0, 1, 3, 5]] == 0).all()
    lp = o["logpsi"].cpu().numpy()
    assert lp[2] == -np.inf and lp[4] == -np.inf


@pytest.mark.parametrize("kind", ["mini_chain", "small_chain"])
def test_tensor_small_matrices_vs_oracle(kind):
    """Matrices of one column tile (20 and 19 rows: no update tile besides the panel's own) and
    of two (49 rows: one update tile, ragged), 130 walkers."""
    from paper_1209_6630_gb300 import QmcSystem
    from synth import tiny_system
    from synth.system import make_system
    s = tiny_system("mini_chain") if kind == "mini_chain" else make_system(8, 2, 2, 20, seed=3)
    q = QmcSystem(s, 0)
    W = 130
    R = make_walkers(s, W, first=40)
    ref = Oracle(s).eval(R)
    q.set_tiles(a4_mode="tensor")
    g = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    g = {k: v.cpu().numpy() for k, v in g.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["sign"], ref["sign"])
    assert np.abs(g["logpsi"] - ref["logpsi"]).max() < 1e-6
    assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5
