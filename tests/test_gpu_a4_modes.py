"""a4 arithmetic of the mixed path: Gauss-Jordan on float pairs with FP64
recomputation of the matrices it flags (kappa_inf above the threshold, zero
pivot, non-finite result), against FP64 Gauss-Jordan and the oracle."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def sysq():
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("434e")
    return s, QmcSystem(s, 0)


def test_float_float_matches_fp64_and_oracle(sysq):
    s, q = sysq
    R = make_walkers(s, 24, first=321)
    Rd = torch.from_numpy(R).to(dev)
    ref = Oracle(s).eval(R)
    # no recomputation here: the comparison is of the two a4 arithmetics on the same C1
    q.set_tiles(a4_mode="float_float", a4_kappa_max=1e30)
    ff = q.eval(Rd, precision="mixed", want_dinv=True)
    q.set_tiles(a4_mode="fp64")
    fp = q.eval(Rd, precision="mixed", want_dinv=True)
    q.set_tiles(a4_mode="float_float", a4_kappa_max=1e8)
    for o in (ff, fp):
        lp, el = o["logpsi"].cpu().numpy(), o["e_loc"].cpu().numpy()
        assert np.abs(lp - ref["logpsi"]).max() < 1e-6
        assert (np.abs(el - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5
    # float pairs carry ~48 bits: the two a4 arithmetics agree far inside the bounds
    assert (ff["logpsi"] - fp["logpsi"]).abs().max().item() < 1e-8
    d_ff, d_fp = ff["dinv"].cpu().numpy(), fp["dinv"].cpu().numpy()
    assert np.abs(d_ff - d_fp).max() <= 1e-8 * np.abs(d_fp).max()


def test_threshold_one_recomputes_every_matrix_in_fp64(sysq):
    """Every matrix flagged: C1 and the elimination are recomputed in FP64, so
    log|Psi| and D^-1 are those of the FP64 path (same screening, FP64 AO
    values and products, the same Gauss-Jordan arithmetic and panel width)."""
    s, q = sysq
    Rd = torch.from_numpy(make_walkers(s, 10, first=55)).to(dev)
    f64 = q.eval(Rd, precision="f64", want_dinv=True)
    q.set_tiles(a4_mode="float_float", a4_kappa_max=1.0)   # every kappa_inf >= 1: all flagged
    try:
        rec = q.eval(Rd, precision="mixed", want_dinv=True)
    finally:
        q.set_tiles(a4_kappa_max=1e8)
    assert torch.equal(rec["status"], f64["status"]) and torch.equal(rec["sign"], f64["sign"])
    assert ((rec["logpsi"] - f64["logpsi"]).abs() / f64["logpsi"].abs()).max().item() < 1e-12
    assert (rec["dinv"] - f64["dinv"]).abs().max().item() <= 1e-10 * f64["dinv"].abs().max().item()
    assert ((rec["e_loc"] - f64["e_loc"]).abs() / f64["e_loc"].abs()).max().item() < 1e-5


def test_singular_walker_decided_in_fp64(sysq):
    s, q = sysq
    R = make_walkers(s, 6, first=99)
    R[2, 7] = [2e3, 0.0, 0.0]                    # alpha electron without AOs: exactly singular Det_up
    R[4, s.n_up + 3] = [0.0, 2e3, 0.0]           # beta electron without AOs
    q.set_tiles(a4_mode="float_float", a4_kappa_max=1e8)
    o = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    st = o["status"].cpu().numpy()
    assert st[2] == 1 and st[4] == 2 and (st[[0, 1, 3, 5]] == 0).all()
    lp = o["logpsi"].cpu().numpy()
    assert lp[2] == -np.inf and lp[4] == -np.inf
