"""GPU parity of the mixed-precision path (tensor-core C2..C4, FP64-accurate
C1 and C5, FP64 inverse and energies) against the FP64 CPU oracle, through
the C ABI.

Bars (per result, against the oracle): Slater entries (all five matrices)
within 1e-5 relative, normwise per row; log|Psi| within 1e-6 absolute; E_L
within 1e-5 relative.  The BF16 split is checked against a looser bound that
documents what it reaches.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers, tiny_system

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


def _q(system):
    from paper_1209_6630_gb300 import QmcSystem
    return QmcSystem(system, 0)


def _rowwise_rel(a, b):
    den = np.abs(b).max(axis=-1, keepdims=True)
    den = np.where(den == 0, 1.0, den)
    return float((np.abs(a - b) / den).max())


@pytest.fixture(scope="module")
def sys158():
    s = config_system("158e")
    return s, Oracle(s), _q(s)


@pytest.mark.parametrize("prec,tol_d", [("mixed", 1e-5), ("mixed_bf16", 5e-5)])
def test_mixed_slater_matrices(sys158, prec, tol_d):
    s, o, q = sys158
    W = 130                                   # two walker tiles, the second ragged (2 of 128 rows)
    R = make_walkers(s, W, first=300)
    up, dn = q.slater(torch.from_numpy(R).to(dev), precision=prec)
    up, dn = up.cpu().numpy(), dn.cpu().numpy()
    worst_ff, worst_d = 0.0, 0.0
    for w in (0, 1, 64, 127, 128, 129):
        d = o.eval_debug(R[w])
        for got, ref in ((up[w], d["C_up"]), (dn[w], d["C_dn"])):
            worst_ff = max(worst_ff, _rowwise_rel(got[0], ref[0]), _rowwise_rel(got[4], ref[4]))
            worst_d = max(worst_d, max(_rowwise_rel(got[l], ref[l]) for l in range(1, 4)))
    # C1, C5: exact float-float accumulation (~3e-11 measured).  Bound derived from the
    # log|Psi| requirement: |dlog|det|| <= 1e-6 at kappa ~ 1e5 needs C1 to ~1e-9 row-normwise.
    assert worst_ff < 1e-9, worst_ff
    assert worst_d < tol_d, worst_d            # C2..C4: tensor-core split products


@pytest.mark.parametrize("key,W", [("158e", 100), ("434e", 40)])
def test_mixed_eval_vs_oracle(key, W):
    s = config_system(key)
    o, q = Oracle(s), _q(s)
    R = make_walkers(s, W, first=11)
    out = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    ref = o.eval(R)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["sign"], ref["sign"])
    assert np.abs(g["logpsi"] - ref["logpsi"]).max() < 1e-6
    assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5
    dr = np.abs(g["drift"] - ref["drift"]).max(axis=(1, 2)) / np.abs(ref["drift"]).max(axis=(1, 2))
    assert dr.max() < 1e-4


def test_mixed_open_shell_and_edge_walkers():
    s = tiny_system("mini_chain")            # 20 up / 19 down, separate MO matrices
    o, q = Oracle(s), _q(s)
    R = make_walkers(s, 5)
    R[2, 3] = [2e3, 0, 0]                    # an up electron with no AO: singular Det_up
    out = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    ref = o.eval(R)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    ok = ref["status"] == 0
    assert np.abs(g["logpsi"][ok] - ref["logpsi"][ok]).max() < 1e-6
    assert g["logpsi"][2] == -np.inf


def test_mixed_matches_f64_path_on_gpu(sys158):
    s, o, q = sys158
    R = torch.from_numpy(make_walkers(s, 64, first=77)).to(dev)
    a = q.eval(R, precision="mixed")
    b = q.eval(R, precision="f64")
    assert (a["logpsi"] - b["logpsi"]).abs().max().item() < 1e-6
    assert ((a["e_loc"] - b["e_loc"]).abs() / b["e_loc"].abs()).max().item() < 1e-5


@pytest.mark.parametrize("prec,tol_d", [("mixed", 1e-5), ("mixed_bf16", 5e-5)])
def test_float_float_c15_mode_vs_oracle(prec, tol_d):
    """The alternative C1/C5 arithmetic (c15_mode = float_float: float-float products for
    C1 and C5, C2..C4 by the separate tensor-core contraction), Slater entries and the
    evaluation against the oracle at the same bars."""
    s = config_system("158e")
    o, q = Oracle(s), _q(s)
    q.set_tiles(c15_mode="float_float")
    W = 130
    R = make_walkers(s, W, first=500)
    Rd = torch.from_numpy(R).to(dev)
    up, dn = q.slater(Rd, precision=prec)
    up, dn = up.cpu().numpy(), dn.cpu().numpy()
    worst_ff, worst_d = 0.0, 0.0
    for w in (0, 63, 127, 128, 129):
        d = o.eval_debug(R[w])
        for got, ref in ((up[w], d["C_up"]), (dn[w], d["C_dn"])):
            worst_ff = max(worst_ff, _rowwise_rel(got[0], ref[0]), _rowwise_rel(got[4], ref[4]))
            worst_d = max(worst_d, max(_rowwise_rel(got[l], ref[l]) for l in range(1, 4)))
    assert worst_ff < 1e-9, worst_ff
    assert worst_d < tol_d, worst_d
    out = q.eval(Rd, precision=prec)
    ref = o.eval(R)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["sign"], ref["sign"])
    assert np.abs(g["logpsi"] - ref["logpsi"]).max() < 1e-6
    assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5
