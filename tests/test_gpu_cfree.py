"""The C-free variant (c15_mode = cfree): only C1 is formed; after a4 the
drift and the Laplacian come from v_e = D^-1[e,:] A^T (Sec. II.C vector
products with the MO expansion, Eq. mo): drift_e = sum_mu v_e,mu grad chi_mu,
lap_e = sum_mu v_e,mu lap chi_mu.  Checked against the FP64 oracle at the
mixed path's bars (log|Psi| 1e-6 absolute, E_L 1e-5 relative; drift 1e-5
normwise, tighter than the C2..C4 products reach), with ragged walker tiles,
open shells, singular and non-finite walkers, and against the tensor-core
mode on the GPU."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers, tiny_system

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


def _q(s):
    from paper_1209_6630_gb300 import QmcSystem
    return QmcSystem(s, 0)


@pytest.mark.parametrize("key,W", [("158e", 130), ("434e", 40), ("1056e", 140), ("1731e", 24)])
def test_cfree_vs_oracle(key, W):
    s = config_system(key)
    q = _q(s)
    R = make_walkers(s, W, first=40000)
    q.set_tiles(c15_mode="cfree")
    got = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    g = {k: v.cpu().numpy() for k, v in got.items()}
    sample = np.unique(np.linspace(0, W - 1, min(W, 12)).astype(int))
    ref = Oracle(s).eval(R[sample], nthreads=8)
    np.testing.assert_array_equal(g["status"][sample], ref["status"])
    d_lp = np.abs(g["logpsi"][sample] - ref["logpsi"]).max()
    d_el = (np.abs(g["e_loc"][sample] - ref["e_loc"]) / np.abs(ref["e_loc"])).max()
    d_dr = (np.abs(g["drift"][sample] - ref["drift"]).max(axis=(1, 2)) /
            np.abs(ref["drift"]).max(axis=(1, 2))).max()
    d_T = (np.abs(g["e_parts"][sample, 0] - ref["e_parts"][:, 0]) / np.abs(ref["e_parts"][:, 0])).max()
    print(f"{key}: |dlogpsi| {d_lp:.2e}, E_L rel {d_el:.2e}, drift normwise {d_dr:.2e}, T rel {d_T:.2e}")
    assert d_lp < 1e-6
    assert d_el < 1e-5
    assert d_dr < 1e-5


def test_cfree_matches_tensor_mode_on_gpu():
    s = config_system("434e")
    q = _q(s)
    Rd = torch.from_numpy(make_walkers(s, 300, first=41000)).to(dev)
    q.set_tiles(c15_mode="tensor")
    a = q.eval(Rd, precision="mixed")
    q.set_tiles(c15_mode="cfree")
    b = q.eval(Rd, precision="mixed")
    assert torch.equal(a["status"], b["status"])
    assert torch.equal(a["logpsi"], b["logpsi"])          # C1 and a4 are the same kernels
    assert ((a["e_loc"] - b["e_loc"]).abs() / b["e_loc"].abs()).max().item() < 1e-5
    assert ((a["drift"] - b["drift"]).abs().amax(dim=(1, 2)) / b["drift"].abs().amax(dim=(1, 2))).max().item() < 1e-4


def test_cfree_open_shell_and_edge_walkers():
    s = tiny_system("mini_chain")                          # 20 up / 19 down, separate MO matrices
    q = _q(s)
    q.set_tiles(c15_mode="cfree")
    R = make_walkers(s, 6)
    R[2, 3] = [2e3, 0, 0]                                  # an up electron with no AO: singular Det_up
    R[4, 30] = [np.nan, 0.0, 0.0]                           # a non-finite coordinate
    got = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    ref = Oracle(s).eval(R)
    g = {k: v.cpu().numpy() for k, v in got.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    ok = ref["status"] == 0
    assert np.abs(g["logpsi"][ok] - ref["logpsi"][ok]).max() < 1e-6
    assert (np.abs(g["e_loc"][ok] - ref["e_loc"][ok]) / np.abs(ref["e_loc"][ok])).max() < 1e-5
    assert g["logpsi"][2] == -np.inf
