"""The Jastrow factor on the GPU (Psi_T = e^J Det_up Det_dn, Sec. II.C) against
the oracle with the same factor: FP64 path to 1e-10 relative, mixed paths
(tensor-core C1..C5, and the C-free variant) to the mixed bars; switching the
factor off restores the results bit for bit; its parameters enter the CRC-32
key."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers, tiny_system

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


def _jas(s):
    return dict(a_par=0.25, a_anti=0.5, b_ee=1.1, a_en=np.linspace(0.4, 1.2, s.n_atom),
                b_en=np.linspace(1.5, 2.5, s.n_atom))


@pytest.mark.parametrize("key,W", [("158e", 64), ("434e", 16)])
@pytest.mark.parametrize("mode", ["f64", "mixed", "cfree"])
def test_jastrow_vs_oracle(key, W, mode):
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system(key)
    q = QmcSystem(s, 0)
    jas = _jas(s)
    q.set_jastrow(jas)
    if mode == "cfree":
        q.set_tiles(c15_mode="cfree")
    R = make_walkers(s, W, first=60000)
    got = q.eval(torch.from_numpy(R).to(dev), precision="f64" if mode == "f64" else "mixed")
    g = {k: v.cpu().numpy() for k, v in got.items()}
    ref = Oracle(s, jastrow=jas).eval(R, nthreads=8)
    np.testing.assert_array_equal(g["status"], ref["status"])
    d_lp = np.abs(g["logpsi"] - ref["logpsi"])
    d_el = np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])
    d_dr = np.abs(g["drift"] - ref["drift"]).max(axis=(1, 2)) / np.abs(ref["drift"]).max(axis=(1, 2))
    if mode == "f64":
        assert (d_lp / np.abs(ref["logpsi"])).max() < 1e-10
        assert d_el.max() < 1e-10 and d_dr.max() < 1e-10
    else:
        assert d_lp.max() < 1e-6 and d_el.max() < 1e-5
        assert d_dr.max() < (1e-4 if mode == "mixed" else 1e-5)


def test_jastrow_off_restores_and_keys():
    from paper_1209_6630_gb300 import QmcSystem
    s = tiny_system("mini_chain")
    q = QmcSystem(s, 0)
    Rd = torch.from_numpy(make_walkers(s, 8)).to(dev)
    base = q.eval(Rd, precision="f64")
    k0 = q.crc32()
    q.set_jastrow(_jas(s))
    with_j = q.eval(Rd, precision="f64")
    k1 = q.crc32()
    assert k1 != k0
    assert (with_j["logpsi"] - base["logpsi"]).abs().min().item() > 1e-6
    q.set_jastrow(None)
    again = q.eval(Rd, precision="f64")
    assert q.crc32() == k0
    for k in ("logpsi", "e_loc", "drift"):
        assert torch.equal(again[k], base[k]), k
