"""Multi-determinant trial function on the GPU (qmc_multidet_eval; Sec. II.C,
Eq. psit: Psi = e^J sum_K c_K Det_K,up Det_K,dn) against the oracle's
combination of the same determinants: FP64 path to 1e-10 relative, mixed path
to the mixed bars; with the Jastrow factor; one nonzero coefficient gives that
determinant's own evaluation."""
import math

import numpy as np
import pytest
import torch

import oracle
from synth import config_system, excited_determinants, make_walkers, tiny_system

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)
JAS = dict(a_par=0.25, a_anti=0.5, b_ee=1.1, a_en=0.7, b_en=1.9)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
@pytest.mark.parametrize("jastrow", [False, True])
def test_multidet_vs_oracle(prec, jastrow):
    from paper_1209_6630_gb300 import QmcSystem, multidet_eval
    s = config_system("158e")
    dets = excited_determinants(s, 3)
    qs = [QmcSystem(d, 0) for d in dets]
    if jastrow:
        for q in qs:
            q.set_jastrow(JAS)
    coef = [1.0, 0.25, -0.15]
    W = 64
    R = make_walkers(s, W, first=70000)
    got = multidet_eval(qs, coef, torch.from_numpy(R).to(dev), precision=prec)
    g = {k: v.cpu().numpy() for k, v in got.items()}
    ref = oracle.multidet_eval([oracle.Oracle(d, jastrow=JAS if jastrow else None) for d in dets], coef, R,
                               nthreads=8)
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_array_equal(g["sign"], ref["sign"])
    d_lp = np.abs(g["logpsi"] - ref["logpsi"])
    d_el = np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])
    d_dr = np.abs(g["drift"] - ref["drift"]).max(axis=(1, 2)) / np.abs(ref["drift"]).max(axis=(1, 2))
    if prec == "f64":
        assert (d_lp / np.abs(ref["logpsi"])).max() < 1e-10
        assert d_el.max() < 1e-10 and d_dr.max() < 1e-10
    else:
        assert d_lp.max() < 1e-6 and d_el.max() < 1e-5 and d_dr.max() < 1e-4
    assert np.isnan(g["logabs"]).all()


def test_single_coefficient_matches_single_determinant():
    from paper_1209_6630_gb300 import QmcSystem, multidet_eval
    s = tiny_system("mini_chain")
    dets = excited_determinants(s, 2)
    qs = [QmcSystem(d, 0) for d in dets]
    Rd = torch.from_numpy(make_walkers(s, 16)).to(dev)
    got = multidet_eval(qs, [0.0, 3.0], Rd, precision="f64")
    ref = qs[1].eval(Rd, precision="f64")
    assert torch.allclose(got["logpsi"], ref["logpsi"] + math.log(3.0), rtol=1e-14, atol=0)
    assert torch.allclose(got["e_loc"], ref["e_loc"], rtol=1e-13, atol=0)
    assert torch.allclose(got["drift"], ref["drift"], rtol=1e-13, atol=1e-14)
