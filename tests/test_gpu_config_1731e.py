"""The 1731-electron open-shell workload (866 up / 865 down electrons, 4985
AOs, FP32 MO coefficients): forward parity on sampled walkers against the
FP64 oracle, and the adjoint d log|Psi| / dA (plain and E_L-weighted) against
the oracle's analytic gradient and against central finite differences with
h = 1e-4 on 64 sampled coefficients (32 of A_up, 32 of A_dn), the objective
L = sum_w g_w log|Psi_w| evaluated by the FP64 GPU path with E_L frozen; the
same differences check the tensor-core adjoint of the mixed path.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def big():
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("1731e")
    assert s.A_up.dtype == np.float32 and s.n_up == 866 and s.n_dn == 865 and s.n_ao == 4985
    return s, QmcSystem(s, 0)


def test_forward_parity_sampled(big):
    s, q = big
    W = 256                                    # two tensor-core walker tiles
    R = make_walkers(s, W)
    Rd = torch.from_numpy(R).to(dev)
    sample = [0, 127, 200, 255]
    ref = Oracle(s).eval(R[sample], nthreads=0)
    for prec, tl, te in (("f64", 1e-10, 1e-10), ("mixed", 1e-6, 1e-5)):
        out = q.eval(Rd, precision=prec)
        lp = out["logpsi"].cpu().numpy()[sample]
        el = out["e_loc"].cpu().numpy()[sample]
        np.testing.assert_array_equal(out["status"].cpu().numpy()[sample], ref["status"])
        np.testing.assert_array_equal(out["sign"].cpu().numpy()[sample], ref["sign"])
        if prec == "f64":
            assert (np.abs(lp - ref["logpsi"]) / np.abs(ref["logpsi"])).max() < tl
        else:
            assert np.abs(lp - ref["logpsi"]).max() < tl
        assert (np.abs(el - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < te


def test_adjoint_vs_oracle_gradient(big):
    s, q = big
    W = 6
    R = make_walkers(s, W, first=40)
    Rd = torch.from_numpy(R).to(dev)
    out = q.eval(Rd, precision="f64", want_dinv=True)
    el = out["e_loc"].cpu().numpy()
    g = 2.0 * (el - el.mean()) / W                      # E_L-weighted
    dA_up, dA_dn = q.backward(Rd, out["dinv"], torch.from_numpy(g).to(dev))
    ru, rd = Oracle(s).logpsi_grad(R, g)
    for got, exp in ((dA_up, ru), (dA_dn, rd)):
        got = got.cpu().numpy()
        assert np.abs(got - exp).max() <= 1e-9 * np.abs(exp).max()


@pytest.mark.parametrize("weighting", ["plain", "eloc"])
def test_adjoint_vs_central_differences(big, weighting):
    s, q = big
    W = 8
    R = make_walkers(s, W, first=80)
    Rd = torch.from_numpy(R).to(dev)
    base = q.eval(Rd, precision="f64", want_dinv=True)
    el = base["e_loc"].cpu().numpy()
    g = np.full(W, 1.0 / W) if weighting == "plain" else 2.0 * (el - el.mean()) / W
    gd = torch.from_numpy(g).to(dev)
    dA_up, dA_dn = q.backward(Rd, base["dinv"], gd)
    dA = {"up": dA_up.cpu().numpy(), "dn": dA_dn.cpu().numpy()}
    mixed = q.eval(Rd, precision="mixed", want_dinv=True)
    mA_up, mA_dn = q.backward(Rd, mixed["dinv"], gd, precision="mixed")
    mA = {"up": mA_up.cpu().numpy(), "dn": mA_dn.cpu().numpy()}
    rng = np.random.default_rng(1731)
    h = 1e-4
    A = {"up": s.A_up.copy(), "dn": s.A_dn.copy()}
    errs, errs_m = [], []
    try:
        for spin in ("up", "dn"):
            for _ in range(32):
                mu = int(rng.integers(0, s.n_ao))
                k = int(rng.integers(0, A[spin].shape[1]))
                a0 = A[spin][mu, k]
                vals = []
                steps = []
                for sgn in (+1, -1):
                    A[spin][mu, k] = np.float32(a0 + sgn * h)
                    steps.append(float(A[spin][mu, k]) - float(a0))   # the step the FP32 matrix really took
                    q.set_mo(A["up"], A["dn"])
                    lp = q.eval(Rd, precision="f64")["logpsi"].cpu().numpy()
                    vals.append(float((g * lp).sum()))
                A[spin][mu, k] = a0
                fd = (vals[0] - vals[1]) / (steps[0] - steps[1])
                errs.append(abs(fd - dA[spin][mu, k]))
                errs_m.append(abs(fd - mA[spin][mu, k]))
    finally:
        q.set_mo(s.A_up, s.A_dn)
    scale = max(np.abs(dA["up"]).max(), np.abs(dA["dn"]).max())
    # FD truncation ~h^2 and FP64 rounding of L / h: well below 1e-6 of the gradient scale
    assert max(errs) <= 1e-6 * scale, (max(errs), scale)
    # the tensor-core adjoint: FP32 accumulation per block of walkers (normwise ~1e-5)
    assert max(errs_m) <= 5e-5 * scale, (max(errs_m), scale)
