"""QMC_PREC_F64_TCA4: the plain FP64 path with a4 by the tensor-core
Gauss-Jordan (float-float panels, exact-slice rank-32 updates) and FP64
recomputation above f64_kappa_max -- the cheaper FP64-accurate a4 of the
inversion step (Sec. IV.B; Table 2 caption: inversion in double precision).
Held to the FP64 path's bar: log|Psi| and E_L within 1e-10 relative of the
FP64 path (same FP64 C1..C5; only the elimination differs), and of the
oracle."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.mark.parametrize("key,W", [("158e", 200), ("434e", 64), ("1056e", 64), ("1731e", 12)])
def test_f64_tca4_meets_fp64_bar(key, W):
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system(key)
    q = QmcSystem(s, 0)
    R = make_walkers(s, W, first=50000)
    Rd = torch.from_numpy(R).to(dev)
    f64 = q.eval(Rd, precision="f64", want_dinv=True)
    tc = q.eval(Rd, precision="f64_tca4", want_dinv=True)
    assert torch.equal(f64["status"], tc["status"]) and torch.equal(f64["sign"], tc["sign"])
    rlp = ((tc["logpsi"] - f64["logpsi"]).abs() / f64["logpsi"].abs()).max().item()
    rel = ((tc["e_loc"] - f64["e_loc"]).abs() / f64["e_loc"].abs()).max().item()
    rdi = ((tc["dinv"] - f64["dinv"]).abs().amax(dim=1) / f64["dinv"].abs().amax(dim=1)).max().item()
    print(f"{key}: log|Psi| rel {rlp:.2e}, E_L rel {rel:.2e}, D^-1 normwise {rdi:.2e}")
    assert rlp <= 1e-10 and rel <= 1e-10
    sample = [0, W - 1]
    ref = Oracle(s).eval(R[sample], nthreads=4)
    g = {k: v.cpu().numpy()[sample] for k, v in tc.items()}
    assert (np.abs(g["logpsi"] - ref["logpsi"]) / np.abs(ref["logpsi"])).max() <= 1e-10
    assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() <= 1e-10
