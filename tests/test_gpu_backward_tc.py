"""a7 on the tensor cores (qmc_logpsi_backward_ex, precision mixed) against
the FP64 adjoint (itself pinned to the oracle and to central differences) and
the oracle: D^-1 rounded to FP32 and g_w chi_mu in FP32, both split exactly
into three BF16 slices, six slice products per pair in FP32, blocks of
walkers (qmc_tiles.bw_walkers, 8 by default) summed in FP64.  Each term
carries a relative error of a few 2^-24 (D^-1, g and chi in FP32 cost ~1e-7 normwise), and each MMA rounds the FP32
accumulator: that accumulation dominates (measured 0.4-1.2e-5 normwise at 8
walkers per CTA, 2-4x more at 32).  The bar below is normwise,
max |dA - dA_ref| <= 5e-5 max |dA_ref|; a dropped slice product (2^-8) or a
misplaced AO row or D^-1 row (O(1)) is far above it.
Covers ragged walker blocks, several passes through a small workspace
(bit-identical to one pass), failed walkers (g_w = 0, D^-1 not finite),
the open-shell 1731-electron system (64-AO blocks, seven MO tiles) and W = 0."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)
TOL = 5e-5


def _rel(got, ref):
    ref = ref.cpu().numpy() if torch.is_tensor(ref) else ref
    got = got.cpu().numpy() if torch.is_tensor(got) else got
    den = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (den if den > 0 else 1.0))


def _setup(key, W, first, weighting="eloc"):
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system(key)
    q = QmcSystem(s, 0)
    R = torch.from_numpy(make_walkers(s, W, first=first)).to(dev)
    out = q.eval(R, precision="mixed", want_dinv=True)
    el = out["e_loc"]
    g = torch.full((W,), 1.0 / W, dtype=torch.float64, device=dev) if weighting == "plain" else \
        (2.0 * (el - el.mean()) / W).contiguous()
    g = torch.where(out["status"] == 0, g, torch.zeros_like(g))
    return s, q, R, out, g


@pytest.mark.parametrize("key,W,weighting", [("158e", 70, "plain"), ("158e", 70, "eloc"), ("434e", 40, "eloc")])
def test_mixed_adjoint_vs_fp64(key, W, weighting):
    s, q, R, out, g = _setup(key, W, 410, weighting)
    f_up, f_dn = q.backward(R, out["dinv"], g, precision="f64")
    m_up, m_dn = q.backward(R, out["dinv"], g, precision="mixed")
    e_up, e_dn = _rel(m_up, f_up), _rel(m_dn, f_dn)
    print(f"{key} W={W} {weighting}: normwise rel err up {e_up:.3e} dn {e_dn:.3e}")
    assert e_up <= TOL and e_dn <= TOL


def test_mixed_adjoint_vs_oracle():
    s, q, R, out, g = _setup("158e", 12, 420, "eloc")
    ru, rd = Oracle(s).logpsi_grad(R.cpu().numpy(), g.cpu().numpy())
    m_up, m_dn = q.backward(R, out["dinv"], g, precision="mixed")
    assert _rel(m_up, ru) <= TOL and _rel(m_dn, rd) <= TOL


def test_passes_through_small_workspace_are_bit_identical():
    s, q, R, out, g = _setup("158e", 70, 430, "eloc")
    one_up, one_dn = q.backward(R, out["dinv"], g, precision="mixed")
    ws = torch.empty(q.backward_workspace_size(32, "mixed"), dtype=torch.uint8, device=dev)
    ch_up, ch_dn = q.backward(R, out["dinv"], g, precision="mixed", ws=ws)   # passes of 32, 32, 6 walkers
    assert torch.equal(one_up, ch_up) and torch.equal(one_dn, ch_dn)


def test_failed_walker_is_skipped():
    s, q, R, out, g = _setup("158e", 40, 440, "eloc")
    g = g.clone()
    g[5] = 0.0
    ref_up, ref_dn = q.backward(R, out["dinv"], g, precision="mixed")
    dinv = out["dinv"].clone()
    dinv[5] = float("nan")
    got_up, got_dn = q.backward(R, dinv, g, precision="mixed")
    assert torch.equal(ref_up, got_up) and torch.equal(ref_dn, got_dn)
    assert torch.isfinite(got_up).all() and torch.isfinite(got_dn).all()


def test_open_shell_1731e():
    s, q, R, out, g = _setup("1731e", 6, 450, "eloc")
    f_up, f_dn = q.backward(R, out["dinv"], g, precision="f64")
    m_up, m_dn = q.backward(R, out["dinv"], g, precision="mixed")
    e_up, e_dn = _rel(m_up, f_up), _rel(m_dn, f_dn)
    print(f"1731e W=6: normwise rel err up {e_up:.3e} dn {e_dn:.3e}")
    assert e_up <= TOL and e_dn <= TOL


def test_no_walkers_gives_zero():
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("158e")
    q = QmcSystem(s, 0)
    R = torch.empty(0, s.n_up + s.n_dn, 3, dtype=torch.float64, device=dev)
    dinv = torch.empty(0, s.n_up ** 2 + s.n_dn ** 2, dtype=torch.float64, device=dev)
    g = torch.empty(0, dtype=torch.float64, device=dev)
    up, dn = q.backward(R, dinv, g, precision="mixed", ws=torch.empty(256, dtype=torch.uint8, device=dev))
    assert (up == 0).all() and (dn == 0).all()


def test_walkers_per_cta_tile():
    s, q, R, out, g = _setup("434e", 40, 460, "plain")
    f_up, f_dn = q.backward(R, out["dinv"], g, precision="f64")
    errs = {}
    try:
        for wb in (2, 32):
            q.set_tiles(bw_walkers=wb)
            assert q.tiles()["bw_walkers"] == wb
            m_up, m_dn = q.backward(R, out["dinv"], g, precision="mixed")
            errs[wb] = max(_rel(m_up, f_up), _rel(m_dn, f_dn))
    finally:
        q.set_tiles(bw_walkers=8)
    print("434e plain, normwise rel err by walkers per CTA:", errs)
    assert max(errs.values()) <= TOL
