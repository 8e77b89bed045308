"""Bounded device waits of the tensor-core kernels, made to run out on
purpose (qmc_tiles.expire_walker: the chosen CTAs wait on a flag that nothing
sets, for qmc_tiles.wait_s).  The paper's rule for failures (Sec. V: a
failure loses only the block of work it hit) applied to one step:

* C1..C5: the CTA gives up, marks the walkers of its tile of 128 with
  QMC_STATUS_TIMEOUT, and every other walker of the batch is unchanged;
* a4 with tensor-core updates: the CTA gives up and hands its matrices to the
  FP64 recomputation, so the walker's log|Psi| and D^-1 are the FP64 path's;
* the tensor-core adjoint: the CTAs give up and leave NaN in exactly the rows
  of dA they owned; every other entry is unchanged.

No GPU fault and no hang: each wait ends after wait_s, the CTA waits (bounded)
for its own MMAs, frees its tensor memory and returns; the context stays
usable, which the last check of each test shows.
"""
import numpy as np
import pytest
import torch

from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)
TIMEOUT = 8


@pytest.fixture(scope="module")
def sysq():
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("158e")
    return s, QmcSystem(s, 0)


def _reset(q):
    q.set_tiles(wait_s=2.0, expire_walker=-1, expire_kernels=7, a4_mode="float_float", a4_kappa_max=1e7)


def test_c15_expired_wait_marks_its_tile_only(sysq):
    s, q = sysq
    assert q.tiles()["c15_mode"] in ("tensor", "cfree")      # both run the C1 MMA kernel with the hook
    W = 300                                         # tiles 0..127, 128..255, 256..299
    Rd = torch.from_numpy(make_walkers(s, W, first=4100)).to(dev)
    try:
        ref = q.eval(Rd, precision="mixed")
        q.set_tiles(wait_s=0.01, expire_walker=150, expire_kernels=1)  # a walker of tile 1, C1..C5
        got = q.eval(Rd, precision="mixed")
        torch.cuda.synchronize()
    finally:
        _reset(q)
    st = got["status"].cpu().numpy()
    flagged = (st & TIMEOUT) != 0
    assert flagged[128:256].all(), "every walker of the expired CTA's tile is marked"
    assert not flagged[:128].any() and not flagged[256:].any()
    keep = np.r_[0:128, 256:300]
    for k in ("logpsi", "e_loc", "drift", "sign", "status"):
        assert torch.equal(got[k][keep], ref[k][keep]), k
    again = q.eval(Rd, precision="mixed")            # the context is still usable
    for k in ("logpsi", "e_loc", "status"):
        assert torch.equal(again[k], ref[k]), k


def test_a4_tensor_expired_wait_recomputed_in_fp64(sysq):
    s, q = sysq
    W = 40
    Rd = torch.from_numpy(make_walkers(s, W, first=4200)).to(dev)
    f64 = q.eval(Rd, precision="f64", want_dinv=True)
    try:
        q.set_tiles(a4_mode="tensor", a4_kappa_max=1e30)   # no matrix flagged by its condition
        ref = q.eval(Rd, precision="mixed", want_dinv=True)
        q.set_tiles(wait_s=0.01, expire_walker=7, expire_kernels=2)
        got = q.eval(Rd, precision="mixed", want_dinv=True)
        torch.cuda.synchronize()
    finally:
        _reset(q)
    assert (got["status"].cpu().numpy() == 0).all()          # recovered: no walker lost
    # walker 7: both spin matrices went to the FP64 recomputation (FP64 C1 and elimination)
    assert abs(got["logpsi"][7].item() - f64["logpsi"][7].item()) <= 1e-12 * abs(f64["logpsi"][7].item())
    d7 = (got["dinv"][7] - f64["dinv"][7]).abs().max().item()
    assert d7 <= 1e-10 * f64["dinv"][7].abs().max().item()
    # the tensor-core result of walker 7 was not that close to FP64 (so the recomputation did happen)
    r7 = (ref["dinv"][7] - f64["dinv"][7]).abs().max().item()
    assert r7 > d7
    others = [w for w in range(W) if w != 7]
    for k in ("logpsi", "dinv", "e_loc"):
        assert torch.equal(got[k][others], ref[k][others]), k


def test_adjoint_expired_wait_leaves_nan_in_its_rows_only(sysq):
    s, q = sysq
    W = 32                                            # four blocks of 8 walkers
    Rd = torch.from_numpy(make_walkers(s, W, first=4300)).to(dev)
    o = q.eval(Rd, precision="mixed", want_dinv=True)
    el = o["e_loc"]
    g = (2.0 * (el - el.mean()) / W).contiguous()
    q.set_tiles(bw_walkers=8)
    try:
        ref_up, ref_dn = q.backward(Rd, o["dinv"], g, precision="mixed")
        q.set_tiles(wait_s=0.01, expire_walker=9, expire_kernels=4)   # spin-up CTAs of walkers 8..15
        got_up, got_dn = q.backward(Rd, o["dinv"], g, precision="mixed")
        torch.cuda.synchronize()
    finally:
        _reset(q)
    assert torch.equal(got_dn, ref_dn)                # spin down untouched
    nan_rows = torch.isnan(got_up).any(dim=1)
    assert nan_rows.any()
    assert torch.isnan(got_up[nan_rows]).all()        # a CTA owns whole rows (its AO block, every MO)
    ok = ~nan_rows
    assert torch.equal(got_up[ok], ref_up[ok])
    rows = torch.nonzero(nan_rows).flatten().cpu().numpy()
    # the expired CTAs' AO blocks: runs of consecutive AOs, each a run of whole atoms
    ao_atom = s.shell_atom[s.ao_shell]
    for r in rows:
        assert nan_rows[np.flatnonzero(ao_atom == ao_atom[r])].all()
    again_up, _ = q.backward(Rd, o["dinv"], g, precision="mixed")
    assert torch.equal(again_up, ref_up)
