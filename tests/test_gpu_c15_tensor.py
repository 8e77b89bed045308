"""C1 and C5 on the tensor cores from exact BF16 slices (c15_mode = tensor)
against the oracle, at the bar of the float-float kernel: C1 and C5 within
1e-9 row-normwise (what |dlog|det|| <= 1e-6 needs at kappa ~ 1e5), log|Psi|
within 1e-6, E_L within 1e-5 relative.  Covers ragged walker tiles, the
open-shell system, and a union of more than 1024 AOs (accumulated in
chunks)."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


def _rowwise_rel(a, b):
    den = np.abs(b).max(axis=-1, keepdims=True)
    den = np.where(den == 0, 1.0, den)
    return float((np.abs(a - b) / den).max())


def _tensor_q(s):
    from paper_1209_6630_gb300 import QmcSystem
    q = QmcSystem(s, 0)
    q.set_tiles(c15_mode="tensor")
    return q


@pytest.mark.parametrize("key,W,rows", [("158e", 130, (0, 1, 64, 127, 128, 129)), ("434e", 40, (0, 17, 39))])
def test_tensor_c15_vs_oracle(key, W, rows):
    s = config_system(key)
    o, q = Oracle(s), _tensor_q(s)
    R = make_walkers(s, W, first=310)
    up, dn = q.slater(torch.from_numpy(R).to(dev), precision="mixed")
    up, dn = up.cpu().numpy(), dn.cpu().numpy()
    worst = 0.0
    for w in rows:
        d = o.eval_debug(R[w])
        for got, ref in ((up[w], d["C_up"]), (dn[w], d["C_dn"])):
            worst = max(worst, _rowwise_rel(got[0], ref[0]), _rowwise_rel(got[4], ref[4]))
    assert worst < 1e-9, worst


@pytest.mark.parametrize("key,W", [("158e", 60), ("434e", 24)])
def test_tensor_c15_eval_vs_oracle(key, W):
    s = config_system(key)
    o, q = Oracle(s), _tensor_q(s)
    R = make_walkers(s, W, first=320)
    g = q.eval(torch.from_numpy(R).to(dev), precision="mixed")
    ref = o.eval(R)
    g = {k: v.cpu().numpy() for k, v in g.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    assert np.abs(g["logpsi"] - ref["logpsi"]).max() < 1e-6
    assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5


def test_tensor_c15_union_above_1024_aos():
    """Electron 0 of each of 128 walkers on a different nucleus: the tile's
    union list exceeds 1024 AOs, so the exact accumulation runs in chunks."""
    s = config_system("1056e")
    o, q = Oracle(s), _tensor_q(s)
    W = 128
    R = make_walkers(s, W, first=330)
    atoms = np.linspace(0, s.n_atom - 1, W).astype(int)
    R[:, 0] = s.Q[atoms] + 0.05
    pts = R[:, 0]
    cnt, idx = o.screen_points(pts)
    union = np.unique(np.concatenate([idx[p, : cnt[p]] for p in range(W)]))
    assert len(union) > 1024, len(union)
    up, dn = q.slater(torch.from_numpy(R).to(dev), precision="mixed")
    up = up.cpu().numpy()
    worst = 0.0
    for w in (0, 5, 63, 127):
        d = o.eval_debug(R[w])
        worst = max(worst, _rowwise_rel(up[w, 0, 0], d["C_up"][0, 0]), _rowwise_rel(up[w, 4, 0], d["C_up"][4, 0]))
    assert worst < 1e-9, worst


def test_tensor_c15_open_shell_and_modes_agree():
    s = config_system("1731e")
    from paper_1209_6630_gb300 import QmcSystem
    q = QmcSystem(s, 0)
    R = torch.from_numpy(make_walkers(s, 6, first=340)).to(dev)
    ff = q.eval(R, precision="mixed")
    q.set_tiles(c15_mode="tensor")
    tc = q.eval(R, precision="mixed")
    assert torch.equal(ff["status"], tc["status"])
    assert (ff["logpsi"] - tc["logpsi"]).abs().max().item() < 1e-7
    assert ((ff["e_loc"] - tc["e_loc"]).abs() / tc["e_loc"].abs()).max().item() < 1e-7
