"""The mixed-precision path against the FP64 CPU oracle at the sizes the
benchmark times, element by element (Sec. II.C: the Slater matrix and its
gradient and Laplacian companions; Sec. III Eq. "abc": the five products).

* 1056 electrons with 1024 walkers in one call: eight walker tiles of 128 and
  electron batches of 64, the tiling of the timed batch.  All five Slater
  matrices (C1, C5 to 1e-9, C2..C4 to 1e-5 row-normwise), log|Psi| (1e-6
  absolute) and E_L (1e-5 relative) on walkers spread over the tiles plus the
  three worst-conditioned walkers of the batch (largest ||D^-1||_inf from the
  FP64 path: the near-node walkers whose matrices the FP64 recomputation
  takes over).  The whole batch's log|Psi| against the FP64 GPU path.
* The gradient matrices C2..C4 at 434 and 1731 electrons, for both split
  precisions (FP16 hi/lo to 1e-5; BF16 hi/lo to 5e-5, what 8 + 8 bits reach).
* The mixed batch of the four systems (1731 electrons included) in one CUDA
  graph launch, each segment's first and last walker against the oracle.
"""
from concurrent.futures import ThreadPoolExecutor

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


def _debug_many(o, R, idx):
    with ThreadPoolExecutor(max_workers=len(idx)) as ex:
        return dict(zip(idx, ex.map(lambda w: o.eval_debug(R[w]), idx)))


def _slater_errors(up, dn, refs):
    ff, grad = 0.0, 0.0
    for w, d in refs.items():
        for got, ref in ((up[w], d["C_up"]), (dn[w], d["C_dn"])):
            ff = max(ff, _rowwise_rel(got[0], ref[0]), _rowwise_rel(got[4], ref[4]))
            grad = max(grad, max(_rowwise_rel(got[l], ref[l]) for l in (1, 2, 3)))
    return ff, grad


def test_1056e_1024_walkers_vs_oracle():
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("1056e")
    q = QmcSystem(s, 0)
    W = 1024
    R = make_walkers(s, W, first=20000)
    Rd = torch.from_numpy(R).to(dev)
    mx = q.eval(Rd, precision="mixed")
    f64 = q.eval(Rd, precision="f64", want_dinv=True)
    # the whole batch against the FP64 GPU path
    ok = (mx["status"] == 0) & (f64["status"] == 0)
    assert torch.equal(mx["status"], f64["status"])
    assert (mx["logpsi"] - f64["logpsi"]).abs()[ok].max().item() <= 1e-6
    # conditioning proxy from the FP64 inverse: ||D^-1||_inf per walker (max over spins)
    nu = s.n_up
    di = f64["dinv"]
    n_up_inf = di[:, : nu * nu].reshape(W, nu, nu).abs().sum(dim=2).amax(dim=1)
    n_dn_inf = di[:, nu * nu:].reshape(W, s.n_dn, s.n_dn).abs().sum(dim=2).amax(dim=1)
    worst = torch.argsort(torch.maximum(n_up_inf, n_dn_inf), descending=True)[:3].cpu().tolist()
    del f64, di
    q._ws.pop("f64", None)
    torch.cuda.empty_cache()
    sample = sorted(set([0, 127, 128, 383, 640, 1023] + worst))
    up, dn = q.slater(Rd, precision="mixed")          # the same call's tiling: one chunk of 1024
    up = up[sample].cpu().numpy()
    dn = dn[sample].cpu().numpy()
    torch.cuda.empty_cache()
    o = Oracle(s)
    refs = _debug_many(o, R, sample)
    ff, grad = _slater_errors({w: u for w, u in zip(sample, up)}, {w: d for w, d in zip(sample, dn)}, refs)
    print(f"1056e x 1024: C1/C5 {ff:.2e}, C2..C4 {grad:.2e}, worst-conditioned walkers {worst}")
    assert ff < 1e-9, ff
    assert grad < 1e-5, grad
    g = {k: v.cpu().numpy() for k, v in mx.items()}
    for w, d in refs.items():
        assert g["status"][w] == d["status"]
        la = d["logabs"].sum()
        assert abs(g["logpsi"][w] - la) < 1e-6, (w, g["logpsi"][w], la)
        assert abs(g["e_loc"][w] - d["e_loc"]) < 1e-5 * abs(d["e_loc"]), (w, g["e_loc"][w], d["e_loc"])
        dr = np.abs(g["drift"][w] - d["drift"]).max() / np.abs(d["drift"]).max()
        assert dr < 1e-4, (w, dr)


@pytest.mark.parametrize("key", ["434e", "1731e"])
@pytest.mark.parametrize("prec,tol", [("mixed", 1e-5), ("mixed_bf16", 5e-5)])
def test_gradient_matrices_vs_oracle(key, prec, tol):
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system(key)
    q = QmcSystem(s, 0)
    W = 130                                            # two walker tiles, the second ragged
    R = make_walkers(s, W, first=21000)
    up, dn = q.slater(torch.from_numpy(R).to(dev), precision=prec)
    sample = [0, 77, 129]
    upn = {w: up[w].cpu().numpy() for w in sample}
    dnn = {w: dn[w].cpu().numpy() for w in sample}
    del up, dn
    q._ws.clear()
    torch.cuda.empty_cache()
    refs = _debug_many(Oracle(s), R, sample)
    ff, grad = _slater_errors(upn, dnn, refs)
    print(f"{key} {prec}: C1/C5 {ff:.2e}, C2..C4 {grad:.2e}")
    assert ff < 1e-9, ff
    assert grad < tol, grad


def test_mixed_batch_with_1731e_vs_oracle():
    from paper_1209_6630_gb300 import QmcBatch, QmcSystem
    spec = [("158e", 64), ("434e", 24), ("1056e", 130), ("1731e", 40)]
    parts, hosts, systems = [], [], []
    for i, (k, W) in enumerate(spec):
        s = config_system(k)
        Rh = make_walkers(s, W, first=22000 + i)
        parts.append((QmcSystem(s, 0), torch.from_numpy(Rh).to(dev)))
        hosts.append(Rh)
        systems.append(s)
    b = QmcBatch(parts, precision="mixed", graph=True)
    outs = b.launch()
    torch.cuda.synchronize()
    for (k, W), s, Rh, o in zip(spec, systems, hosts, outs):
        sample = [0, W - 1]
        ref = Oracle(s).eval(Rh[sample], nthreads=2)
        g = {kk: v.cpu().numpy()[sample] for kk, v in o.items()}
        np.testing.assert_array_equal(g["status"], ref["status"])
        assert np.abs(g["logpsi"] - ref["logpsi"]).max() < 1e-6, k
        assert (np.abs(g["e_loc"] - ref["e_loc"]) / np.abs(ref["e_loc"])).max() < 1e-5, k
