"""GPU parity of the plain FP64 path against the FP64 CPU oracle, through
the C ABI.  Bars: screening lists and radii bit-exact; FP64 path log|Psi|
and E_L within 1e-10 relative; the other FP64 results within tolerances
derived from FP64 rounding (see each assert)."""
import numpy as np
import pytest
import torch

from oracle import Oracle, lu_inverse
from synth import config_system, make_walkers, tiny_system
from tests.helpers import one_atom_system

pytestmark = pytest.mark.gpu

dev = torch.device("cuda", 0)


def _q(system):
    from paper_1209_6630_gb300 import QmcSystem
    return QmcSystem(system, 0)


def _rowwise_rel(a, b):
    """max over rows of max|a-b| / max|b| (normwise per row)."""
    a, b = np.asarray(a), np.asarray(b)
    den = np.abs(b).max(axis=-1, keepdims=True)
    den = np.where(den == 0, 1.0, den)
    return float((np.abs(a - b) / den).max())


@pytest.fixture(scope="module")
def sys158():
    s = config_system("158e")
    return s, Oracle(s), _q(s)


@pytest.fixture(scope="module")
def sys434():
    s = config_system("434e")
    return s, Oracle(s), _q(s)


@pytest.mark.parametrize("key", ["158e", "434e", "1056e"])
def test_shell_radii_bit_exact(key):
    s = config_system(key)
    assert np.array_equal(_q(s).shell_r2(), Oracle(s).R2)


@pytest.mark.parametrize("which", ["sys158", "sys434"])
def test_screening_lists_bit_exact_and_ao_values(which, request):
    s, o, q = request.getfixturevalue(which)
    W = 6
    R = make_walkers(s, W, first=500)
    # a few electrons far away (empty lists) and one exactly on a nucleus
    R[0, 3] = [500.0, 0.0, 0.0]
    R[1, 2] = s.Q[0]
    cap = s.n_ao
    cnt, idx, B = q.screen_ao(torch.from_numpy(R).to(dev), cap)
    cnt, idx, B = cnt.cpu().numpy(), idx.cpu().numpy(), B.cpu().numpy()
    for w in range(W):
        d = o.eval_debug(R[w])
        np.testing.assert_array_equal(cnt[w], d["cnt"])
        for e in range(s.n_elec):
            K = d["cnt"][e]
            np.testing.assert_array_equal(idx[w, e, :K], d["idx"][e, :K])
            if K:
                # FP64, different but equivalent formula: agreement to ~1e-13 of the row scale
                assert _rowwise_rel(B[w, e, :, :K], d["B"][e, :, :K]) < 1e-12
    assert cnt[0, 3] == 0


def test_slater_matrices_f64(sys158):
    s, o, q = sys158
    R = make_walkers(s, 5, first=40)
    up, dn = q.slater(torch.from_numpy(R).to(dev))
    up, dn = up.cpu().numpy(), dn.cpu().numpy()
    for w in range(5):
        d = o.eval_debug(R[w])
        # sums of ~130 FP64 products in another order: 1e-13 of the row scale
        assert _rowwise_rel(up[w], d["C_up"]) < 1e-12
        assert _rowwise_rel(dn[w], d["C_dn"]) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 7, 16, 17, 33, 79, 130, 217, 528])
def test_det_inverse_vs_oracle(n):
    from paper_1209_6630_gb300 import det_inverse
    rng = np.random.default_rng(n)
    b = 3
    M = rng.normal(size=(b, n, n))
    la, sg, Dinv, sing = det_inverse(torch.from_numpy(M.copy()).to(dev))
    la, sg, Dinv, sing = la.cpu().numpy(), sg.cpu().numpy(), Dinv.cpu().numpy(), sing.cpu().numpy()
    for i in range(b):
        la_o, sg_o, inv_o = lu_inverse(M[i])
        assert sing[i] == 0 and sg[i] == sg_o
        assert abs(la[i] - la_o) <= 1e-11 * max(1.0, abs(la_o))
        # Dinv = M^-T; FP64 inverse of a Gaussian matrix: error ~ n * kappa * 1e-16
        kappa = np.linalg.cond(M[i])
        assert np.abs(Dinv[i] - inv_o.T).max() <= 1e-15 * n * kappa * np.abs(inv_o).max() * 10


def test_det_inverse_singular_and_nan():
    from paper_1209_6630_gb300 import det_inverse
    rng = np.random.default_rng(0)
    M = rng.normal(size=(3, 20, 20))
    M[1, 7, :] = 0.0            # exact zero row: exact zero pivot
    M[2, 3, 3] = np.nan
    la, sg, Dinv, sing = det_inverse(torch.from_numpy(M.copy()).to(dev))
    la, sg, Dinv, sing = la.cpu().numpy(), sg.cpu().numpy(), Dinv.cpu().numpy(), sing.cpu().numpy()
    assert sing[0] == 0 and np.isfinite(Dinv[0]).all()
    assert sing[1] == 1 and la[1] == -np.inf and sg[1] == 0 and np.isnan(Dinv[1]).all()
    assert sing[2] == 1 or not np.isfinite(la[2])


def _check_eval(s, o, q, R, tol_rel=1e-10):
    out = q.eval(torch.from_numpy(R).to(dev), want_dinv=True)
    ref = o.eval(R, want_dinv=True)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(g["status"], ref["status"])
    ok = ref["status"] == 0
    np.testing.assert_array_equal(g["sign"], ref["sign"])
    rel = np.abs(g["logpsi"][ok] - ref["logpsi"][ok]) / np.abs(ref["logpsi"][ok])
    assert rel.max() < tol_rel
    rel = np.abs(g["e_loc"][ok] - ref["e_loc"][ok]) / np.abs(ref["e_loc"][ok])
    assert rel.max() < tol_rel
    np.testing.assert_allclose(g["e_parts"][ok][:, 1:], ref["e_parts"][ok][:, 1:], rtol=1e-12)
    # drift: FP64, normwise per walker
    dr = np.abs(g["drift"][ok] - ref["drift"][ok]).max(axis=(1, 2)) / np.abs(ref["drift"][ok]).max(axis=(1, 2))
    assert dr.max() < 1e-9
    nu2 = s.n_up ** 2
    dinv_ref = np.concatenate([ref["dinv_up"].reshape(len(R), -1), ref["dinv_dn"].reshape(len(R), -1)], 1)
    assert _rowwise_rel(g["dinv"][ok], dinv_ref[ok]) < 1e-8
    return g, ref


def test_eval_f64_158e_full_config(sys158):
    s, o, q = sys158
    R = make_walkers(s, 100)        # the 158-electron workload: 100 walkers
    _check_eval(s, o, q, R)


def test_eval_f64_434e_sample(sys434):
    s, o, q = sys434
    R = make_walkers(s, 12, first=7)
    _check_eval(s, o, q, R)


def test_eval_edge_cases(sys158):
    s, o, q = sys158
    R = make_walkers(s, 4, first=900)
    R[1, 5] = [1e3, 0, 0]                   # alpha electron with no AO: exactly singular Det_up
    R[2, s.n_up + 4] = [0, 1e3, 0]          # beta electron with no AO: exactly singular Det_dn
    R[3, 0, 0] = np.nan                     # non-finite input
    out = q.eval(torch.from_numpy(R).to(dev))
    st = out["status"].cpu().numpy()
    assert st[0] == 0
    assert st[1] & 1 and not st[1] & 2
    assert st[2] & 2 and not st[2] & 1
    assert st[3] & 4
    lp = out["logpsi"].cpu().numpy()
    assert lp[1] == -np.inf and lp[2] == -np.inf
    assert out["sign"].cpu().numpy()[1] == 0
    ref = o.eval(R[:1])
    assert abs(lp[0] - ref["logpsi"][0]) < 1e-10 * abs(ref["logpsi"][0])
    # zero walkers is a no-op
    empty = q.eval(torch.empty(0, s.n_elec, 3, dtype=torch.float64, device=dev))
    assert empty["logpsi"].numel() == 0


def test_eval_one_electron_and_open_shell():
    gam = 0.9
    s = one_atom_system(1.0, [(0, [gam], [1.0])], n_up=1, n_dn=0, A_up=[[1.0]])
    q, o = _q(s), Oracle(s)
    R = np.random.default_rng(3).normal(size=(7, 1, 3))
    g, ref = _check_eval(s, o, q, R)
    r2 = (R[:, 0] ** 2).sum(1)
    np.testing.assert_allclose(g["e_loc"], 3 * gam - 2 * gam ** 2 * r2 - 1 / np.sqrt(r2), rtol=1e-12)
    s2 = tiny_system("h2o_like")
    s2 = type(s2)(**{**s2.__dict__})
    # open shell: move one electron from beta to alpha (6 up, 4 down) with a separate MO matrix
    rng = np.random.default_rng(4)
    A_up, _ = np.linalg.qr(rng.normal(size=(s2.n_ao, 6)))
    A_dn, _ = np.linalg.qr(rng.normal(size=(s2.n_ao, 4)))
    s2.n_up, s2.n_dn, s2.A_up, s2.A_dn = 6, 4, A_up, A_dn
    _check_eval(s2, Oracle(s2), _q(s2), make_walkers(s2, 9))


def test_workspace_chunking(sys158):
    s, o, q = sys158
    R = torch.from_numpy(make_walkers(s, 10)).to(dev)
    full = q.eval(R)
    ws = torch.empty(q.workspace_size(3), dtype=torch.uint8, device=dev)   # 3 walkers per chunk
    part = q.eval(R, ws=ws)
    for k in ("logpsi", "e_loc", "drift"):
        assert torch.equal(full[k], part[k])
    from paper_1209_6630_gb300 import QmcError
    with pytest.raises(QmcError):
        q.eval(R, ws=torch.empty(16, dtype=torch.uint8, device=dev))


@pytest.mark.parametrize("weighting", ["plain", "eloc"])
def test_backward_f64_vs_oracle(weighting):
    s = tiny_system("mini_chain")
    o, q = Oracle(s), _q(s)
    W = 40
    R = make_walkers(s, W)
    ref = o.eval(R)
    g = np.full(W, 1.0 / W) if weighting == "plain" else 2 * (ref["e_loc"] - ref["e_loc"].mean()) / W
    out = q.eval(torch.from_numpy(R).to(dev), want_dinv=True)
    dA_up, dA_dn = q.backward(torch.from_numpy(R).to(dev), out["dinv"], torch.from_numpy(g).to(dev))
    ru, rd = o.logpsi_grad(R, g)
    for got, exp in ((dA_up, ru), (dA_dn, rd)):
        got = got.cpu().numpy()
        assert np.abs(got - exp).max() <= 1e-10 * np.abs(exp).max()


def test_autograd_function_matches_backward():
    from paper_1209_6630_gb300 import LogPsi
    s = tiny_system("mini_chain")
    q = _q(s)
    W = 16
    R = torch.from_numpy(make_walkers(s, W)).to(dev)
    A_up = torch.tensor(s.A_up, device=dev, requires_grad=True)
    A_dn = torch.tensor(s.A_dn, device=dev, requires_grad=True)
    lp, el = LogPsi.apply(A_up, A_dn, R, q)
    lp.mean().backward()
    ru, rd = Oracle(s).logpsi_grad(R.cpu().numpy(), np.full(W, 1.0 / W))
    assert np.abs(A_up.grad.cpu().numpy() - ru).max() <= 1e-10 * np.abs(ru).max()
    assert np.abs(A_dn.grad.cpu().numpy() - rd).max() <= 1e-10 * np.abs(rd).max()
