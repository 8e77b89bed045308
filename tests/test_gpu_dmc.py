"""The Monte Carlo step on the GPU (Sec. II.A Eqs. 1-3 with the fixed-node
rule; Sec. II.B reconfiguration) through the C ABI, against the oracle:

* the reconfiguration's drawn indices bit-exact for the same weights (exact
  integer drawing), with dead and non-finite weights, ragged sizes, one
  walker, and all weights zero;
* the move to 1e-12 relative (the same Philox numbers; the GPU's and the C
  library's log / sin / cos may differ in the last bit);
* accept flags exact and weights to 1e-14 relative;
* whole steps (move, evaluation, weight, draw, copy) on the 158-electron
  system: drawn indices exact, positions and energies to the FP64 path's
  bounds, three steps in a row; the mixed path for one step;
* the same steps replayed from one captured CUDA graph, the step counter
  advanced on the device;
* physics: DMC of the hydrogen atom on the GPU projects to -1/2 Ha.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import one_atom_system
from synth import config_system, make_walkers

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.mark.parametrize("W", [1, 5, 1024, 2049, 5000])
def test_srmc_indices_bit_exact(W):
    from paper_1209_6630_gb300 import srmc_reconfigure
    rng = np.random.default_rng(W)
    w = np.exp(2.0 * rng.normal(size=W))
    if W > 4:
        w[rng.choice(W, size=W // 5, replace=False)] = 0.0
        w[1] = np.nan
        w[2] = -1.0
        w[3] = np.inf
    for step in (0, 7, 2 ** 40 + 3):
        idx, stats = srmc_reconfigure(torch.from_numpy(w).to(dev), seed=1234, step=step)
        ref, sw, alive, zero = oracle.srmc(w, 1234, step)
        np.testing.assert_array_equal(idx.cpu().numpy(), ref)
        st = stats.cpu().numpy()
        assert st[1] == alive
        assert abs(st[0] - sw) <= 1e-13 * sw
    idx, stats = srmc_reconfigure(torch.zeros(W, dtype=torch.float64, device=dev), seed=1, step=1)
    assert (idx.cpu().numpy() == np.arange(W)).all() and stats[1].item() == 0


def test_move_matches_oracle():
    from paper_1209_6630_gb300 import dmc_move
    W, N, tau = 300, 158, 0.013
    rng = np.random.default_rng(3)
    R = rng.normal(size=(W, N, 3)) * 4.0
    b = rng.normal(size=(W, N, 3)) * 10.0
    got = dmc_move(torch.from_numpy(R).to(dev), torch.from_numpy(b).to(dev), tau, seed=77, step=12).cpu().numpy()
    ref = oracle.dmc_move(R, b, tau, 77, 12)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the noise is the oracle's normal stream, walker by walker
    eta = (got - R - tau * b) / math.sqrt(tau)
    ref_eta = oracle.move_normals(W, 3 * N, 77, 12)
    assert np.abs(eta.reshape(W, -1) - ref_eta).max() < 1e-9


def test_weight_matches_oracle():
    from paper_1209_6630_gb300 import dmc_weight
    W, tau, eT = 4097, 0.02, -310.0
    rng = np.random.default_rng(5)
    e_old = eT + rng.normal(size=W) * 20
    e_new = eT + rng.normal(size=W) * 20
    s_old = rng.choice([-1.0, 1.0], size=W)
    s_new = np.where(rng.random(W) < 0.1, -s_old, s_old)
    st_old = np.where(rng.random(W) < 0.03, 4, 0).astype(np.int32)
    st_new = np.where(rng.random(W) < 0.03, 1, 0).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    w, acc = dmc_weight(t(e_old), t(s_old), t(st_old), t(e_new), t(s_new), t(st_new), tau, eT)
    rw, racc = oracle.dmc_weight(e_old, s_old, st_old.astype(np.uint32), e_new, s_new, st_new.astype(np.uint32),
                                 tau, eT)
    np.testing.assert_array_equal(acc.cpu().numpy(), racc.astype(np.int32))
    w = w.cpu().numpy()
    assert np.all((rw == 0) == (w == 0))
    nz = rw > 0
    assert np.abs(w[nz] - rw[nz]).max() <= 1e-14 * np.abs(rw[nz]).max()
    assert (np.abs(w[nz] - rw[nz]) / rw[nz]).max() < 1e-14


def _state_from_oracle(ev, R):
    return {"R": R.copy(), "drift": ev["drift"], "e_loc": ev["e_loc"], "logpsi": ev["logpsi"], "sign": ev["sign"],
            "status": ev["status"]}


def _to_dev(st):
    out = {}
    for k, v in st.items():
        a = np.ascontiguousarray(v)
        out[k] = torch.from_numpy(a.astype(np.int32) if k == "status" else a.astype(np.float64)).to(dev)
    return out


@pytest.fixture(scope="module")
def sys158():
    from paper_1209_6630_gb300 import QmcSystem
    s = config_system("158e")
    return s, oracle.Oracle(s), QmcSystem(s, 0)


def test_dmc_steps_fp64_vs_oracle(sys158):
    s, o, q = sys158
    W, tau, eT, seed = 64, 0.01, -300.0, 99
    R = make_walkers(s, W, first=30000)
    st_o = _state_from_oracle(o.eval(R), R)
    st_g = q.init_state(torch.from_numpy(R).to(dev), precision="f64")
    nxt = q.walker_state(W)
    stats = torch.zeros(4, dtype=torch.float64, device=dev)
    for step in range(3):
        st_o, info = oracle.dmc_step(o, st_o, tau, eT, seed, step)
        q.dmc_step(st_g, nxt, tau, eT, seed, step, precision="f64", stats=stats)
        st_g, nxt = nxt, st_g
        g = {k: v.cpu().numpy() for k, v in st_g.items()}
        np.testing.assert_array_equal(g["status"], st_o["status"].astype(np.int32))
        np.testing.assert_array_equal(g["sign"], st_o["sign"])
        assert np.abs(g["R"] - st_o["R"]).max() <= 1e-12 * np.abs(st_o["R"]).max(), step
        assert np.abs(g["logpsi"] - st_o["logpsi"]).max() <= 1e-10 * np.abs(st_o["logpsi"]).max()
        assert (np.abs(g["e_loc"] - st_o["e_loc"]) / np.abs(st_o["e_loc"])).max() <= 1e-9
        sv = stats.cpu().numpy()
        assert sv[1] == info["alive"] and sv[3] == info["accept"].sum()
        # the weights carry E_L's 1e-12 relative differences amplified by tau |E_L| / 2
        assert abs(sv[0] - info["sum_w"]) <= 1e-10 * info["sum_w"]
        assert abs(sv[2] - info["sum_w_eloc"]) <= 1e-9 * abs(info["sum_w_eloc"])


def test_dmc_step_mixed_vs_oracle(sys158):
    s, o, q = sys158
    W, tau, eT, seed = 256, 0.01, -300.0, 5
    R = make_walkers(s, W, first=31000)
    ev = o.eval(R)
    st_o, info = oracle.dmc_step(o, _state_from_oracle(ev, R), tau, eT, seed, 0)
    st_g = _to_dev(_state_from_oracle(ev, R))
    nxt = q.walker_state(W)
    q.dmc_step(st_g, nxt, tau, eT, seed, 0, precision="mixed")
    g = {k: v.cpu().numpy() for k, v in nxt.items()}
    np.testing.assert_array_equal(g["status"], st_o["status"].astype(np.int32))
    # the mixed drift (1e-4 normwise) moves the positions by tau * 1e-4 |b|
    assert np.abs(g["R"] - st_o["R"]).max() <= 1e-5 * np.abs(st_o["R"]).max()
    assert np.abs(g["logpsi"] - st_o["logpsi"]).max() < 1e-4
    assert (np.abs(g["e_loc"] - st_o["e_loc"]) / np.abs(st_o["e_loc"])).max() < 1e-4


def test_dmc_steps_in_one_cuda_graph(sys158):
    s, o, q = sys158
    W, tau, eT, seed = 96, 0.01, -300.0, 31
    R = torch.from_numpy(make_walkers(s, W, first=32000)).to(dev)
    a = q.init_state(R, precision="f64")
    b = q.walker_state(W)
    ref_a = {k: v.clone() for k, v in a.items()}
    ref_b = q.walker_state(W)
    # explicit steps 0..3
    for step in range(4):
        q.dmc_step(ref_a, ref_b, tau, eT, seed, step, precision="f64")
        ref_a, ref_b = ref_b, ref_a
    # two steps (a -> b -> a) captured once, replayed twice, the counter on the device
    step_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(q.dmc_workspace_size(W, "f64"), dtype=torch.uint8, device=dev)
    q.dmc_step(a, b, tau, eT, seed, 0, precision="f64", ws=ws, step_ptr=step_dev)   # first call outside capture
    step_dev.zero_()
    a2 = q.init_state(R, precision="f64")
    for k in a:
        a[k].copy_(a2[k])
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s_cap = torch.cuda.Stream()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(g, stream=s_cap, capture_error_mode="relaxed"):
            q.dmc_step(a, b, tau, eT, seed, 0, precision="f64", ws=ws, step_ptr=step_dev)
            q.dmc_step(b, a, tau, eT, seed, 0, precision="f64", ws=ws, step_ptr=step_dev)
    step_dev.zero_()
    for k in a:
        a[k].copy_(a2[k])
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert step_dev.item() == 4
    for k in a:
        assert torch.equal(a[k], ref_a[k]), k


def test_dmc_hydrogen_atom_on_gpu():
    """DMC of the hydrogen atom with a nodeless single-Gaussian trial function
    (variational energy -4 / (3 pi) = -0.4244 Ha) projects to -1/2 Ha."""
    from paper_1209_6630_gb300 import QmcSystem
    g = 8.0 / (9.0 * math.pi)
    c = (2.0 * g / math.pi) ** 0.75
    s = one_atom_system(1, [(0, [g], [c])], 1, 0, [[1.0]])
    q = QmcSystem(s, 0)
    M, tau, nstep, neq, L = 2000, 0.02, 2000, 400, 50
    R = torch.from_numpy(np.random.default_rng(2).normal(size=(M, 1, 3)) * 1.2).to(dev)
    a, b = q.init_state(R, precision="f64"), q.walker_state(M)
    stats = torch.zeros(nstep, 4, dtype=torch.float64, device=dev)
    eT = -0.45
    num = den = 0.0
    logw = []
    for n in range(nstep):
        q.dmc_step(a, b, tau, eT, 8, n, precision="f64", stats=stats[n])
        a, b = b, a
        if n % 100 == 99 or n == neq:        # E_T follows the running estimate
            sv = stats[: n + 1].cpu().numpy()
            lw = np.log(sv[:, 0] / M)
            num = den = 0.0
            for k in range(neq, n + 1):
                P = math.exp(lw[max(0, k - L):k].sum())
                num += P * sv[k, 2]
                den += P * sv[k, 0]
            if den > 0:
                eT = num / den
    e_dmc = num / den
    assert abs(e_dmc + 0.5) < 0.02, e_dmc
