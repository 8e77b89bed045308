"""Mixed batches (several systems in one call / one CUDA-graph launch), tile
choices and the autotuner, through the C ABI, against per-system evaluation
and the oracle."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import config_system, make_walkers, tiny_system

pytestmark = pytest.mark.gpu
dev = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def systems():
    from paper_1209_6630_gb300 import QmcSystem
    out = []
    for s, W in ((config_system("158e"), 64), (tiny_system("mini_chain"), 10), (config_system("434e"), 20)):
        out.append((s, QmcSystem(s, 0), W))
    return out


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_batch_and_graph_match_single_system_calls(systems, precision):
    from paper_1209_6630_gb300 import QmcBatch
    parts = []
    for i, (s, q, W) in enumerate(systems):
        parts.append((q, torch.from_numpy(make_walkers(s, W, first=100 * i)).to(dev)))
    b = QmcBatch(parts, precision=precision, graph=True)
    for rnd in range(2):
        if rnd == 1:   # refill the positions in place; the graph reads the same buffers
            for i, ((s, q, W), (_, R)) in enumerate(zip(systems, parts)):
                R.copy_(torch.from_numpy(make_walkers(s, W, first=5000 + 100 * i)))
        outs = b.launch() if rnd == 1 else b.eval()
        torch.cuda.synchronize()
        for (s, q, W), (_, R), o in zip(systems, parts, outs):
            ref = q.eval(R, precision=precision)
            assert torch.equal(o["status"], ref["status"])
            for k in ("logpsi", "e_loc", "drift", "sign"):
                assert torch.allclose(o[k], ref[k], rtol=1e-12, atol=0), (s.name, k)


def test_every_tile_choice_agrees_with_oracle(systems):
    s, q, W = systems[0]
    R = make_walkers(s, 12, first=777)
    Rd = torch.from_numpy(R).to(dev)
    ref = Oracle(s).eval(R)
    start = {k: v for k, v in q.tiles().items() if k in ("gj_panel", "c15_walkers")}
    try:
        for nb in (8, 16, 32):
            for g in (2, 4):
                q.set_tiles(gj_panel=nb, c15_walkers=g)
                for prec in ("mixed", "f64"):
                    o = q.eval(Rd, precision=prec)
                    lp = o["logpsi"].cpu().numpy()
                    tol = 1e-6 if prec == "mixed" else 1e-10 * np.abs(ref["logpsi"]).max()
                    assert np.abs(lp - ref["logpsi"]).max() < tol, (nb, g, prec)
    finally:
        q.set_tiles(**start)
    from paper_1209_6630_gb300 import QmcError
    with pytest.raises(QmcError):
        q.set_tiles(gj_panel=12)


def test_autotune_chooses_valid_tiles_and_caches(systems, tmp_path):
    from paper_1209_6630_gb300.autotune import autotune
    s, q, W = systems[2]
    R = torch.from_numpy(make_walkers(s, 64, first=9)).to(dev)
    cache = str(tmp_path / "tiles.json")
    e1 = autotune(q, R, precision="mixed", cache=cache)
    assert e1["tiles"]["gj_panel"] in (8, 16, 32) and e1["tiles"]["c15_walkers"] in (2, 4)
    assert {k: q.tiles()[k] for k in e1["tiles"]} == e1["tiles"]
    table = json.load(open(cache))
    assert len(table) == 1
    e2 = autotune(q, R, precision="mixed", cache=cache)      # served from the cache
    assert e2 == e1
