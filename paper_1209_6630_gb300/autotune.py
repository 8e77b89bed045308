"""Tile-shape autotuner for a loaded system.

Candidates (see qmc_tiles in include/qmcgb.h): the Gauss-Jordan panel width
(8, 16, 32 columns), on the mixed path the a4 arithmetic (float-float
elimination with that panel width, or panels of 32 with the updates on the
tensor cores), the walkers per CTA of the float-float C1/C5 kernel (2, 4),
and the C1..C5 products on the tensor cores against the C-free variant.
Each candidate is timed with the library's own per-stage CUDA events
(qmc_walkers_eval_timed) on a sample batch; the choices act on different
stages and are picked one after the other.  Results are cached in JSON,
keyed by the size class (N_up, N_dn, n_ao, mean active AOs per electron
rounded to 32, precision).
"""
from __future__ import annotations

import json
import os

import torch

from ._lib import QmcError
from .build import BUILD

DEFAULT_CACHE = os.environ.get("QMCGB_TILE_CACHE", os.path.join(BUILD, "tiles.json"))


def size_key(q, R, precision):
    cnt, _, _ = q.screen_ao(R[: min(16, R.shape[0])], cap=0, want_B=False)
    kbar = float(cnt.float().mean().item())
    return f"{q.n_up}x{q.n_dn}_ao{q.n_ao}_k{int(round(kbar / 32)) * 32}_{precision}"


def _time(q, R, precision, reps=2):
    q.eval(R, precision=precision)                      # warm-up (attributes, caches)
    stages = []
    for _ in range(reps):
        q.eval(R, precision=precision, stage_ms=stages)
    return [min(s[i] for s in stages) for i in range(8)]


def autotune(q, R, precision="mixed", cache=DEFAULT_CACHE, force=False, verbose=False):
    """Choose and apply tiles for system q using the walker sample R (cuda)."""
    key = size_key(q, R, precision)
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    if key in table and not force:
        q.set_tiles(**table[key]["tiles"])
        return table[key]
    start = {k: v for k, v in q.tiles().items() if k in ("gj_panel", "c15_walkers", "a4_mode")}
    timings = {}
    mixed = precision != "f64"
    best_gj, best_gj_ms = start["gj_panel"], float("inf")
    for nb in (8, 16, 32):
        try:
            q.set_tiles(gj_panel=nb, c15_walkers=start["c15_walkers"], a4_mode="float_float" if mixed else None)
            ms = _time(q, R, precision)
        except QmcError:                       # e.g. shared memory above the limit for this size
            continue
        timings[f"gj_panel={nb}"] = ms[1]
        if ms[1] < best_gj_ms:
            best_gj, best_gj_ms = nb, ms[1]
    best_a4 = start["a4_mode"]
    if mixed:
        best_a4, best_a4_ms = "float_float", best_gj_ms
        try:
            q.set_tiles(gj_panel=best_gj, a4_mode="tensor")
            ms = _time(q, R, precision)
            timings["a4_mode=tensor"] = ms[1]
            if ms[1] < best_a4_ms:
                best_a4, best_a4_ms = "tensor", ms[1]
        except QmcError:                       # the panel kernel's shared memory: at most 880 per spin
            pass
        q.set_tiles(a4_mode=best_a4)
    best_g = start["c15_walkers"]
    if mixed:
        best_g_ms = float("inf")
        for g in (2, 4):
            try:
                q.set_tiles(gj_panel=best_gj, c15_walkers=g)
                ms = _time(q, R, precision)
            except QmcError:
                continue
            timings[f"c15_walkers={g}"] = ms[5]
            if ms[5] < best_g_ms:
                best_g, best_g_ms = g, ms[5]
    q.set_tiles(gj_panel=best_gj, c15_walkers=best_g, a4_mode=best_a4)
    # C1..C5 on the tensor cores against the C-free variant, by the whole evaluation's time
    best_c15 = q.tiles()["c15_mode"]
    if mixed and best_c15 in ("tensor", "cfree"):
        best_c15_ms = float("inf")
        for mode in ("tensor", "cfree"):
            try:
                q.set_tiles(c15_mode=mode)
                ms = _time(q, R, precision)
            except QmcError:
                continue
            timings[f"c15_mode={mode}"] = ms[3]
            if ms[3] < best_c15_ms:
                best_c15, best_c15_ms = mode, ms[3]
        q.set_tiles(c15_mode=best_c15)
    entry = {"tiles": {"gj_panel": best_gj, "c15_walkers": best_g, "a4_mode": best_a4, "c15_mode": best_c15},
             "stage_ms": timings,
             "sample_walkers": int(R.shape[0])}
    if verbose:
        print("autotune", key, entry)
    if cache:
        table[key] = entry
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    torch.cuda.synchronize()
    return entry
