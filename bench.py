#!/usr/bin/env python
"""Throughput of the batched walker evaluation on GB300 (walker-steps/s).

One step = one qmc_walkers_eval (screening, AOs, products, log|det| +
inverse, drift, local energy) over the whole batch of the 1056-electron
synthetic peptide chain (528 + 528 electrons, 3040 AOs, 2048 walkers), with
the positions already resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|f64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU (torchrun, one process per GPU): every rank evaluates its own
2048-walker batch (walkers are independent; no collective on the data path),
value = all walkers / max-over-ranks time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "1056e"
METRIC = "walker-steps/s at 1056 e, mixed-prec vs FP64 GPU path, at <=1e-6 log|Psi| err"


def launches_per_step(q, prec, n_walk):
    """Library kernels launched by one qmc_walkers_eval of a single walker chunk."""
    if prec == "f64":
        return 3                      # contraction, Gauss-Jordan, energy
    t = q.tiles()
    n = 2                             # masks, energy
    if t["c15_mode"] in ("tensor", "cfree"):
        b = 128 if n_walk > 7 * 128 else (32 if n_walk > 128 else 16)
        n += 2 * -(-q.N // b)          # slice producer + MMA kernel per batch of electrons (C1..C5, or C1)
        if t["c15_mode"] == "cfree":
            bv = 264 if n_walk > 128 else 64
            n += 1 + -(-q.N // bv)    # row exponents of D^-1; v = D^-1 A^T with the drift / Laplacian per
                                      # batch of up to 264 electrons (up to 64 for one walker tile)
    else:
        n += 2                        # float-float C1/C5, tensor-core C2..C4
    nmax = max(q.n_up, q.n_dn)
    if t["a4_mode"] in ("float_float", "tensor"):
        panels = -(-nmax // t["gj_panel"])
        redo = 1 + 1 + 2 * panels + 1 + 1     # list, FP64 C1 rows, panel+update per panel, final, FP64 pass
        if t["a4_mode"] == "float_float":
            n += 1 + redo                      # float-float GJ
        else:
            n += 1 + 2 * -(-nmax // 32) + 1 + redo   # init, panel + tensor-core update per 32 columns, final
    else:
        n += 1
    return n
DTYPE = {"f64": "f64", "mixed": "f64 (C1,C5 bf16 exact slices on tcgen05; C2-C4 fp16x3 tcgen05; a4 float-float)",
         "mixed_bf16": "f64 (C1,C5 bf16 exact slices on tcgen05; C2-C4 bf16x3 tcgen05; a4 float-float)"}


def dtype_of(q, prec):
    if prec == "f64":
        return "f64"
    t = q.tiles()
    c15 = "bf16 exact slices on tcgen05" if t["c15_mode"] in ("tensor", "cfree") else "float-float FP32 pipes"
    c24 = "fp16x3" if prec == "mixed" else "bf16x3"
    if t["c15_mode"] == "cfree":
        c24 = "none (C-free: v = D^-1 A^T bf16 exact slices on tcgen05, AO derivatives fp32 / float-float)"
    a4 = {"float_float": "float-float + FP64 near nodes",
          "tensor": "float-float panels, bf16 exact-slice tcgen05 updates + FP64 near nodes"}.get(t["a4_mode"], "FP64")
    return f"f64 (C1,C5 {c15}; C2-C4 {c24} tcgen05; a4 {a4})"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["f64", "mixed", "mixed_bf16"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--walkers", type=int, default=0, help="override the batch size")
    p.add_argument("--cpu-sample", type=int, default=0, help="walkers in the oracle sample")
    p.add_argument("--no-compare", action="store_true", help="skip the FP64-path comparison")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--adjoint-walkers", type=int, default=512, help="walkers of the adjoint's 1731e workload")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="keep default tiles (no autotuner)")
    p.add_argument("--no-dmc", action="store_true", help="skip the full DMC step timing")
    p.add_argument("--no-cfree", action="store_true", help="skip the C-free variant's timing")
    p.add_argument("--c15-mode", default=None, choices=["float_float", "tensor", "cfree"],
                   help="override the C1..C5 arithmetic of the timed evaluation")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the 1731-electron forward comparison and the mixed batch")
    return p.parse_args()


def aggregate(t_local_ms, walkers_local, world, dist=None, device=None):
    """Whole-job throughput over `world` ranks: every rank evaluates its own
    batch; the step time is the maximum over ranks."""
    t = t_local_ms
    if world > 1:
        import torch
        x = torch.tensor([t_local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, world * walkers_local / (t / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9 or f[0] != str(self.gpu_index):
                    continue
                rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp64_peak_tflops(pk):
    # 152 SMs x 2 DFMA (4 flop) per clock per SM x maximum SM clock
    mhz = pk.get("sm_max_mhz", 2070.0)
    return 152 * 4 * mhz * 1e6 / 1e12


def kernel_traffic(kernel, workload):
    """DRAM bytes per launch from profiles/ncu_traffic.txt, if the kernel's
    source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
        if kv.get("kernel") != kernel or kv.get("workload") != workload:
            continue
        src = os.path.join(ROOT, "paper_1209_6630_gb300", "csrc", kv.get("source", ""))
        if not os.path.exists(src):
            return None
        h = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
        if h != kv.get("source_sha1"):
            return None
        return float(kv["bytes_per_launch"])
    return None


def stage_roofline(q, prec, stage_mean, kbar, W, pk):
    """Roofline of the dominant stage of one step.  `achieved` counts the
    method's own work (the algorithmic flop of the paper's formulation:
    2 sum_s N_s^3 for log|det| + inverse, 10 sum_s N_s^2 Kbar for the five
    products), divided by the stage's CUDA-event time, against the measured
    peak of the pipe that executes it; `frac_issued` counts what the kernels
    issue on that pipe (the exact-slice products of the emulated FP64-class
    arithmetic), and `fp64_equiv_ratio` compares the achieved rate with the
    measured FP64 DFMA rate."""
    n_up, n_dn = q.n_up, q.n_dn
    prod = kbar * (n_up * n_up + n_dn * n_dn) * W          # sum_s N_s Kbar N_s multiply-adds per output
    flop_a4 = 2.0 * (n_up ** 3 + n_dn ** 3) * W
    flop_a3 = 10.0 * prod
    bf16 = pk.get("bf16_tflops_sustained")
    fp64_peak = fp64_peak_tflops(pk)
    fp32_inst_peak = 152 * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12      # T instructions/s
    t = q.tiles()
    if prec == "f64":
        kern_ms = {"k_contract_f64": stage_mean[0], "k_gj": stage_mean[1], "k_drift_energy": stage_mean[2]}
    else:
        a4_kern = {"float_float": "k_gj_ff+k_gj", "tensor": "k_gt_panel+k_gt_update+k_gj"}.get(t["a4_mode"], "k_gj")
        c15_kern = {"tensor": "k_c15_prep+k_c15_mma", "cfree": "k_c15_prep+k_c15_mma (C1)"}.get(t["c15_mode"],
                                                                                           "k_c15_ff")
        kern_ms = {"k_shell_mask": stage_mean[4], c15_kern: stage_mean[5], "k_tc_contract": stage_mean[6],
                   a4_kern: stage_mean[1],
                   "k_vd_mma+k_drift_energy" if t["c15_mode"] == "cfree" else "k_drift_energy": stage_mean[2]}
    kern = max(kern_ms, key=kern_ms.get)
    ts = kern_ms[kern] / 1e3
    fp64_src = "FP64 DFMA: 152 SMs x 4 flop/clk x sm_max_mhz (the measured DFMA rate is 1.20 TFLOP/s)"
    if kern == "k_gj":
        roof = {"bound": "alu", "achieved": flop_a4 / ts / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                "peak_source": fp64_src, "work": "2 (N_up^3 + N_dn^3) flop per walker"}
    elif kern == "k_contract_f64":
        roof = {"bound": "alu", "achieved": flop_a3 / ts / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                "peak_source": fp64_src, "work": "10 sum_s N_s^2 Kbar flop per walker"}
    elif kern == "k_gj_ff+k_gj":
        roof = {"bound": "alu", "achieved": flop_a4 / ts / 1e12, "peak": fp32_inst_peak / 6.0, "unit": "TFLOP/s",
                "peak_source": "FP32 pipe (152 SMs x 128 lanes x sm_max_mhz) / 6: 12 FP32 instructions "
                               "per float-float multiply-add",
                "work": "2 (N_up^3 + N_dn^3) flop per walker (float-float elimination + FP64 near nodes)"}
    elif kern == "k_gt_panel+k_gt_update+k_gj":
        roof = {"bound": "tensor", "achieved": flop_a4 / ts / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_source": "measured dense bf16 sustained (MEASURED_PEAKS.json), the pipe that executes the "
                               "rank-32 updates",
                "work": "2 (N_up^3 + N_dn^3) flop per walker (the LU + inverse of the paper's accounting)",
                "issued": "28 BF16 slice-pair products per multiply-add of the updates"}
        roof["frac_issued"] = 28 * flop_a4 / ts / 1e12 / bf16 if bf16 else None
    elif kern == "k_c15_prep+k_c15_mma":
        roof = {"bound": "tensor", "achieved": flop_a3 / ts / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_source": "measured dense bf16 sustained (MEASURED_PEAKS.json)",
                "work": "10 sum_s N_s^2 Kbar flop per walker (the five products C1..C5)",
                "issued": "C1, C5: 21 BF16 slice-pair products each; C2..C4: 3 fp16 split products each"}
        roof["frac_issued"] = (2 * 21 + 3 * 3) * 2.0 * prod / ts / 1e12 / bf16 if bf16 else None
    elif kern == "k_c15_prep+k_c15_mma (C1)":
        roof = {"bound": "tensor", "achieved": 2.0 * prod / ts / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_source": "measured dense bf16 sustained (MEASURED_PEAKS.json)",
                "work": "2 sum_s N_s^2 Kbar flop per walker (C1)", "issued": "21 BF16 slice-pair products"}
        roof["frac_issued"] = 21 * 2.0 * prod / ts / 1e12 / bf16 if bf16 else None
    elif kern == "k_vd_mma+k_drift_energy":
        roof = {"bound": "tensor", "achieved": 2.0 * prod / ts / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_source": "measured dense bf16 sustained (MEASURED_PEAKS.json)",
                "work": "2 sum_s N_s^2 Kbar flop per walker (v = D^-1 A^T)", "issued": "21 BF16 slice-pair products"}
        roof["frac_issued"] = 21 * 2.0 * prod / ts / 1e12 / bf16 if bf16 else None
    elif kern == "k_c15_ff":
        roof = {"bound": "alu", "achieved": 4.0 * prod / ts / 1e12, "peak": fp32_inst_peak / 4.5, "unit": "TFLOP/s",
                "peak_source": "FP32 pipe / 4.5: 9 FP32 instructions per float-float product",
                "work": "2 outputs x 2 sum_s N_s^2 Kbar flop per walker (C1, C5)"}
    elif kern == "k_tc_contract":
        roof = {"bound": "tensor", "achieved": 6.0 * prod / ts / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "peak_source": "measured dense bf16 (= fp16) sustained", "work": "3 outputs x 2 sum_s N_s^2 Kbar flop"}
        roof["frac_issued"] = 3 * 6.0 * prod / ts / 1e12 / bf16 if bf16 else None
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s"}
    roof["kernel"] = kern
    roof["kernel_ms_per_launch_region"] = kern_ms[kern]
    roof["frac"] = roof["achieved"] / roof["peak"] if roof.get("peak") and roof.get("achieved") else None
    if roof.get("achieved") and roof.get("unit") == "TFLOP/s":
        roof["fp64_equiv_ratio"] = roof["achieved"] / 1.20     # against the measured FP64 DFMA rate
    return roof, kern_ms


def config4_forward(a, flush, e0, e1):
    """The 1731-electron open-shell chain (866 + 865 electrons, 4985 AOs, FP32
    MO coefficients) with 512 walkers: the mixed path against the plain FP64
    GPU path on the same batch, with the accuracy of every walker against the
    FP64 path."""
    import torch
    from paper_1209_6630_gb300 import QmcSystem
    from synth import config_system, make_walkers
    s = config_system("1731e")
    q = QmcSystem(s, 0)
    W = 512
    R = torch.from_numpy(make_walkers(s, W, first=9000)).cuda()

    def timed(prec, reps):
        ws = q.workspace(W, prec)
        out = q.alloc_out(W)
        q.eval(R, precision=prec, out=out, ws=ws)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0.record()
            q.eval(R, precision=prec, out=out, ws=ws)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts), out

    t_m, om = timed("mixed", 3)
    t_f, of = timed("f64", 1)
    ok = (om["status"] == 0) & (of["status"] == 0)
    dlp = (om["logpsi"] - of["logpsi"]).abs()[ok]
    del_ = ((om["e_loc"] - of["e_loc"]).abs() / of["e_loc"].abs())[ok]
    q.close()
    return {"workload": "1731e synthetic open-shell chain (866+865 e, 4985 AOs, FP32 A), 512 walkers",
            "mixed": {"walker_steps_per_s": W / (t_m / 1e3), "ms_per_step": t_m},
            "fp64_path": {"walker_steps_per_s": W / (t_f / 1e3), "ms_per_step": t_f},
            "speedup_vs_fp64_path": t_f / t_m,
            "accuracy_vs_fp64_path": {"walkers": int(ok.sum().item()), "max_abs_logpsi_err": float(dlp.max().item()),
                                      "p99_abs_logpsi_err": float(torch.quantile(dlp, 0.99).item()),
                                      "max_rel_eloc_err": float(del_.max().item()),
                                      "status_mismatch": int((om["status"] != of["status"]).sum().item())}}


def config2_precision_report(a, flush, e0, e1):
    """The 434-electron chain (two 217 x 217 Slater matrices) with 4096 walkers:
    the contraction's precision modes with the LU / inverse in FP64 (a4_mode
    fp64), each result's error against the plain FP64 GPU path over every walker
    (that path meets the oracle at 1e-10), the Slater entries against the FP64
    oracle on sampled walkers, and the time per step.  Modes: C1/C5 from exact
    BF16 slices on the tensor cores with C2..C4 split FP16x3 (mixed) or BF16x3
    (mixed_bf16); C1/C5 in float-float on the FP32 pipes with C2..C4 FP16x3;
    and the default mixed step (C-free variant, its a4)."""
    import numpy as np
    import torch
    import oracle
    from paper_1209_6630_gb300 import QmcSystem
    from synth import config_system, make_walkers
    s = config_system("434e")
    q = QmcSystem(s, 0)
    W = 4096
    Rn = make_walkers(s, W, first=21000)
    R = torch.from_numpy(Rn).cuda()
    defaults = q.tiles()

    def timed(prec, reps):
        ws = q.workspace(W, prec)
        out = q.alloc_out(W)
        q.eval(R, precision=prec, out=out, ws=ws)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0.record()
            q.eval(R, precision=prec, out=out, ws=ws)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts), out

    t_f, of = timed("f64", 1)
    sample = [0, 1, 2047, 4095]
    dbg = [oracle.Oracle(s).eval_debug(Rn[w]) for w in sample]

    def rowwise(a_, b_):
        den = np.abs(b_).max(axis=-1, keepdims=True)
        return float((np.abs(a_ - b_) / np.where(den == 0, 1.0, den)).max())

    modes = {}
    for label, prec, tiles in (("c1c5_exact_slices_c2c4_fp16x3", "mixed", dict(c15_mode="tensor", a4_mode="fp64")),
                               ("c1c5_exact_slices_c2c4_bf16x3", "mixed_bf16", dict(c15_mode="tensor", a4_mode="fp64")),
                               ("c1c5_float_float_c2c4_fp16x3", "mixed", dict(c15_mode="float_float", a4_mode="fp64")),
                               ("default_mixed_step", "mixed", {})):
        q.set_tiles(**{**{k: defaults[k] for k in ("c15_mode", "a4_mode")}, **tiles})
        t_m, om = timed(prec, 2)
        ok = (om["status"] == 0) & (of["status"] == 0)
        dlp = (om["logpsi"] - of["logpsi"]).abs()[ok]
        del_ = ((om["e_loc"] - of["e_loc"]).abs() / of["e_loc"].abs())[ok]
        ddr = ((om["drift"] - of["drift"]).abs().amax(dim=(1, 2)) / of["drift"].abs().amax(dim=(1, 2)))[ok]
        rec = {"precision": prec, "tiles": tiles or "library defaults",
               "walker_steps_per_s": W / (t_m / 1e3), "ms_per_step": t_m,
               "vs_fp64_path": {"walkers": int(ok.sum().item()), "max_abs_logpsi_err": float(dlp.max().item()),
                                "p99_abs_logpsi_err": float(torch.quantile(dlp, 0.99).item()),
                                "max_rel_eloc_err": float(del_.max().item()),
                                "max_drift_normwise_err": float(ddr.max().item()),
                                "status_mismatch": int((om["status"] != of["status"]).sum().item())}}
        if tiles:
            up, dn = q.slater(R[sample], precision=prec)
            up, dn = up.cpu().numpy(), dn.cpu().numpy()
            err = {"C1": 0.0, "C2..C4": 0.0, "C5": 0.0}
            for k, d in enumerate(dbg):
                for got, ref in ((up[k], d["C_up"]), (dn[k], d["C_dn"])):
                    err["C1"] = max(err["C1"], rowwise(got[0], ref[0]))
                    err["C5"] = max(err["C5"], rowwise(got[4], ref[4]))
                    err["C2..C4"] = max(err["C2..C4"], max(rowwise(got[l], ref[l]) for l in range(1, 4)))
            rec["slater_vs_oracle_rowwise"] = {"walkers": len(sample), **err}
        modes[label] = rec
    q.set_tiles(c15_mode=defaults["c15_mode"], a4_mode=defaults["a4_mode"])
    q.close()
    return {"workload": "434e synthetic chain (217+217 e, 1260 AOs), 4096 walkers; LU/inverse in FP64 (a4_mode fp64) "
                        "for the contraction modes",
            "fp64_path": {"walker_steps_per_s": W / (t_f / 1e3), "ms_per_step": t_f},
            "modes": modes,
            "not_built": "TF32x1 / TF32x3 contraction modes (the exact BF16 slices reach FP64-class entries instead)"}


def cfree_bench(q, R, prec, flush, e0, e1, mode):
    """The other C1..C5 arithmetic on the same batch (c15_mode tensor: C1..C5 on
    the tensor cores; cfree: C1 alone, then the drift and Laplacian from
    v = D^-1 A^T), timed like the default; returns the timing and its outputs
    for the accuracy check against the FP64 path."""
    import numpy as np
    import torch
    W = int(R.shape[0])
    old = q.tiles()["c15_mode"]
    q.set_tiles(c15_mode=mode)
    try:
        ws = q.workspace(W, prec)
        out = q.alloc_out(W)
        for _ in range(2):
            q.eval(R, precision=prec, out=out, ws=ws)
        torch.cuda.synchronize()
        ts, stages = [], []
        for _ in range(3):
            flush.zero_()
            e0.record()
            q.eval(R, precision=prec, out=out, ws=ws, stage_ms=stages)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    finally:
        q.set_tiles(c15_mode=old)
    st = np.array(stages).mean(axis=0)
    t = sum(ts) / len(ts)
    res = {"walker_steps_per_s": W / (t / 1e3), "ms_per_step": t,
           "stage_ms": {"masks": st[4], "products": st[5], "a4": st[1], "drift_energy": st[2]},
           "what": {"cfree": "C1 only, then v = D^-1 A^T on the tensor cores and the drift / Laplacian from the "
                             "AO derivatives",
                    "tensor": "C1..C5 on the tensor cores (exact slices for C1, C5; fp16x3 for C2..C4)"}[mode]}
    return res, out


def dmc_bench(q, R, prec, flush, e0, e1):
    """One fixed-node DMC step with constant population (qmc_dmc_step: move
    Eq. 1, evaluation, weight Eq. 3, reconfiguration Sec. II.B, copy of the
    drawn walkers) on the same batch, timed like the evaluation; the MC
    kernels (move, weight, reconfiguration) are also timed on their own
    through their entry points.  (The step evaluates the moved walkers, so
    its time minus the evaluation of the unmoved batch is not the MC share.)"""
    import torch
    W = int(R.shape[0])
    a0 = q.init_state(R, precision=prec)
    a = {k: v.clone() for k, v in a0.items()}
    b = q.walker_state(W)
    e_t = float(a["e_loc"].mean().item())
    ws = torch.empty(q.dmc_workspace_size(W, prec), dtype=torch.uint8, device=R.device)
    stats = torch.zeros(4, dtype=torch.float64, device=R.device)
    tau = 1e-4          # all-electron moves of 1056 electrons: larger steps cross nodes (fixed-node rejections)
    for n in range(2):
        q.dmc_step(a, b, tau, e_t, 17, n, precision=prec, stats=stats, ws=ws)
        a, b = b, a
    torch.cuda.synchronize()
    # every timed step starts from the same evaluated population (the walkers of the batch):
    # without drift limiting or equilibration a population of unequilibrated all-electron walkers
    # collapses onto near-nucleus configurations within a few steps (E_L -> -inf without the cusp)
    ts = []
    for n in range(2, 5):
        for k in a:
            a[k].copy_(a0[k])
        flush.zero_()
        e0.record()
        q.dmc_step(a, b, tau, e_t, 17, n, precision=prec, stats=stats, ws=ws)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    t = sum(ts) / len(ts)
    sv = stats.cpu().numpy()
    from paper_1209_6630_gb300 import dmc_move, dmc_weight, srmc_reconfigure
    st0 = a0

    def one(fn):
        fn()
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)
    mc = {"move": one(lambda: dmc_move(st0["R"], st0["drift"], tau, 17, 9)),
          "weight": one(lambda: dmc_weight(st0["e_loc"], st0["sign"], st0["status"], st0["e_loc"], st0["sign"],
                                           st0["status"], tau, e_t)),
          "reconfiguration": one(lambda: srmc_reconfigure(st0["e_loc"].abs(), 17, 9))}
    res = {"walker_steps_per_s": W / (t / 1e3), "ms_per_step": t, "tau": tau,
           "mc_kernels_ms": mc, "accepted": int(sv[3]), "walkers_alive": int(sv[1]),
           "what": "move (Eq. 1) + evaluation + fixed-node weight (Eq. 3) + SRMC draw (Sec. II.B) + copy"}
    del a, a0, b, ws
    torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
def cpu_oracle_sample(system, R, n_sample):
    import oracle
    o = oracle.Oracle(system)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = o.eval(R[:n_sample], nthreads=cores)
    dt = time.perf_counter() - t0
    return ref, dt, cores


def adjoint_bench(a, prec, flush, e0, e1, pk, fp64_peak):
    import torch
    from paper_1209_6630_gb300 import QmcSystem
    from synth import config_system, make_walkers
    s = config_system("1731e")
    q = QmcSystem(s, 0)
    W = a.adjoint_walkers
    R = torch.from_numpy(make_walkers(s, W, first=7000)).cuda()
    o = q.eval(R, precision=prec, want_dinv=True)
    el = o["e_loc"]
    g = torch.where(o["status"] == 0, 2.0 * (el - el.mean()) / W, torch.zeros_like(el)).contiguous()
    cnt, _, _ = q.screen_ao(R[:8], cap=0, want_B=False)
    kbar = float(cnt.float().mean().item())
    flop = 2.0 * kbar * (s.n_up ** 2 + s.n_dn ** 2) * W
    aprec = "f64" if prec == "f64" else "mixed"

    def timed(p, reps):
        q.backward(R, o["dinv"], g, precision=p)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0.record()
            q.backward(R, o["dinv"], g, precision=p)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts)

    t_a = timed(aprec, 3 if aprec == "mixed" else 1)
    adj = {"workload": "1731e synthetic open-shell chain (866+865 e, 4985 AOs), E_L-weighted g",
           "walkers": W, "precision": aprec, "ms": t_a, "walkers_per_s": W / (t_a / 1e3), "kbar_active_aos": kbar,
           "work": "2 sum_s N_s Kbar N_s flop per walker (the sparse contraction's own products)"}
    ach = flop / (t_a / 1e3) / 1e12
    if aprec == "mixed":
        # the method's flop against the executed pipe's measured peak; the six BF16 slice
        # products issued per FP32-accurate product are reported as frac_issued
        bf = pk.get("bf16_tflops_sustained")
        adj["roofline"] = {"bound": "tensor", "achieved": ach, "peak": bf, "unit": "TFLOP/s",
                           "peak_source": "measured dense bf16 sustained (MEASURED_PEAKS.json)",
                           "frac": ach / bf if bf else None, "frac_issued": 6 * ach / bf if bf else None,
                           "fp64_equiv_ratio": ach / 1.20}
        if not a.no_compare:
            adj["fp64_adjoint_ms"] = timed("f64", 1)
            n = min(W, 64)
            m_up, m_dn = q.backward(R[:n], o["dinv"][:n], g[:n], precision="mixed")
            f_up, f_dn = q.backward(R[:n], o["dinv"][:n], g[:n], precision="f64")
            err = max(float(((m - f).abs().max() / f.abs().max()).item()) for m, f in ((m_up, f_up), (m_dn, f_dn)))
            adj["vs_fp64_adjoint"] = {"walkers": n, "normwise_rel_err": err}
    else:
        adj["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                           "peak_source": "FP64: 152 SMs x 4 flop/clk x sm_max_mhz",
                           "frac": ach / fp64_peak if fp64_peak else None}
    return adj


def reference_arm(a, ws, rank):
    if rank != 0:
        return
    from synth import config_system, make_walkers
    s = config_system(a.workload)
    n = a.cpu_sample or {"158e": 100, "434e": 96, "1056e": 32, "1731e": 16}.get(a.workload, 16)
    R = make_walkers(s, n)
    import oracle
    o = oracle.Oracle(s)
    cores = os.cpu_count() or 1
    for _ in range(a.warmup):
        o.eval(R[: max(1, n // 4)], nthreads=cores)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        o.eval(R, nthreads=cores)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = n / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "walker-steps/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{a.workload} synthetic peptide chain", "walkers_per_step": n,
                       "sample": f"{n} walkers of the {a.workload} workload per step"},
            "cpu_baseline": {"value": v, "unit": "walker-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} walkers per step, OpenMP over walkers"},
            "e2e": {"value": v, "unit": "walker-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def mixed_batch_run(W, local, rank, precision, tune, steps, warmup, oracle_sample):
    """The mixed batch: W walkers of each of the 158-, 434-, 1056- and
    1731-electron systems (walker seeds interleaved: global walker 4j + s is
    walker j of system s), replayed as one CUDA graph per step.  Returns the
    step time, the clocks, the tiles and (rank 0, oracle_sample) the
    per-system errors against the oracle on the first and last walker of each
    system, with the oracle's time as the CPU baseline."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1209_6630_gb300 import QmcBatch, QmcSystem
    from synth import config_system, make_walkers
    keys = ["158e", "434e", "1056e", "1731e"]
    parts, systems, hosts, tiles = [], [], [], {}
    for k in keys:
        s = config_system(k)
        q = QmcSystem(s, local)
        Rh = make_walkers(s, W, first=rank * W)
        R = torch.from_numpy(Rh).to(dev)
        if tune:
            from paper_1209_6630_gb300.autotune import autotune
            tiles[k] = autotune(q, R, precision=precision)["tiles"]
        else:
            tiles[k] = q.tiles()
        parts.append((q, R))
        systems.append(s)
        hosts.append(Rh)
    b = QmcBatch(parts, precision=precision, graph=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(warmup, 0)):
        b.launch()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(steps):
        flush.zero_()
        e0.record()
        b.launch()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = clk.stop()
    res = {"ms": sum(times) / len(times), "clocks": clocks, "tiles": tiles}
    if rank == 0 and oracle_sample:
        # the oracle on the first and last walker of each system: the per-system errors of
        # the graph's results, and its time as the CPU baseline
        errs = {}
        outs = b.launch()
        torch.cuda.synchronize()
        t_cpu, n_cpu, cores = 0.0, 0, os.cpu_count() or 1
        for k, s, Rh, o in zip(keys, systems, hosts, outs):
            sample = [0, W - 1]
            ref, dt, cores = cpu_oracle_sample(s, Rh[sample], len(sample))
            t_cpu += dt
            n_cpu += len(sample)
            lp = o["logpsi"].cpu().numpy()[sample]
            el = o["e_loc"].cpu().numpy()[sample]
            st = o["status"].cpu().numpy()[sample]
            errs[k] = {"max_abs_logpsi_err": float(np.abs(lp - ref["logpsi"]).max()),
                       "max_rel_eloc_err": float((np.abs(el - ref["e_loc"]) / np.abs(ref["e_loc"])).max()),
                       "status_mismatch": int((st != ref["status"]).sum()), "walkers": len(sample)}
        res["parity"] = errs
        res["cpu_baseline"] = {"value": n_cpu / t_cpu, "unit": "walker-steps/s", "cores": cores, "kind": "oracle",
                               "sample": "first and last walker of each of the four systems, FP64 oracle"}
    del b, parts
    torch.cuda.synchronize()
    return res


def mixed_batch_arm(a, ws, rank, local):
    """The mixed batch as its own bench line (--workload mixed4)."""
    W = a.walkers or 1024
    r = mixed_batch_run(W, local, rank, a.precision, not a.no_tune, a.steps, a.warmup, not a.no_cpu)
    t, value = aggregate(r["ms"], 4 * W, ws)
    line = {"metric": "walker-steps/s, mixed batch of 158/434/1056/1731-electron systems in one CUDA graph",
            "value": value, "unit": "walker-steps/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[a.precision], "data": "synthetic",
            "config": {"workload": "mixed batch 4 x 1024 walkers (158, 434, 1056, 1731 e)", "walkers_per_system": W,
                       "precision": a.precision, "l2": "flushed between timed steps", "tiles": r["tiles"]},
            "gpu_launches": "one CUDA graph per step"}
    if r["clocks"]:
        line["clocks"] = r["clocks"]
    for k in ("parity", "cpu_baseline"):
        if k in r:
            line[k] = r[k]
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    a = parse()
    ws, rank, local = dist_env()
    if a.impl == "reference":
        reference_arm(a, ws, rank)
        return
    if a.workload == "mixed4":
        mixed_batch_arm(a, ws, rank, local)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    if ws > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1209_6630_gb300 import QmcSystem
    from synth import WALKERS, config_system, make_walkers

    s = config_system(a.workload)
    W = a.walkers or WALKERS[a.workload]
    R_host = make_walkers(s, W, first=rank * W)
    q = QmcSystem(s, local)
    R = torch.from_numpy(R_host).to(dev)
    prec = a.precision
    tiles = q.tiles()
    if not a.no_tune:
        from paper_1209_6630_gb300.autotune import autotune
        tuned = autotune(q, R[: min(W, 1024)], precision=prec)
        tiles = dict(tuned["tiles"], stage_ms=tuned.get("stage_ms"))
    if a.c15_mode:
        q.set_tiles(c15_mode=a.c15_mode)
        tiles = dict(tiles, c15_mode=a.c15_mode)
    wsbuf = q.workspace(W, prec)
    out = q.alloc_out(W, want_dinv=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()

    for _ in range(max(a.warmup, 0)):
        q.eval(R, precision=prec, out=out, ws=wsbuf)
    barrier()

    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local])
        except ValueError:
            pass
    clk = ClockSampler(gpu_index)
    clk.start()
    stages = []
    step_ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    for _ in range(a.steps):
        flush.zero_()          # evict L2 between timed steps (not timed)
        e0.record()
        q.eval(R, precision=prec, out=out, ws=wsbuf, stage_ms=stages)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    barrier()
    clocks = clk.stop()
    t_step, value = aggregate(sum(step_ms) / len(step_ms), W, ws, dist, dev)
    st = np.array(stages)            # [K, 8]
    stage_mean = st.mean(axis=0)
    n_launch = launches_per_step(q, prec, W)   # one walker chunk

    # screening statistics of this batch (a1 on a sample, outside the timed region)
    ns = 16
    cnt, _, _ = q.screen_ao(R[:ns], cap=0, want_B=False)
    kbar = float(cnt.float().mean().item())

    n_up, n_dn = s.n_up, s.n_dn
    pk = peaks()
    fp64_peak = fp64_peak_tflops(pk)
    roof, kern_ms = stage_roofline(q, prec, stage_mean, kbar, W, pk)
    kern = roof["kernel"]
    roof["traffic"] = kernel_traffic(kern, a.workload)
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel's unchanged source, "
                              "scaled to this launch (profiles/ncu_traffic.txt)") if roof["traffic"] else None
    roof["kernel_ms"] = kern_ms
    roof["stage_ms"] = {"a1_a3": stage_mean[0], "a4": stage_mean[1], "a5_a6": stage_mean[2]}

    line = {"metric": METRIC, "value": value, "unit": "walker-steps/s", "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(q, prec), "data": "synthetic",
            "config": {"workload": f"{a.workload} synthetic peptide chain (528+528 e, 3040 AOs)"
                       if a.workload == "1056e" else a.workload,
                       "walkers_per_gpu": W, "precision": prec, "l2": "flushed between timed steps",
                       "parallelism": f"walker replicas x{ws}", "kbar_active_aos": kbar, "tiles": tiles},
            "roofline": roof, "gpu_launches": n_launch * a.steps}
    if clocks:
        line["clocks"] = clocks

    # end to end through the public API: pinned host positions in, results out
    R_pin = torch.from_numpy(R_host).pin_memory()
    host_out = {k: torch.empty(out[k].shape, dtype=out[k].dtype).pin_memory()
                for k in ("logpsi", "sign", "e_loc", "drift", "status")}
    R_dev = torch.empty_like(R)
    q.eval(R, precision=prec, out=out, ws=wsbuf)
    barrier()
    e2e_ms = []
    for _ in range(max(1, min(a.steps, 3))):
        flush.zero_()
        e0.record()
        R_dev.copy_(R_pin, non_blocking=True)
        q.eval(R_dev, precision=prec, out=out, ws=wsbuf)
        for k, hb in host_out.items():
            hb.copy_(out[k], non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    t_e2e, v_e2e = aggregate(sum(e2e_ms) / len(e2e_ms), W, ws, dist, dev)
    line["e2e"] = {"value": v_e2e, "unit": "walker-steps/s",
                   "h2d_bytes_per_step": int(R_pin.numel() * 8),
                   "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in host_out.values()))}

    if not a.no_dmc:
        line["dmc_step"] = dmc_bench(q, R, prec, flush, e0, e1)
    cf_out = None
    if prec != "f64" and not a.no_cfree and q.tiles()["c15_mode"] in ("tensor", "cfree"):
        alt = "tensor" if q.tiles()["c15_mode"] == "cfree" else "cfree"
        line["c15_mode_" + alt], cf_out = cfree_bench(q, R, prec, flush, e0, e1, alt)

    # the plain FP64 GPU path on the same batch (the metric's comparison)
    if prec != "f64" and not a.no_compare:
        mixed_lp = out["logpsi"].clone()
        mixed_el = out["e_loc"].clone()
        mixed_st = out["status"].clone()
        ws64 = q.workspace(W, "f64")
        q.eval(R, precision="f64", out=out, ws=ws64)
        # accuracy of the timed mixed-precision step over the whole batch, against the FP64 path
        ok = (mixed_st == 0) & (out["status"] == 0)
        dlp = (mixed_lp - out["logpsi"]).abs()[ok]
        del_ = ((mixed_el - out["e_loc"]).abs() / out["e_loc"].abs())[ok]
        line["accuracy_vs_fp64_path"] = {
            "walkers": int(ok.sum().item()), "max_abs_logpsi_err": float(dlp.max().item()),
            "p99_abs_logpsi_err": float(torch.quantile(dlp, 0.99).item()),
            "max_rel_eloc_err": float(del_.max().item()),
            "status_mismatch": int((mixed_st != out["status"]).sum().item())}
        if cf_out is not None:
            okc = (cf_out["status"] == 0) & (out["status"] == 0)
            dlc = (cf_out["logpsi"] - out["logpsi"]).abs()[okc]
            dec = ((cf_out["e_loc"] - out["e_loc"]).abs() / out["e_loc"].abs())[okc]
            ddc = ((cf_out["drift"] - out["drift"]).abs().amax(dim=(1, 2)) /
                   out["drift"].abs().amax(dim=(1, 2)))[okc]
            line["c15_mode_" + alt]["accuracy_vs_fp64_path"] = {
                "walkers": int(okc.sum().item()), "max_abs_logpsi_err": float(dlc.max().item()),
                "max_rel_eloc_err": float(dec.max().item()), "max_drift_normwise_err": float(ddc.max().item()),
                "status_mismatch": int((cf_out["status"] != out["status"]).sum().item())}
            del cf_out
        t64 = []
        for _ in range(2):
            flush.zero_()
            e0.record()
            q.eval(R, precision="f64", out=out, ws=ws64)
            e1.record()
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        m64 = sum(t64) / len(t64)
        line["fp64_path"] = {"value": ws * W / (m64 / 1e3), "ms_per_step": m64}
        # the FP64 path with the tensor-core a4 and FP64 recomputation above f64_kappa_max
        # (QMC_PREC_F64_TCA4), gated against the FP64 path's 1e-10 relative bar
        f64_lp, f64_el, f64_st = out["logpsi"].clone(), out["e_loc"].clone(), out["status"].clone()
        ws_tc = q.workspace(W, "f64_tca4")
        o_tc = q.alloc_out(W)
        q.eval(R, precision="f64_tca4", out=o_tc, ws=ws_tc)
        flush.zero_()
        e0.record()
        q.eval(R, precision="f64_tca4", out=o_tc, ws=ws_tc)
        e1.record()
        e1.synchronize()
        m_tc = e0.elapsed_time(e1)
        okt = (o_tc["status"] == 0) & (f64_st == 0)
        rlp = ((o_tc["logpsi"] - f64_lp).abs() / f64_lp.abs())[okt]
        rel = ((o_tc["e_loc"] - f64_el).abs() / f64_el.abs())[okt]
        line["fp64_tca4_path"] = {
            "value": ws * W / (m_tc / 1e3), "ms_per_step": m_tc, "f64_kappa_max": q.tiles()["f64_kappa_max"],
            "vs_fp64_path": {"walkers": int(okt.sum().item()), "max_rel_logpsi_err": float(rlp.max().item()),
                             "max_rel_eloc_err": float(rel.max().item()),
                             "walkers_within_1e-10": int(((rlp <= 1e-10) & (rel <= 1e-10)).sum().item()),
                             "status_mismatch": int((o_tc["status"] != f64_st).sum().item())}}
        del ws_tc, o_tc
        q._ws.pop("f64_tca4", None)
        del ws64
        q._ws.pop("f64", None)
        torch.cuda.empty_cache()

    # adjoint d log|Psi| / dA (E_L-weighted) on its own workload: the 1731-electron
    # open-shell system with 512 walkers; FP64 after the FP64 path, the tensor-core
    # contraction after the mixed one, the FP64 adjoint timed beside it
    if not a.no_adjoint:
        line["adjoint"] = adjoint_bench(a, prec, flush, e0, e1, pk, fp64_peak)

    # parity on a sample and the CPU baseline (rank 0 only, N = 1 only)
    if rank == 0 and ws == 1 and not a.no_cpu:
        n_s = a.cpu_sample or 32
        ref, dt, cores = cpu_oracle_sample(s, R_host, n_s)
        got = q.eval(R[:n_s], precision=prec)
        lp = got["logpsi"].cpu().numpy()
        el = got["e_loc"].cpu().numpy()
        ok = ref["status"] == 0
        line["parity"] = {"walkers": n_s,
                          "max_abs_logpsi_err": float(np.abs(lp[ok] - ref["logpsi"][ok]).max()),
                          "max_rel_eloc_err": float((np.abs(el[ok] - ref["e_loc"][ok]) /
                                                     np.abs(ref["e_loc"][ok])).max()),
                          "status_mismatch": int((got["status"].cpu().numpy() != ref["status"]).sum())}
        line["cpu_baseline"] = {"value": n_s / dt, "unit": "walker-steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"{n_s} walkers of the same batch, FP64 oracle, OpenMP over walkers"}

    # the other configurations the comparison names, as extra keys (1 GPU): the 1731-electron
    # forward pass against the FP64 path, and the mixed batch in one CUDA graph
    if prec != "f64" and ws == 1 and not a.no_configs:
        q.close()
        q._ws.clear()
        del wsbuf, out
        torch.cuda.empty_cache()
        line["config4_forward"] = config4_forward(a, flush, e0, e1)
        torch.cuda.empty_cache()
        line["config2_precision_report"] = config2_precision_report(a, flush, e0, e1)
        torch.cuda.empty_cache()
        r5 = mixed_batch_run(1024, local, rank, prec, False, 3, 3, not a.no_cpu)
        line["config5_mixed_batch"] = {
            "workload": "1024 walkers each of the 158/434/1056/1731-electron systems, one CUDA graph per step",
            "walker_steps_per_s": 4096 / (r5["ms"] / 1e3), "ms_per_step": r5["ms"], "tiles": "library defaults",
            "clocks": r5["clocks"], "parity_vs_oracle": r5.get("parity"), "cpu_baseline": r5.get("cpu_baseline")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
