"""PyTorch-facing binding of libqmcgb: argument marshalling only.

Every step of the walker evaluation runs in the library's CUDA kernels;
torch provides device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
import zlib

import numpy as np
import torch

from ._lib import (PREC, DTYPE_F32, DTYPE_F64, DmcParams, EvalOut, Jastrow, QmcError, Segment, SystemDesc, Tiles,
                   WalkerState, check, lib)

__all__ = ["QmcSystem", "QmcBatch", "det_inverse", "LogPsi", "QmcError", "dmc_move", "dmc_weight",
           "srmc_reconfigure", "multidet_eval"]


def _stream(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def desc_crc32(arrays, eps):
    """CRC-32 key of a system description (the qmc_system_desc.crc32 rule):
    zlib's CRC-32 over the arrays' bytes in declaration order, then eps as an
    8-byte IEEE double in host byte order."""
    c = 0
    for a in arrays:
        c = zlib.crc32(memoryview(np.ascontiguousarray(a)).cast("B"), c)
    c = zlib.crc32(np.array([eps], dtype=np.float64).tobytes(), c)
    return c & 0xFFFFFFFF


def _req_cuda(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def system_desc(s):
    """qmc_system_desc of a synthetic system (host arrays kept alive in the
    returned list) with its CRC-32 key; returns (desc, keep, A dtype)."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        if a.ndim > 1:
            a = a.reshape(-1)
        keep.append(a)
        return C.c_void_p(a.ctypes.data)

    d = SystemDesc()
    d.n_atom = s.n_atom
    d.Z, d.Q = arr(s.Z, np.float64), arr(s.Q, np.float64)
    d.n_shell = s.n_shell
    d.shell_atom, d.shell_L = arr(s.shell_atom, np.int32), arr(s.shell_L, np.int32)
    d.shell_nprim, d.shell_pstart = arr(s.shell_nprim, np.int32), arr(s.shell_pstart, np.int32)
    d.n_prim = int(np.asarray(s.prim_gamma).size)
    d.prim_gamma, d.prim_coef = arr(s.prim_gamma, np.float64), arr(s.prim_coef, np.float64)
    d.n_ao = s.n_ao
    d.ao_shell, d.ao_pow, d.ao_scale = arr(s.ao_shell, np.int32), arr(s.ao_pow, np.int32), arr(s.ao_scale, np.float64)
    d.n_up, d.n_dn = s.n_up, s.n_dn
    f32 = np.asarray(s.A_up).dtype == np.float32
    a_dtype = np.float32 if f32 else np.float64
    d.a_dtype = DTYPE_F32 if f32 else DTYPE_F64
    d.A_up, d.A_dn = arr(s.A_up, a_dtype), arr(s.A_dn, a_dtype)
    d.eps = float(s.eps)
    # keep[] holds Z, Q, shell_atom, shell_L, shell_nprim, shell_pstart, prim_gamma, prim_coef,
    # ao_shell, ao_pow, ao_scale, A_up, A_dn: the order of the key
    d.crc32 = desc_crc32(keep, d.eps)
    return d, keep, a_dtype


class QmcSystem:
    """A molecular system resident on one GPU (qmc_system_load)."""

    def __init__(self, system, device: int = 0):
        s = system
        self.device = torch.device("cuda", device)
        self.n_up, self.n_dn, self.n_ao = int(s.n_up), int(s.n_dn), int(s.n_ao)
        self.N = self.n_up + self.n_dn
        self.n_atom, self.n_shell = int(s.n_atom), int(s.n_shell)
        d, self._keep, self.a_dtype = system_desc(s)
        h = C.c_void_p()
        check(lib().qmc_system_load(C.byref(d), device, C.byref(h)))
        self._h = h
        self._ws = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().qmc_system_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def shell_r2(self):
        out = np.zeros(self.n_shell, np.float64)
        check(lib().qmc_system_shell_r2(self._h, C.c_void_p(out.ctypes.data)))
        return out

    def set_jastrow(self, jastrow=None):
        """The Jastrow factor (qmc_system_set_jastrow): None switches it off, else a
        dict(a_par, a_anti, b_ee, a_en, b_en) with a_en, b_en scalars or [n_atom]."""
        if jastrow is None:
            check(lib().qmc_system_set_jastrow(self._h, C.byref(Jastrow(enabled=0))))
            return
        a_en = np.ascontiguousarray(np.broadcast_to(np.asarray(jastrow["a_en"], np.float64), (self.n_atom,)))
        b_en = np.ascontiguousarray(np.broadcast_to(np.asarray(jastrow["b_en"], np.float64), (self.n_atom,)))
        j = Jastrow(enabled=1, a_par=float(jastrow["a_par"]), a_anti=float(jastrow["a_anti"]),
                    b_ee=float(jastrow["b_ee"]), a_en=C.c_void_p(a_en.ctypes.data), b_en=C.c_void_p(b_en.ctypes.data))
        check(lib().qmc_system_set_jastrow(self._h, C.byref(j)))

    def crc32(self) -> int:
        """The system's CRC-32 key (qmc_system_crc32)."""
        c = C.c_uint32()
        check(lib().qmc_system_crc32(self._h, C.byref(c)))
        return int(c.value)

    def tiles(self):
        t = Tiles()
        check(lib().qmc_system_get_tiles(self._h, C.byref(t)))
        return {"gj_panel": t.gj_panel, "c15_walkers": t.c15_walkers,
                "a4_mode": {0: "fp64", 1: "float_float", 2: "tensor"}[t.a4_mode], "a4_kappa_max": t.a4_kappa_max,
                "c15_mode": {0: "float_float", 1: "tensor", 2: "cfree"}[t.c15_mode], "bw_walkers": t.bw_walkers,
                "wait_s": t.wait_s, "expire_walker": t.expire_walker, "expire_kernels": t.expire_kernels,
                "f64_kappa_max": t.f64_kappa_max}

    def set_tiles(self, gj_panel=None, c15_walkers=None, a4_mode=None, a4_kappa_max=None, c15_mode=None,
                  bw_walkers=None, wait_s=None, expire_walker=None, expire_kernels=None, f64_kappa_max=None):
        from ._lib import A4_MODE, C15_MODE
        cur = self.tiles()
        t = Tiles(gj_panel=gj_panel or cur["gj_panel"], c15_walkers=c15_walkers or cur["c15_walkers"],
                  a4_mode=A4_MODE[a4_mode or cur["a4_mode"]],
                  a4_kappa_max=a4_kappa_max if a4_kappa_max is not None else cur["a4_kappa_max"],
                  c15_mode=C15_MODE[c15_mode or cur["c15_mode"]], bw_walkers=bw_walkers or cur["bw_walkers"],
                  wait_s=wait_s if wait_s is not None else cur["wait_s"],
                  expire_walker=expire_walker if expire_walker is not None else cur["expire_walker"],
                  expire_kernels=expire_kernels if expire_kernels is not None else cur["expire_kernels"],
                  f64_kappa_max=f64_kappa_max if f64_kappa_max is not None else cur["f64_kappa_max"])
        check(lib().qmc_system_set_tiles(self._h, C.byref(t)))

    def set_mo(self, A_up, A_dn):
        """Replace the MO coefficients (qmc_system_set_mo); host arrays [n_ao, n_s]."""
        f32 = np.asarray(A_up).dtype == np.float32
        dt = np.float32 if f32 else np.float64
        au = np.ascontiguousarray(A_up, dtype=dt)
        ad = np.ascontiguousarray(A_dn, dtype=dt)
        assert au.shape == (self.n_ao, self.n_up) and ad.shape == (self.n_ao, self.n_dn)
        check(lib().qmc_system_set_mo(self._h, DTYPE_F32 if f32 else DTYPE_F64, C.c_void_p(au.ctypes.data),
                                      C.c_void_p(ad.ctypes.data)))

    def workspace_size(self, n_walk: int, precision: str = "f64") -> int:
        b = C.c_size_t()
        check(lib().qmc_workspace_size(self._h, n_walk, PREC[precision], C.byref(b)))
        return int(b.value)

    def workspace(self, n_walk: int, precision: str = "f64"):
        need = self.workspace_size(n_walk, precision)
        ws = self._ws.get(precision)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            self._ws[precision] = ws
        return ws

    def alloc_out(self, W: int, want_dinv: bool = False):
        dev, f64 = self.device, torch.float64
        o = dict(logpsi=torch.empty(W, dtype=f64, device=dev), sign=torch.empty(W, dtype=f64, device=dev),
                 logabs=torch.empty(W, 2, dtype=f64, device=dev),
                 drift=torch.empty(W, self.N, 3, dtype=f64, device=dev),
                 e_loc=torch.empty(W, dtype=f64, device=dev), e_parts=torch.empty(W, 4, dtype=f64, device=dev),
                 status=torch.empty(W, dtype=torch.int32, device=dev))
        if want_dinv:
            o["dinv"] = torch.empty(W, self.n_up ** 2 + self.n_dn ** 2, dtype=f64, device=dev)
        return o

    def eval(self, R, precision: str = "f64", want_dinv: bool = False, out=None, ws=None, stage_ms=None):
        """Steps a1..a6 (qmc_walkers_eval).  R: cuda f64 [W, N, 3].
        With stage_ms (a list), qmc_walkers_eval_timed is called instead and
        the per-stage device milliseconds are appended (blocking)."""
        W = int(R.shape[0])
        _req_cuda(R, torch.float64, "R", (W, self.N, 3))
        o = out if out is not None else self.alloc_out(W, want_dinv)
        if ws is None:
            ws = self.workspace(W, precision)
        eo = EvalOut(logpsi=_ptr(o["logpsi"]), sign=_ptr(o["sign"]), logabs=_ptr(o.get("logabs")),
                     drift=_ptr(o["drift"]), e_loc=_ptr(o["e_loc"]), e_parts=_ptr(o.get("e_parts")),
                     status=_ptr(o["status"]), dinv=_ptr(o.get("dinv")))
        if stage_ms is None:
            check(lib().qmc_walkers_eval(self._h, W, _ptr(R), PREC[precision], C.byref(eo), _ptr(ws), ws.numel(),
                                         _stream(self.device)))
        else:
            ms = (C.c_float * 8)()
            check(lib().qmc_walkers_eval_timed(self._h, W, _ptr(R), PREC[precision], C.byref(eo), _ptr(ws),
                                               ws.numel(), _stream(self.device), ms))
            stage_ms.append([float(x) for x in ms])
        return o

    def screen_ao(self, R, cap: int, want_B: bool = True):
        """Steps a1+a2 (qmc_screen_ao): cnt [W,N], idx [W,N,cap], B [W,N,5,cap]."""
        W = int(R.shape[0])
        _req_cuda(R, torch.float64, "R", (W, self.N, 3))
        cnt = torch.empty(W, self.N, dtype=torch.int32, device=self.device)
        idx = torch.full((W, self.N, cap), -1, dtype=torch.int32, device=self.device)
        B = torch.zeros(W, self.N, 5, cap, dtype=torch.float64, device=self.device) if want_B else None
        check(lib().qmc_screen_ao(self._h, W, _ptr(R), cap, _ptr(cnt), _ptr(idx), _ptr(B), _stream(self.device)))
        return cnt, idx, B

    def shell_masks(self, R):
        """Step a1 of the mixed path (qmc_shell_masks): active-shell bitmasks [W, N, words] (int32 view)."""
        W = int(R.shape[0])
        _req_cuda(R, torch.float64, "R", (W, self.N, 3))
        words = C.c_int(0)
        check(lib().qmc_shell_masks(self._h, 0, None, None, C.byref(words), _stream(self.device)))
        masks = torch.zeros(W, self.N, words.value, dtype=torch.int32, device=self.device)
        check(lib().qmc_shell_masks(self._h, W, _ptr(R), _ptr(masks), C.byref(words), _stream(self.device)))
        return masks

    def slater(self, R, precision: str = "f64", ws=None):
        """Steps a1..a3 (qmc_slater_matrices): per walker [5][n_up][n_up] then [5][n_dn][n_dn]."""
        W = int(R.shape[0])
        _req_cuda(R, torch.float64, "R", (W, self.N, 3))
        msz = self.n_up ** 2 + self.n_dn ** 2
        Cm = torch.empty(W, 5 * msz, dtype=torch.float64, device=self.device)
        if ws is None:
            ws = self.workspace(W, precision)
        check(lib().qmc_slater_matrices(self._h, W, _ptr(R), PREC[precision], _ptr(Cm), _ptr(ws), ws.numel(),
                                        _stream(self.device)))
        nu2 = self.n_up ** 2
        up = Cm[:, : 5 * nu2].reshape(W, 5, self.n_up, self.n_up)
        dn = Cm[:, 5 * nu2:].reshape(W, 5, self.n_dn, self.n_dn)
        return up, dn

    # --- the Monte Carlo step (qmc_dmc_step) --------------------------------
    def walker_state(self, W: int):
        """Device buffers of W walkers' state: R, drift, e_loc, logpsi, sign, status."""
        dev, f64 = self.device, torch.float64
        return dict(R=torch.empty(W, self.N, 3, dtype=f64, device=dev),
                    drift=torch.empty(W, self.N, 3, dtype=f64, device=dev),
                    e_loc=torch.empty(W, dtype=f64, device=dev), logpsi=torch.empty(W, dtype=f64, device=dev),
                    sign=torch.empty(W, dtype=f64, device=dev), status=torch.empty(W, dtype=torch.int32, device=dev))

    def init_state(self, R, precision: str = "f64"):
        """The state of walkers at positions R (one evaluation)."""
        W = int(R.shape[0])
        st = self.walker_state(W)
        st["R"].copy_(R)
        o = self.eval(st["R"], precision=precision)
        for k in ("drift", "e_loc", "logpsi", "sign", "status"):
            st[k].copy_(o[k])
        return st

    def dmc_workspace_size(self, n_walk: int, precision: str = "f64") -> int:
        b = C.c_size_t()
        check(lib().qmc_dmc_workspace_size(self._h, n_walk, PREC[precision], C.byref(b)))
        return int(b.value)

    def dmc_step(self, state_in, state_out, tau, e_trial, seed, step, precision="f64", stats=None, ws=None,
                 step_ptr=None, e_trial_ptr=None):
        """One fixed-node DMC step with constant population (qmc_dmc_step):
        state_in -> state_out (dicts of walker_state buffers).  stats: optional
        cuda f64 [4] (sum w, walkers with w > 0, sum w E_L, accepted moves)."""
        W = int(state_in["R"].shape[0])
        for k, t in list(state_in.items()) + list(state_out.items()):
            _req_cuda(t, torch.int32 if k == "status" else torch.float64, k)
        if ws is None:
            need = self.dmc_workspace_size(W, precision)
            ws = self._ws.get("dmc")
            if ws is None or ws.numel() < need:
                ws = torch.empty(need, dtype=torch.uint8, device=self.device)
                self._ws["dmc"] = ws
        si, so = _state_struct(state_in), _state_struct(state_out)
        p = DmcParams(tau=float(tau), e_trial=float(e_trial), seed=int(seed), step=int(step),
                      precision=PREC[precision], step_ptr=_ptr(step_ptr), e_trial_ptr=_ptr(e_trial_ptr))
        check(lib().qmc_dmc_step(self._h, W, C.byref(si), C.byref(so), C.byref(p), _ptr(stats), _ptr(ws),
                                 ws.numel(), _stream(self.device)))
        return state_out

    def backward_workspace_size(self, n_walk: int, precision: str = "mixed") -> int:
        b = C.c_size_t()
        check(lib().qmc_backward_workspace_size(self._h, n_walk, PREC[precision], C.byref(b)))
        return int(b.value)

    def backward(self, R, dinv, g, precision: str = "f64", ws=None):
        """Step a7: dA_up [n_ao, n_up], dA_dn [n_ao, n_dn], FP64 arrays.
        precision "f64": qmc_logpsi_backward; "mixed": the tensor-core
        contraction of qmc_logpsi_backward_ex (ws: optional uint8 scratch)."""
        W = int(R.shape[0])
        _req_cuda(R, torch.float64, "R", (W, self.N, 3))
        _req_cuda(dinv, torch.float64, "dinv", (W, self.n_up ** 2 + self.n_dn ** 2))
        _req_cuda(g, torch.float64, "g", (W,))
        dA_up = torch.empty(self.n_ao, self.n_up, dtype=torch.float64, device=self.device)
        dA_dn = torch.empty(self.n_ao, self.n_dn, dtype=torch.float64, device=self.device)
        if precision in ("f64", "f64_tca4"):
            check(lib().qmc_logpsi_backward(self._h, W, _ptr(R), _ptr(dinv), _ptr(g), _ptr(dA_up), _ptr(dA_dn),
                                            _stream(self.device)))
            return dA_up, dA_dn
        if ws is None:
            need = self.backward_workspace_size(W, precision)
            ws = self._ws.get("backward")
            if ws is None or ws.numel() < need:
                ws = torch.empty(need, dtype=torch.uint8, device=self.device)
                self._ws["backward"] = ws
        check(lib().qmc_logpsi_backward_ex(self._h, W, _ptr(R), _ptr(dinv), _ptr(g), PREC[precision],
                                           _ptr(dA_up), _ptr(dA_dn), _ptr(ws), ws.numel(), _stream(self.device)))
        return dA_up, dA_dn


def _eval_out_struct(o):
    return EvalOut(logpsi=_ptr(o["logpsi"]), sign=_ptr(o["sign"]), logabs=_ptr(o.get("logabs")),
                   drift=_ptr(o["drift"]), e_loc=_ptr(o["e_loc"]), e_parts=_ptr(o.get("e_parts")),
                   status=_ptr(o["status"]), dinv=_ptr(o.get("dinv")))


class QmcBatch:
    """Walkers of several systems evaluated together (qmc_batch_eval), and
    the same batch captured once as a CUDA graph (qmc_batch_graph_create)."""

    def __init__(self, parts, precision: str = "mixed", graph: bool = True):
        """parts: list of (QmcSystem, R) with R cuda f64 [W, N, 3]."""
        self.parts = parts
        self.precision = precision
        self.outs = [q.alloc_out(int(R.shape[0])) for q, R in parts]
        segs = (Segment * len(parts))()
        for i, ((q, R), o) in enumerate(zip(parts, self.outs)):
            _req_cuda(R, torch.float64, "R", (int(R.shape[0]), q.N, 3))
            segs[i].sys = q.handle
            segs[i].n_walk = int(R.shape[0])
            segs[i].R = _ptr(R)
            segs[i].out = _eval_out_struct(o)
        self._segs = segs
        b = C.c_size_t()
        check(lib().qmc_batch_workspace_size(segs, len(parts), PREC[precision], C.byref(b)))
        self.device = parts[0][0].device
        self.ws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=self.device)
        self._g = None
        if graph:
            h = C.c_void_p()
            check(lib().qmc_batch_graph_create(segs, len(parts), PREC[precision], _ptr(self.ws), self.ws.numel(),
                                               C.byref(h)))
            self._g = h

    def eval(self):
        check(lib().qmc_batch_eval(self._segs, len(self.parts), PREC[self.precision], _ptr(self.ws), self.ws.numel(),
                                   _stream(self.device)))
        return self.outs

    def launch(self):
        """One CUDA-graph launch of the whole batch on the current stream."""
        if self._g is None:
            raise RuntimeError("QmcBatch created without a graph")
        check(lib().qmc_graph_launch(self._g, _stream(self.device)))
        return self.outs

    def __del__(self):
        try:
            if self._g is not None and self._g.value:
                lib().qmc_graph_free(self._g)
        except Exception:
            pass


def multidet_eval(systems, coef, R, precision: str = "f64"):
    """Psi = e^J sum_K c_K Det_K (qmc_multidet_eval): systems = QmcSystem per determinant
    (same device, basis, nuclei, electrons, Jastrow), coef = host sequence of n_det
    coefficients, R cuda f64 [W, N, 3].  Returns the outputs of QmcSystem.eval
    (logabs NaN, no dinv)."""
    q0 = systems[0]
    W = int(R.shape[0])
    _req_cuda(R, torch.float64, "R", (W, q0.N, 3))
    K = len(systems)
    hs = (C.c_void_p * K)(*[q.handle.value for q in systems])
    cf = np.ascontiguousarray(coef, dtype=np.float64)
    assert cf.shape == (K,)
    b = C.c_size_t()
    check(lib().qmc_multidet_workspace_size(hs, K, W, PREC[precision], C.byref(b)))
    ws = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=q0.device)
    o = q0.alloc_out(W)
    eo = _eval_out_struct(o)
    check(lib().qmc_multidet_eval(hs, C.c_void_p(cf.ctypes.data), K, W, _ptr(R), PREC[precision], C.byref(eo),
                                  _ptr(ws), ws.numel(), _stream(q0.device)))
    return o


def _state_struct(st):
    return WalkerState(R=_ptr(st["R"]), drift=_ptr(st["drift"]), e_loc=_ptr(st["e_loc"]), logpsi=_ptr(st["logpsi"]),
                       sign=_ptr(st["sign"]), status=_ptr(st["status"]))


def dmc_move(R, drift, tau, seed, step, step_ptr=None):
    """Eq. (1) on cuda f64 [W, N, 3] (qmc_dmc_move); returns R'."""
    _req_cuda(R, torch.float64, "R")
    _req_cuda(drift, torch.float64, "drift", tuple(R.shape))
    Rn = torch.empty_like(R)
    check(lib().qmc_dmc_move(int(R.shape[0]), int(R.shape[1]), _ptr(R), _ptr(drift), float(tau), int(seed), int(step),
                             _ptr(step_ptr), _ptr(Rn), _stream(R.device)))
    return Rn


def dmc_weight(e_old, sign_old, status_old, e_new, sign_new, status_new, tau, e_trial):
    """Eq. (3) with the fixed-node rule (qmc_dmc_weight): (weight, accept)."""
    W = int(e_old.shape[0])
    for name, t in (("e_old", e_old), ("sign_old", sign_old), ("e_new", e_new), ("sign_new", sign_new)):
        _req_cuda(t, torch.float64, name, (W,))
    for name, t in (("status_old", status_old), ("status_new", status_new)):
        _req_cuda(t, torch.int32, name, (W,))
    w = torch.empty(W, dtype=torch.float64, device=e_old.device)
    acc = torch.empty(W, dtype=torch.int32, device=e_old.device)
    check(lib().qmc_dmc_weight(W, _ptr(e_old), _ptr(sign_old), _ptr(status_old), _ptr(e_new), _ptr(sign_new),
                               _ptr(status_new), float(tau), float(e_trial), None, _ptr(w), _ptr(acc),
                               _stream(e_old.device)))
    return w, acc


def srmc_reconfigure(weight, seed, step):
    """Sec. II.B draw (qmc_srmc_reconfigure): (idx int32 [W], stats f64 [4])."""
    W = int(weight.shape[0])
    _req_cuda(weight, torch.float64, "weight", (W,))
    idx = torch.empty(W, dtype=torch.int32, device=weight.device)
    stats = torch.zeros(4, dtype=torch.float64, device=weight.device)
    ws = torch.empty(max(8 * W, 8), dtype=torch.uint8, device=weight.device)
    check(lib().qmc_srmc_reconfigure(W, _ptr(weight), int(seed), int(step), None, _ptr(idx), _ptr(stats), _ptr(ws),
                                     ws.numel(), _stream(weight.device)))
    return idx, stats


def det_inverse(X):
    """Step a4 alone (qmc_det_inverse) on cuda f64 [batch, n, n]; X is consumed.
    Returns (logabs, sign, Dinv = X^-T, singular)."""
    _req_cuda(X, torch.float64, "X")
    b, n, n2 = X.shape
    assert n == n2
    dev = X.device
    Dinv = torch.empty_like(X)
    la = torch.empty(b, dtype=torch.float64, device=dev)
    sg = torch.empty(b, dtype=torch.float64, device=dev)
    sing = torch.empty(b, dtype=torch.int32, device=dev)
    check(lib().qmc_det_inverse(b, n, _ptr(X), _ptr(Dinv), _ptr(la), _ptr(sg), _ptr(sing), _stream(dev)))
    return la, sg, Dinv, sing


class LogPsi(torch.autograd.Function):
    """log|Psi| per walker with a hand-written adjoint for the MO coefficients.

    forward(A_up, A_dn, R, qsys, precision): qsys must hold the same A values
    (the library keeps its own copy); returns (logpsi, e_loc).  backward
    receives d L / d logpsi (E_L is treated as constant) and returns
    d L / d A_up, d L / d A_dn through qmc_logpsi_backward_ex, in FP64 after
    an FP64 forward and on the tensor cores after a mixed one.
    """

    @staticmethod
    def forward(ctx, A_up, A_dn, R, qsys, precision="f64"):
        o = qsys.eval(R, precision=precision, want_dinv=True)
        ctx.qsys = qsys
        ctx.precision = "f64" if precision in ("f64", "f64_tca4") else "mixed"
        ctx.save_for_backward(R, o["dinv"], o["status"])
        ctx.a_dtypes = (A_up.dtype, A_dn.dtype)
        ctx.mark_non_differentiable(o["e_loc"])
        return o["logpsi"], o["e_loc"]

    @staticmethod
    def backward(ctx, g_logpsi, g_eloc):
        R, dinv, status = ctx.saved_tensors
        g = torch.where(status == 0, g_logpsi.to(torch.float64), torch.zeros_like(g_logpsi, dtype=torch.float64))
        dA_up, dA_dn = ctx.qsys.backward(R, dinv, g.contiguous(), precision=ctx.precision)
        return dA_up.to(ctx.a_dtypes[0]), dA_dn.to(ctx.a_dtypes[1]), None, None, None
