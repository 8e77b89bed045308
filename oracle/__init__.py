"""FP64 CPU oracle of the walker evaluation -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline /
reference leg may import this package.  It never touches the CUDA library and
the CUDA library never touches it; both read the same seeded inputs from
`synth`.

The arithmetic lives in `qmc_oracle.c` (plain loops, FP64, no FMA
contraction); this module compiles it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.c")
_SRC_MC = os.path.join(_HERE, "qmc_oracle_mc.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_SINGULAR_UP, ST_SINGULAR_DN, ST_NONFINITE = 1, 2, 4

_d = C.POINTER(C.c_double)
_i = C.POINTER(C.c_int)


class _OSys(C.Structure):
    _fields_ = [
        ("n_atom", C.c_int), ("Z", _d), ("Q", _d),
        ("n_shell", C.c_int), ("shell_atom", _i), ("shell_L", _i), ("shell_nprim", _i),
        ("shell_pstart", _i), ("prim_gamma", _d), ("prim_coef", _d),
        ("n_ao", C.c_int), ("ao_shell", _i), ("ao_pow", _i), ("ao_scale", _d),
        ("n_up", C.c_int), ("n_dn", C.c_int), ("A_up", _d), ("A_dn", _d),
        ("eps", C.c_double), ("R2", _d), ("unscreened", C.c_int),
        ("sh_ao0", _i), ("sh_nao", _i),
        ("jas_on", C.c_int), ("ja_par", C.c_double), ("ja_anti", C.c_double), ("jb_ee", C.c_double),
        ("ja_en", _d), ("jb_en", _d),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (idempotent)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_MC))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11",
               "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_MC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.oracle_shell_ranges.argtypes = [vp, _i, _i]
            L.oracle_shell_r2.argtypes = [vp, _d]
            L.oracle_eval.argtypes = [vp, C.c_int, _d, C.c_int, _d, _d, _d, _d, _d, _d,
                                      C.POINTER(C.c_uint), _d]
            L.oracle_eval_debug.argtypes = [vp, _d, C.c_int, _i, _i, _d, _d, _d, _d, _d, _d, _d,
                                            _d, C.POINTER(C.c_uint), _d]
            L.oracle_lu_inverse.argtypes = [C.c_int, _d, _d, _d, _d]
            L.oracle_logpsi_grad.argtypes = [vp, C.c_int, _d, _d, C.c_int, _d, _d]
            L.oracle_ao_points.argtypes = [vp, C.c_int, C.c_int, _d, _d]
            L.oracle_screen_points.argtypes = [vp, C.c_int, _d, C.c_int, _i, _i]
            L.oracle_vnn.argtypes = [vp]
            L.oracle_vnn.restype = C.c_double
            u64 = C.c_uint64
            pu64 = C.POINTER(u64)
            L.oracle_philox4x64.argtypes = [pu64, pu64, pu64]
            L.oracle_move_normals.argtypes = [C.c_int, C.c_int, C.c_int, u64, u64, _d]
            L.oracle_dmc_move.argtypes = [C.c_int, C.c_int, _d, _d, C.c_double, u64, u64, _d]
            L.oracle_dmc_weight.argtypes = [C.c_int, _d, _d, C.POINTER(C.c_uint), _d, _d, C.POINTER(C.c_uint),
                                            C.c_double, C.c_double, _d, C.POINTER(C.c_uint)]
            L.oracle_srmc.argtypes = [C.c_int, _d, u64, u64, _i, _d]
            _lib = L
    return _lib


def _p(a, t=_d):
    return a.ctypes.data_as(t)


class Oracle:
    """Oracle bound to one system.  Keeps its own FP64 copies of the inputs."""

    def __init__(self, system, unscreened: bool = False, jastrow=None):
        """jastrow: None, or dict(a_par, a_anti, b_ee, a_en [n_atom], b_en [n_atom]) -- the
        factor e^J with J = sum_{i<j} a r_ij / (1 + b_ee r_ij) (a = a_par for equal
        spins, a_anti otherwise) - sum_{i,a} a_en[a] r_ia / (1 + b_en[a] r_ia)."""
        s = system
        self.system = s
        self._keep = []

        def f64(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a

        def i32(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self._keep.append(a)
            return a

        self.n_up, self.n_dn, self.n_ao = s.n_up, s.n_dn, s.n_ao
        self.N = s.n_up + s.n_dn
        st = _OSys()
        st.n_atom = s.n_atom
        st.Z, st.Q = _p(f64(s.Z)), _p(f64(s.Q))
        st.n_shell = s.n_shell
        st.shell_atom, st.shell_L = _p(i32(s.shell_atom), _i), _p(i32(s.shell_L), _i)
        st.shell_nprim, st.shell_pstart = _p(i32(s.shell_nprim), _i), _p(i32(s.shell_pstart), _i)
        st.prim_gamma, st.prim_coef = _p(f64(s.prim_gamma)), _p(f64(s.prim_coef))
        st.n_ao = s.n_ao
        st.ao_shell, st.ao_pow = _p(i32(s.ao_shell), _i), _p(i32(s.ao_pow), _i)
        st.ao_scale = _p(f64(s.ao_scale))
        st.n_up, st.n_dn = s.n_up, s.n_dn
        st.A_up, st.A_dn = _p(f64(s.A_up)), _p(f64(s.A_dn))
        st.eps = float(s.eps)
        st.unscreened = 1 if unscreened else 0
        if jastrow is not None:
            st.jas_on = 1
            st.ja_par, st.ja_anti, st.jb_ee = (float(jastrow[k]) for k in ("a_par", "a_anti", "b_ee"))
            st.ja_en = _p(f64(np.broadcast_to(np.asarray(jastrow["a_en"], np.float64), (s.n_atom,))))
            st.jb_en = _p(f64(np.broadcast_to(np.asarray(jastrow["b_en"], np.float64), (s.n_atom,))))
        self._sh_ao0 = np.zeros(s.n_shell, np.int32)
        self._sh_nao = np.zeros(s.n_shell, np.int32)
        st.sh_ao0, st.sh_nao = _p(self._sh_ao0, _i), _p(self._sh_nao, _i)
        self._st = st
        L = lib()
        if L.oracle_shell_ranges(C.byref(st), st.sh_ao0, st.sh_nao) != 0:
            raise ValueError("AOs of a shell must be contiguous")
        self.R2 = np.zeros(s.n_shell, np.float64)
        L.oracle_shell_r2(C.byref(st), _p(self.R2))
        st.R2 = _p(self.R2)

    # --- full batch -----------------------------------------------------
    def eval(self, R, nthreads: int = 0, want_dinv: bool = False):
        R = np.ascontiguousarray(R, dtype=np.float64)
        W = R.shape[0]
        assert R.shape == (W, self.N, 3)
        out = dict(
            logpsi=np.zeros(W), sign=np.zeros(W), logabs=np.zeros((W, 2)),
            drift=np.zeros((W, self.N, 3)), e_loc=np.zeros(W), e_parts=np.zeros((W, 4)),
            status=np.zeros(W, np.uint32),
        )
        dsz = self.n_up ** 2 + self.n_dn ** 2
        dinv = np.zeros((W, dsz)) if want_dinv else None
        lib().oracle_eval(C.byref(self._st), W, _p(R), nthreads, _p(out["logpsi"]), _p(out["sign"]),
                          _p(out["logabs"]), _p(out["drift"]), _p(out["e_loc"]), _p(out["e_parts"]),
                          out["status"].ctypes.data_as(C.POINTER(C.c_uint)),
                          _p(dinv) if dinv is not None else None)
        if want_dinv:
            out["dinv_up"] = dinv[:, : self.n_up ** 2].reshape(W, self.n_up, self.n_up)
            out["dinv_dn"] = dinv[:, self.n_up ** 2:].reshape(W, self.n_dn, self.n_dn)
        return out

    # --- one walker with every intermediate --------------------------------
    def eval_debug(self, R1):
        R1 = np.ascontiguousarray(R1, dtype=np.float64).reshape(self.N, 3)
        cap = self.n_ao
        nu, nd = self.n_up, self.n_dn
        o = dict(cnt=np.zeros(self.N, np.int32), idx=np.full((self.N, cap), -1, np.int32),
                 B=np.zeros((self.N, 5, cap)), C=np.zeros(5 * nu * nu + 5 * nd * nd),
                 logabs=np.zeros(2), sign=np.zeros(2), drift=np.zeros((self.N, 3)),
                 parts=np.zeros(4), e_loc=np.zeros(1), dinv=np.zeros(nu * nu + nd * nd),
                 status=np.zeros(1, np.uint32), jastrow=np.zeros(1))
        rc = lib().oracle_eval_debug(C.byref(self._st), _p(R1), cap, _p(o["cnt"], _i), _p(o["idx"], _i),
                                     _p(o["B"]), _p(o["C"]), _p(o["logabs"]), _p(o["sign"]),
                                     _p(o["drift"]), _p(o["parts"]), _p(o["e_loc"]), _p(o["dinv"]),
                                     o["status"].ctypes.data_as(C.POINTER(C.c_uint)), _p(o["jastrow"]))
        assert rc == 0
        o["C_up"] = o["C"][: 5 * nu * nu].reshape(5, nu, nu)
        o["C_dn"] = o["C"][5 * nu * nu:].reshape(5, nd, nd)
        o["dinv_up"] = o["dinv"][: nu * nu].reshape(nu, nu)
        o["dinv_dn"] = o["dinv"][nu * nu:].reshape(nd, nd)
        o["e_loc"] = float(o["e_loc"][0])
        o["status"] = int(o["status"][0])
        o["jastrow"] = float(o["jastrow"][0])
        o["logpsi"] = float(o["logabs"].sum()) + o["jastrow"]
        return o

    def logpsi_grad(self, R, g, nthreads: int = 0):
        R = np.ascontiguousarray(R, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        W = R.shape[0]
        dA_up = np.zeros((self.n_ao, self.n_up))
        dA_dn = np.zeros((self.n_ao, self.n_dn))
        lib().oracle_logpsi_grad(C.byref(self._st), W, _p(R), _p(g), nthreads, _p(dA_up), _p(dA_dn))
        return dA_up, dA_dn

    def ao_points(self, mu, pts):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 5))
        lib().oracle_ao_points(C.byref(self._st), int(mu), pts.shape[0], _p(pts), _p(out))
        return out

    def screen_points(self, pts):
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        cap = self.n_ao
        cnt = np.zeros(pts.shape[0], np.int32)
        idx = np.full((pts.shape[0], cap), -1, np.int32)
        lib().oracle_screen_points(C.byref(self._st), pts.shape[0], _p(pts), cap, _p(cnt, _i), _p(idx, _i))
        return cnt, idx

    def vnn(self):
        return lib().oracle_vnn(C.byref(self._st))


def lu_inverse(M):
    """(logabs, sign, inverse) of a square FP64 matrix via the oracle's LU."""
    M = np.array(M, dtype=np.float64, order="C", copy=True)
    n = M.shape[0]
    la, sg = np.zeros(1), np.zeros(1)
    inv = np.zeros((n, n))
    rc = lib().oracle_lu_inverse(n, _p(M), _p(la), _p(sg), _p(inv))
    return float(la[0]), float(sg[0]), (inv if rc == 0 else None)


# --- the Monte Carlo step around the evaluation (qmc_oracle_mc.c) -----------
def philox4x64(ctr, key):
    """One Philox4x64-10 block: four uint64 outputs of counter ctr[4], key key[2]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    pu = C.POINTER(C.c_uint64)
    lib().oracle_philox4x64(c.ctypes.data_as(pu), k.ctypes.data_as(pu), out.ctypes.data_as(pu))
    return out


def move_normals(W, n_comp, seed, step, w0=0):
    """The move's Gaussian noise eta [W, n_comp] (Box-Muller on Philox)."""
    eta = np.zeros((W, n_comp))
    lib().oracle_move_normals(W, w0, n_comp, seed, step, _p(eta))
    return eta


def dmc_move(R, drift, tau, seed, step):
    """Eq. (1): R' = R + tau b + sqrt(tau) eta.  R, drift [W, N, 3]."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    drift = np.ascontiguousarray(drift, dtype=np.float64)
    out = np.zeros_like(R)
    lib().oracle_dmc_move(R.shape[0], R.shape[1], _p(R), _p(drift), tau, seed, step, _p(out))
    return out


def dmc_weight(e_old, sign_old, status_old, e_new, sign_new, status_new, tau, e_trial):
    """Eq. (3) with the fixed-node rule: (weight [W], accept [W])."""
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    u = lambda a: np.ascontiguousarray(a, dtype=np.uint32)
    e_old, sign_old, e_new, sign_new = f(e_old), f(sign_old), f(e_new), f(sign_new)
    status_old, status_new = u(status_old), u(status_new)
    W = e_old.shape[0]
    wt = np.zeros(W)
    acc = np.zeros(W, np.uint32)
    pu = C.POINTER(C.c_uint)
    lib().oracle_dmc_weight(W, _p(e_old), _p(sign_old), status_old.ctypes.data_as(pu), _p(e_new), _p(sign_new),
                            status_new.ctypes.data_as(pu), tau, e_trial, _p(wt), acc.ctypes.data_as(pu))
    return wt, acc


def srmc(weight, seed, step):
    """Sec. II.B reconfiguration: (idx [W] int32, sum of weights, alive count, all_zero)."""
    w = np.ascontiguousarray(weight, dtype=np.float64)
    W = w.shape[0]
    idx = np.zeros(W, np.int32)
    ws = np.zeros(2)
    rc = lib().oracle_srmc(W, _p(w), seed, step, _p(idx, _i), _p(ws))
    if rc < 0:
        raise MemoryError("oracle_srmc")
    return idx, float(ws[0]), int(ws[1]), rc == 1


def dmc_step(oracle, state, tau, e_trial, seed, step, nthreads=0):
    """One fixed-node DMC step with constant population (Eqs. 1-4, Sec. II.B),
    in the paper's order: move every walker (Eq. 1), evaluate the proposed
    positions (drift Eq. 2, E_L Eq. 4), keep or reject each move (fixed node),
    weigh it (Eq. 3), then draw the new population (reconfiguration).
    state: dict R [W,N,3], drift, e_loc, logpsi, sign, status of the current
    walkers.  Returns (new state, info) with info = weights, accept, idx,
    sum_w, sum_w_eloc (the weighted local energy of the generation, before the
    draw), alive."""
    R_new = dmc_move(state["R"], state["drift"], tau, seed, step)
    ev = oracle.eval(R_new, nthreads=nthreads)
    wt, acc = dmc_weight(state["e_loc"], state["sign"], state["status"], ev["e_loc"], ev["sign"], ev["status"],
                         tau, e_trial)
    a = acc.astype(bool)
    sel = {"R": np.where(a[:, None, None], R_new, state["R"]),
           "drift": np.where(a[:, None, None], ev["drift"], state["drift"]),
           "e_loc": np.where(a, ev["e_loc"], state["e_loc"]),
           "logpsi": np.where(a, ev["logpsi"], state["logpsi"]),
           "sign": np.where(a, ev["sign"], state["sign"]),
           "status": np.where(a, ev["status"], state["status"]).astype(np.uint32)}
    idx, sw, alive, _ = srmc(wt, seed, step)
    live = np.isfinite(wt) & (wt > 0.0)
    terms = np.where(live, wt * np.where(live, sel["e_loc"], 0.0), 0.0)
    swe = float(np.cumsum(terms)[-1]) if terms.size else 0.0      # summed in walker order
    new = {k: v[idx].copy() for k, v in sel.items()}
    return new, {"weight": wt, "accept": acc, "idx": idx, "sum_w": sw, "sum_w_eloc": swe, "alive": alive,
                 "R_proposed": R_new}


# --- multi-determinant expansion (Sec. II.C, Eq. psit) -----------------------
def multidet_eval(oracles, coef, R, nthreads=0):
    """Psi = sum_K c_K Psi_K with Psi_K = e^J Det_K,up Det_K,dn, from one oracle per
    determinant (same nuclei, basis and Jastrow; its own MO coefficients).
    By the definitions: log|Psi| = log|sum_K c_K s_K e^{L_K}|; drift = grad Psi / Psi =
    sum_K c_K Psi_K b_K / Psi; lap Psi / Psi = sum_K c_K Psi_K (lap Psi_K / Psi_K) / Psi, so
    T and E_L are the same weighted sums (V does not depend on K).  Determinants that are
    exactly singular contribute nothing."""
    evs = [o.eval(R, nthreads=nthreads) for o in oracles]
    W = R.shape[0]
    L = np.stack([e["logpsi"] for e in evs])                      # [K, W]
    S = np.stack([e["sign"] for e in evs])
    live = (S != 0) & np.isfinite(L)
    Lmax = np.max(np.where(live, L, -np.inf), axis=0)
    out = {k: np.zeros_like(v) for k, v in evs[0].items()}
    c = np.asarray(coef, dtype=np.float64)
    for w in range(W):
        terms = [c[k] * S[k, w] * math.exp(L[k, w] - Lmax[w]) if live[k, w] else 0.0 for k in range(len(evs))]
        tot = math.fsum(terms)
        out["status"][w] = 0
        if not np.isfinite(Lmax[w]) or tot == 0.0:
            out["logpsi"][w], out["sign"][w] = -np.inf, 0.0
            out["status"][w] = ST_SINGULAR_UP | ST_SINGULAR_DN
            out["drift"][w], out["e_loc"][w] = np.nan, np.nan
            out["e_parts"][w] = np.nan
            continue
        om = [t / tot for t in terms]
        out["logpsi"][w] = Lmax[w] + math.log(abs(tot))
        out["sign"][w] = 1.0 if tot > 0 else -1.0
        out["drift"][w] = sum(om[k] * evs[k]["drift"][w] for k in range(len(evs)) if live[k, w])
        out["e_loc"][w] = math.fsum(om[k] * evs[k]["e_loc"][w] for k in range(len(evs)) if live[k, w])
        out["e_parts"][w, 0] = math.fsum(om[k] * evs[k]["e_parts"][w, 0] for k in range(len(evs)) if live[k, w])
        out["e_parts"][w, 1:] = evs[0]["e_parts"][w, 1:]
        out["logabs"][w] = np.nan
    return out
