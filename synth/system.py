"""Seeded synthetic inputs: peptide-like molecular systems and walker positions.

This module only *draws* inputs.  It holds none of the walker-evaluation
arithmetic (no screening, no AO/MO evaluation, no determinants, no energies):
both the CUDA path and the CPU oracle consume what it returns.

The paper's benchmark molecules (a copper complex, a beta-strand peptide,
PDB 1ZE7 and 1AMB; Section III, Table 1) and their Hartree-Fock orbitals are
not available, so systems are synthesised with the same shape statistics:

* heavy atoms (C, N, O) on a self-avoiding chain with 2.8 bohr bonds and
  110 +- 5 degree bond angles, uniform dihedrals;
* every H 2.0 bohr from a uniformly chosen heavy atom;
* Cartesian Gaussian basis (Section II.C, the AO form chi = x^nx y^ny z^nz g):
  3s2p1d = 15 AOs per heavy atom, 2s1p = 5 AOs per H;
* a dense MO coefficient matrix (Eq. "mo"), orthonormal columns from the QR
  factorisation of a seeded N(0,1) matrix -- the paper keeps A dense
  (Section IV.B "Sparsity");
* walkers: each nucleus receives Z electrons, the list is dealt alternately to
  the alpha and beta determinants, and each electron sits at its nucleus plus
  N(0, 1 bohr^2) per Cartesian component.

Contraction coefficients are normalised to unit self-overlap per Cartesian
component (closed-form Gaussian overlaps); this is basis-set data preparation,
done once here, and pinned by quadrature in the oracle tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ELEMENT_Z = {"H": 1, "C": 6, "N": 7, "O": 8}
# (L, n_primitives) per shell; n_primitives None = drawn in {1, 2, 3}.
# Heavy atoms: a core s shell with 8 primitives, then s, s, p, p, d (3s2p1d).
HEAVY_SHELLS = [(0, 8), (0, None), (0, None), (1, None), (1, None), (2, None)]
# Hydrogen: s, s, p (2s1p); no core shell.
H_SHELLS = [(0, None), (0, None), (1, None)]

BOND = 2.8          # bohr, heavy-heavy step
ANGLE_DEG = 110.0   # bond angle, +- ANGLE_JITTER
ANGLE_JITTER = 5.0
HEAVY_CLASH = 2.5   # a heavy atom may not come closer than this to a non-bonded heavy atom
H_BOND = 2.0
H_CLASH = 1.8
EXP_MIN, EXP_MAX = 0.1, 30.0
COEF_MIN, COEF_MAX = 0.1, 1.0
SCREEN_EPS = 1e-8


def cart_components(L: int):
    """Cartesian powers (nx, ny, nz) with nx+ny+nz = L, in a fixed order."""
    out = []
    for nx in range(L, -1, -1):
        for ny in range(L - nx, -1, -1):
            out.append((nx, ny, L - nx - ny))
    return out


def _dfact(n: int) -> int:
    """Double factorial with (-1)!! = 0!! = 1."""
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


@dataclass
class System:
    """A molecular system in the layout the C-ABI and the oracle both read.

    Arrays are host numpy arrays; AOs are ordered by shell, shells by atom.
    A_up / A_dn are [n_ao][n_s] row-major (row = AO, column = MO).
    """
    name: str
    seed: int
    Z: np.ndarray            # [n_atom] f64
    Q: np.ndarray            # [n_atom, 3] f64 (bohr)
    shell_atom: np.ndarray   # [n_shell] i32
    shell_L: np.ndarray      # [n_shell] i32
    shell_nprim: np.ndarray  # [n_shell] i32
    shell_pstart: np.ndarray # [n_shell] i32, offset into prim_* arrays
    prim_gamma: np.ndarray   # [n_prim] f64
    prim_coef: np.ndarray    # [n_prim] f64 (normalised contraction coefficient)
    ao_shell: np.ndarray     # [n_ao] i32
    ao_pow: np.ndarray       # [n_ao, 3] i32
    ao_scale: np.ndarray     # [n_ao] f64 (per-component normalisation ratio)
    n_up: int
    n_dn: int
    A_up: np.ndarray         # [n_ao, n_up], float64 or float32
    A_dn: np.ndarray         # [n_ao, n_dn]
    elec_atom: np.ndarray    # [N] i32: nucleus each electron is placed at
    eps: float = SCREEN_EPS
    meta: dict = field(default_factory=dict)

    @property
    def n_atom(self) -> int:
        return int(self.Z.shape[0])

    @property
    def n_shell(self) -> int:
        return int(self.shell_L.shape[0])

    @property
    def n_ao(self) -> int:
        return int(self.ao_shell.shape[0])

    @property
    def n_elec(self) -> int:
        return self.n_up + self.n_dn


def _unit(v):
    return v / np.linalg.norm(v)


def _place(a, b, c, bond, angle, dihedral):
    """Position of d with |cd| = bond, angle(b,c,d) = angle, dihedral(a,b,c,d)."""
    bc = _unit(c - b)
    n = np.cross(b - a, bc)
    if np.linalg.norm(n) < 1e-12:
        n = np.cross(bc, np.array([1.0, 0.0, 0.0]))
        if np.linalg.norm(n) < 1e-12:
            n = np.cross(bc, np.array([0.0, 1.0, 0.0]))
    n = _unit(n)
    m = np.cross(n, bc)
    d2 = np.array([-bond * math.cos(angle),
                   bond * math.sin(angle) * math.cos(dihedral),
                   bond * math.sin(angle) * math.sin(dihedral)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


def _chain(rng, n_heavy):
    pos = np.zeros((n_heavy, 3))
    if n_heavy > 1:
        pos[1] = [BOND, 0.0, 0.0]
    for i in range(2, n_heavy):
        for _ in range(10000):
            ang = math.radians(ANGLE_DEG + rng.uniform(-ANGLE_JITTER, ANGLE_JITTER))
            dih = rng.uniform(-math.pi, math.pi)
            a = pos[i - 3] if i >= 3 else pos[0] + np.array([0.0, 1.0, 0.0])
            p = _place(a, pos[i - 2], pos[i - 1], BOND, ang, dih)
            d = np.linalg.norm(pos[: i - 1] - p, axis=1)
            if np.all(d >= HEAVY_CLASH):
                pos[i] = p
                break
        else:
            raise RuntimeError("self-avoiding chain: no admissible position")
    return pos


def _hydrogens(rng, heavy_pos, n_h):
    placed = [p for p in heavy_pos]
    out = []
    for _ in range(n_h):
        for _ in range(10000):
            parent = int(rng.integers(0, len(heavy_pos)))
            v = rng.normal(size=3)
            p = heavy_pos[parent] + H_BOND * _unit(v)
            d = np.linalg.norm(np.asarray(placed) - p, axis=1)
            d[parent] = np.inf
            if np.all(d >= H_CLASH):
                out.append(p)
                placed.append(p)
                break
        else:
            raise RuntimeError("hydrogen placement: no admissible position")
    return np.asarray(out).reshape(n_h, 3)


def _element_basis(rng, shells):
    """Per-element shells: list of (L, gammas, raw coefficients)."""
    out = []
    for L, npr in shells:
        n = npr if npr is not None else int(rng.integers(1, 4))
        g = np.exp(rng.uniform(math.log(EXP_MIN), math.log(EXP_MAX), size=n))
        g = np.sort(g)[::-1].copy()
        c = rng.uniform(COEF_MIN, COEF_MAX, size=n)
        out.append((L, g, c))
    return out


def normalise_shell(L, gammas, coefs):
    """Contraction coefficients (primitive norm included) giving unit
    self-overlap for the (L,0,0) Cartesian component."""
    g = np.asarray(gammas, dtype=np.float64)
    c = np.asarray(coefs, dtype=np.float64)
    prim_norm = (2.0 * g / math.pi) ** 0.75 * (4.0 * g) ** (0.5 * L) / math.sqrt(_dfact(2 * L - 1))
    gi, gj = np.meshgrid(g, g, indexing="ij")
    ov = (2.0 * np.sqrt(gi * gj) / (gi + gj)) ** (L + 1.5)
    s = float(c @ ov @ c)
    return c * prim_norm / math.sqrt(s)


def component_scale(L, pw):
    nx, ny, nz = pw
    return math.sqrt(_dfact(2 * L - 1) / (_dfact(2 * nx - 1) * _dfact(2 * ny - 1) * _dfact(2 * nz - 1)))


def make_system(n_C, n_N, n_O, n_H, *, seed=None, open_shell=None, a_dtype=np.float64, name=None):
    """Synthetic peptide-like chain; seed defaults to the electron count."""
    n_elec = 6 * n_C + 7 * n_N + 8 * n_O + n_H
    if seed is None:
        seed = n_elec
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0])))
    heavy_types = np.array(["C"] * n_C + ["N"] * n_N + ["O"] * n_O)
    heavy_types = heavy_types[rng.permutation(len(heavy_types))]
    n_heavy = len(heavy_types)
    heavy_pos = _chain(rng, n_heavy)
    h_pos = _hydrogens(rng, heavy_pos, n_H)
    types = list(heavy_types) + ["H"] * n_H
    Q = np.concatenate([heavy_pos, h_pos], axis=0) if n_H else heavy_pos
    Z = np.array([float(ELEMENT_Z[t]) for t in types])

    basis_rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 1])))
    elem_basis = {}
    for el in ("C", "N", "O", "H"):
        elem_basis[el] = _element_basis(basis_rng, H_SHELLS if el == "H" else HEAVY_SHELLS)

    shell_atom, shell_L, shell_nprim, shell_pstart = [], [], [], []
    prim_gamma, prim_coef = [], []
    ao_shell, ao_pow, ao_scale = [], [], []
    for a, el in enumerate(types):
        for (L, g, c) in elem_basis[el]:
            s = len(shell_L)
            shell_atom.append(a)
            shell_L.append(L)
            shell_nprim.append(len(g))
            shell_pstart.append(len(prim_gamma))
            prim_gamma.extend(g.tolist())
            prim_coef.extend(normalise_shell(L, g, c).tolist())
            for pw in cart_components(L):
                ao_shell.append(s)
                ao_pow.append(pw)
                ao_scale.append(component_scale(L, pw))
    n_ao = len(ao_shell)

    # Electrons: nucleus a receives Z_a electrons, in atom order; even list
    # positions become alpha electrons, odd positions beta electrons.
    full = np.repeat(np.arange(len(types)), Z.astype(np.int64))
    elec_alpha = full[0::2]
    elec_beta = full[1::2]
    n_up, n_dn = len(elec_alpha), len(elec_beta)
    if open_shell is None:
        open_shell = n_up != n_dn

    mo_rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 2])))
    A_up, _ = np.linalg.qr(mo_rng.normal(size=(n_ao, n_up)))
    if open_shell:
        mo_rng2 = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed + 1, 2])))
        A_dn, _ = np.linalg.qr(mo_rng2.normal(size=(n_ao, n_dn)))
    else:
        A_dn = A_up[:, :n_dn].copy()
    A_up = np.ascontiguousarray(A_up, dtype=a_dtype)
    A_dn = np.ascontiguousarray(A_dn, dtype=a_dtype)

    return System(
        name=name or f"chain_{n_elec}e",
        seed=seed,
        Z=Z, Q=np.ascontiguousarray(Q, dtype=np.float64),
        shell_atom=np.asarray(shell_atom, dtype=np.int32),
        shell_L=np.asarray(shell_L, dtype=np.int32),
        shell_nprim=np.asarray(shell_nprim, dtype=np.int32),
        shell_pstart=np.asarray(shell_pstart, dtype=np.int32),
        prim_gamma=np.asarray(prim_gamma, dtype=np.float64),
        prim_coef=np.asarray(prim_coef, dtype=np.float64),
        ao_shell=np.asarray(ao_shell, dtype=np.int32),
        ao_pow=np.ascontiguousarray(np.asarray(ao_pow, dtype=np.int32).reshape(n_ao, 3)),
        ao_scale=np.asarray(ao_scale, dtype=np.float64),
        n_up=n_up, n_dn=n_dn, A_up=A_up, A_dn=A_dn,
        elec_atom=np.concatenate([elec_alpha, elec_beta]).astype(np.int32),
        meta={"types": types, "open_shell": bool(open_shell)},
    )


def make_walkers(system: System, n_walk: int, *, first=0, sigma=1.0):
    """[n_walk, N, 3] f64: walker j drawn from seed (system seed, j)."""
    N = system.n_elec
    R = np.empty((n_walk, N, 3), dtype=np.float64)
    centre = system.Q[system.elec_atom]
    for j in range(n_walk):
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([system.seed, 1000 + first + j])))
        R[j] = centre + sigma * rng.normal(size=(N, 3))
    return R


# The workload family: element counts per system (electrons 158/434/1056/1731).
CONFIGS = {
    "158e": dict(n_C=12, n_N=3, n_O=4, n_H=33),
    "434e": dict(n_C=32, n_N=9, n_O=10, n_H=99),
    "1056e": dict(n_C=80, n_N=22, n_O=24, n_H=230),
    "1731e": dict(n_C=130, n_N=36, n_O=40, n_H=379),
}
WALKERS = {"158e": 100, "434e": 4096, "1056e": 2048, "1731e": 512}


def config_system(key: str, **kw):
    spec = dict(CONFIGS[key])
    if key == "1731e":
        kw.setdefault("a_dtype", np.float32)
    return make_system(**spec, name=key, **kw)


def tiny_system(kind: str = "h2o_like", seed=7):
    """Small hand-sized systems for brute-force and parity checks."""
    if kind == "h2o_like":
        return make_system(0, 0, 1, 2, seed=seed, name="O1H2")
    if kind == "ch4_like":
        return make_system(1, 0, 0, 4, seed=seed, name="C1H4")
    if kind == "mini_chain":
        return make_system(3, 1, 1, 6, seed=seed, name="mini")
    raise ValueError(kind)


def excited_determinants(system: System, n_det: int, *, seed=7):
    """Determinants of a multi-determinant expansion built on `system`: the
    reference (its own MO columns) and single excitations of both spins --
    determinant k >= 1 replaces occupied MO column (n_s - k) of each spin with
    virtual orbital k - 1 of an orthonormal extension of the MO set (random
    vectors orthogonalised against the occupied columns, seeded).  Returns a
    list of Systems that differ only in A_up / A_dn."""
    import dataclasses
    rng = np.random.default_rng([int(system.seed), int(seed), 77])
    out = [system]

    def extend(A, m):
        A64 = np.asarray(A, dtype=np.float64)
        V = rng.normal(size=(A64.shape[0], m))
        V -= A64 @ (A64.T @ V)
        V, _ = np.linalg.qr(V)
        return V

    Vu = extend(system.A_up, n_det)
    Vd = extend(system.A_dn, n_det) if system.n_dn else np.zeros((system.n_ao, n_det))
    for k in range(1, n_det):
        Au = np.array(system.A_up, dtype=np.float64, copy=True)
        Au[:, system.n_up - k] = Vu[:, k - 1]
        Ad = np.array(system.A_dn, dtype=np.float64, copy=True)
        if system.n_dn:
            Ad[:, system.n_dn - k] = Vd[:, k - 1]
        dt = np.asarray(system.A_up).dtype
        out.append(dataclasses.replace(system, A_up=np.ascontiguousarray(Au, dtype=dt),
                                       A_dn=np.ascontiguousarray(Ad, dtype=dt), name=f"{system.name}_det{k}"))
    return out
