"""Hand-built systems for closed-form pins (no generator randomness)."""
import numpy as np

from synth.system import System, cart_components


def one_atom_system(Z, shells, n_up, n_dn, A_up, A_dn=None, Q=(0.0, 0.0, 0.0), eps=1e-8,
                    coefs_raw=True):
    """shells: list of (L, gammas, coefs); coefficients are used as given.
    Every Cartesian component gets scale 1 (closed forms below assume it)."""
    shell_atom, shell_L, shell_nprim, shell_pstart = [], [], [], []
    pg, pc, ao_shell, ao_pow, ao_scale = [], [], [], [], []
    for s, (L, g, c) in enumerate(shells):
        shell_atom.append(0); shell_L.append(L); shell_nprim.append(len(g))
        shell_pstart.append(len(pg)); pg.extend(g); pc.extend(c)
        for pw in cart_components(L):
            ao_shell.append(s); ao_pow.append(pw); ao_scale.append(1.0)
    n_ao = len(ao_shell)
    A_up = np.asarray(A_up, dtype=np.float64).reshape(n_ao, n_up)
    A_dn = np.zeros((n_ao, 0)) if A_dn is None else np.asarray(A_dn, dtype=np.float64).reshape(n_ao, n_dn)
    return System(name="one_atom", seed=0, Z=np.array([float(Z)]), Q=np.array([Q], dtype=np.float64),
                  shell_atom=np.array(shell_atom, np.int32), shell_L=np.array(shell_L, np.int32),
                  shell_nprim=np.array(shell_nprim, np.int32), shell_pstart=np.array(shell_pstart, np.int32),
                  prim_gamma=np.array(pg, np.float64), prim_coef=np.array(pc, np.float64),
                  ao_shell=np.array(ao_shell, np.int32), ao_pow=np.array(ao_pow, np.int32).reshape(n_ao, 3),
                  ao_scale=np.array(ao_scale, np.float64), n_up=n_up, n_dn=n_dn,
                  A_up=np.ascontiguousarray(A_up), A_dn=np.ascontiguousarray(A_dn),
                  elec_atom=np.zeros(n_up + n_dn, np.int32), eps=eps)
