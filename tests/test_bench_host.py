"""Host logic of bench.py that needs no GPU: the per-step launch count it
reports as `gpu_launches`, checked against the ncu launch lists of one
evaluation of the 1056-electron system (528 + 528 electrons, 2048 walkers),
and the traffic table lookup."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Sys:
    """The attributes launches_per_step reads from a loaded system."""

    def __init__(self, n_up, n_dn, tiles):
        self.n_up, self.n_dn, self.N = n_up, n_dn, n_up + n_dn
        self._t = tiles

    def tiles(self):
        return dict(self._t)


def _tiles(**kw):
    t = {"gj_panel": 16, "c15_walkers": 4, "a4_mode": "tensor", "a4_kappa_max": 1e8, "c15_mode": "tensor",
         "bw_walkers": 8}
    t.update(kw)
    return t


def test_launches_tensor_a4_1056e():
    # masks 1, C1..C5 9 x (producer + MMA) (batches of 118 electrons), a4 init 1 + 17 x (panel +
    # update) + final 1, FP64 recomputation: list 1, C1 rows 1, 33 x (panel + update), final 1,
    # FP64 pass 1; energy 1
    q = _Sys(528, 528, _tiles())
    assert bench.launches_per_step(q, "mixed", 2048) == 1 + 18 + 1 + 34 + 1 + 1 + 1 + 66 + 1 + 1 + 1


def test_launches_cfree_1056e():
    # the C-free default: C1 alone in 9 x (producer + MMA), then the D^-1 row exponents 1 and
    # v / drift / Laplacian in 4 launches of 264 electrons; a4 and the rest as above
    q = _Sys(528, 528, _tiles(c15_mode="cfree"))
    assert bench.launches_per_step(q, "mixed", 2048) == 1 + 18 + 1 + 4 + 1 + 34 + 1 + 1 + 1 + 66 + 1 + 1 + 1


def test_launches_cfree_1056e_fewer_tiles():
    # 512 walkers (4 tiles): C1 in 33 batches of 32 electrons, v in 4 batches of up to 264;
    # 128 walkers (one tile): C1 in 66 batches of 16, v in 17 batches of up to 64
    q = _Sys(528, 528, _tiles(c15_mode="cfree"))
    assert bench.launches_per_step(q, "mixed", 512) == 1 + 66 + 1 + 4 + 1 + 34 + 1 + 1 + 1 + 66 + 1 + 1 + 1
    assert bench.launches_per_step(q, "mixed", 128) == 1 + 132 + 1 + 17 + 1 + 34 + 1 + 1 + 1 + 66 + 1 + 1 + 1


def test_launches_float_float_a4_1056e():
    # as above with one float-float Gauss-Jordan launch in place of the 36 tensor-core a4 launches
    q = _Sys(528, 528, _tiles(a4_mode="float_float"))
    assert bench.launches_per_step(q, "mixed", 2048) == 1 + 18 + 1 + 1 + 1 + 66 + 1 + 1 + 1


def test_launches_fp64_path():
    q = _Sys(528, 528, _tiles())
    assert bench.launches_per_step(q, "f64", 2048) == 3


def test_traffic_lookup_requires_matching_source():
    # the a4 line is used only while its source hash matches; an unknown kernel gives None
    assert bench.kernel_traffic("no_such_kernel", "1056e") is None
    v = bench.kernel_traffic("k_gj_ff+k_gj", "1056e")
    assert v is None or v > 1e10


def test_bench_calls_only_defined_or_imported_names():
    """Every plain function name bench.py calls is defined in it, imported, or a builtin
    (the GPU legs only run on the GPU machine, so a missing helper would surface there first)."""
    import ast
    import builtins
    src = open(os.path.join(ROOT, "bench.py")).read()
    tree = ast.parse(src)
    known = {n.name for n in ast.walk(tree) if isinstance(n, (ast.FunctionDef, ast.ClassDef))}
    for n in ast.walk(tree):
        if isinstance(n, (ast.Import, ast.ImportFrom)):
            known |= {(a.asname or a.name).split(".")[0] for a in n.names}
        if isinstance(n, ast.arg):                  # parameters (a callable passed in)
            known.add(n.arg)
        if isinstance(n, ast.Assign):               # local callables (lambdas, aliases)
            known |= {t.id for t in n.targets if isinstance(t, ast.Name)}
    calls = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    missing = sorted(c for c in calls if c not in known and not hasattr(builtins, c))
    assert not missing, missing
