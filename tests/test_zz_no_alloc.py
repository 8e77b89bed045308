"""qmc_walkers_eval_static: the walker evaluation for callers that cannot
allocate device memory (code under a memory manager that owns the device,
latency-critical loops that must not hit cudaMalloc's implicit
synchronisation, plug-ins whose host forbids driver allocations).  Its scratch
is a fixed array inside the library instead of a caller workspace.

Checked through the C ABI against qmc_walkers_eval with a caller workspace,
on two calls in a row (the array keeps the previous call's contents), with
batches that need several passes through the array (checked against the
workspace size): the FP64 path to
1e-10 relative; the mixed path within its parity tolerances (log|Psi| 1e-6,
E_L 1e-5 relative, drift 1e-4 normwise), because its tensor-core products
group walkers into tiles by pass and their last accumulator rounds at ~2^-45
of C1 depending on that grouping (amplified near nodal surfaces).
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _eval_static(q, R, precision, want_dinv):
    from paper_1209_6630_gb300._lib import PREC, EvalOut, check, lib
    o = q.alloc_out(R.shape[0], want_dinv=want_dinv)
    p = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    eo = EvalOut(logpsi=p(o["logpsi"]), sign=p(o["sign"]), logabs=p(o["logabs"]), drift=p(o["drift"]),
                 e_loc=p(o["e_loc"]), e_parts=p(o["e_parts"]), status=p(o["status"]), dinv=p(o.get("dinv")))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    check(lib().qmc_walkers_eval_static(q.handle, R.shape[0], p(R), PREC[precision], C.byref(eo), stream))
    return o


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_static_scratch_matches_caller_workspace_twice(precision):
    from paper_1209_6630_gb300 import QmcSystem
    from synth import config_system, make_walkers
    s = config_system("158e")
    q = QmcSystem(s, 0)
    W = 400
    # several passes through the fixed array in both precisions: the batch needs more than
    # twice its size of scratch
    assert q.workspace_size(W, precision) > 2 * (64 << 20), q.workspace_size(W, precision)
    for call, first in enumerate((5000, 6000)):            # two calls in a row, different walkers
        R = torch.from_numpy(make_walkers(s, W, first=first)).cuda()
        got = _eval_static(q, R, precision, want_dinv=(call == 1))
        ref = q.eval(R, precision=precision, want_dinv=(call == 1))
        torch.cuda.synchronize()
        assert torch.equal(got["status"], ref["status"])
        assert torch.equal(got["sign"], ref["sign"])
        lp_g, lp_r = got["logpsi"].cpu().numpy(), ref["logpsi"].cpu().numpy()
        el_g, el_r = got["e_loc"].cpu().numpy(), ref["e_loc"].cpu().numpy()
        dr_g, dr_r = got["drift"].cpu().numpy(), ref["drift"].cpu().numpy()
        if precision == "f64":
            assert np.abs(lp_g - lp_r).max() <= 1e-10 * np.abs(lp_r).max(), call
            assert np.abs(el_g - el_r).max() <= 1e-10 * np.abs(el_r).max(), call
            assert np.abs(dr_g - dr_r).max() <= 1e-10 * np.abs(dr_r).max(), call
        else:
            assert np.abs(lp_g - lp_r).max() < 1e-6, call
            assert (np.abs(el_g - el_r) / np.abs(el_r)).max() < 1e-5, call
            assert np.abs(dr_g - dr_r).max() <= 1e-4 * np.abs(dr_r).max(), call
        if call == 1:
            a, b = got["dinv"].cpu().numpy(), ref["dinv"].cpu().numpy()
            tol = 1e-10 if precision == "f64" else 1e-6
            assert np.abs(a - b).max() <= tol * np.abs(b).max()


def test_static_scratch_rejects_oversized_system():
    from paper_1209_6630_gb300 import QmcSystem
    from paper_1209_6630_gb300._lib import PREC, EvalOut, lib
    from synth import config_system, make_walkers
    s = config_system("1731e")           # one FP64 walker needs ~72 MB of scratch
    q = QmcSystem(s, 0)
    R = torch.from_numpy(make_walkers(s, 1)).cuda()
    o = q.alloc_out(1)
    p = lambda t: C.c_void_p(t.data_ptr())
    eo = EvalOut(logpsi=p(o["logpsi"]), sign=p(o["sign"]), logabs=None, drift=p(o["drift"]),
                 e_loc=p(o["e_loc"]), e_parts=None, status=p(o["status"]), dinv=None)
    rc = lib().qmc_walkers_eval_static(q.handle, 1, p(R), PREC["f64"], C.byref(eo), None)
    assert rc == -4                      # QMC_ERR_CAPACITY
    assert b"fixed" in lib().qmc_last_error()
