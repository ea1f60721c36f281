"""hps_condense_noalloc: the allocation-free FP64 condensation entry point.

It exists for callers that cannot call cudaMalloc when they condense (a host
framework that owns all device memory through its own pool, or a
latency-critical loop where an allocation could stall or fail).  Its
scratch is a fixed array inside the library, shared by every call on a
device, so this test checks two calls in a row against the plan-based
hps_condense on the same inputs, through the C ABI.  It lives in its own
file, collected last, and passes alone or after the other tests.
"""

import ctypes

import numpy as np
import pytest
import torch

from gpu_cases import gpu_inputs
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 parity bar of the other GPU tests


def _noalloc(lib, n_leaves, p, kappa, box, coef, f, m, out, stream):
    lib.hps_condense_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double] + [ctypes.c_void_p] * 10
    lib.hps_condense_noalloc.restype = ctypes.c_int
    ptr = lambda t: ctypes.c_void_p(0 if t is None else t.data_ptr())
    return lib.hps_condense_noalloc(n_leaves, p, kappa, ptr(box), ptr(coef), ptr(f), m, ptr(out["S"]),
                                    ptr(out["T"]), ptr(out["h"]), ptr(out["W"]), ptr(out["info"]),
                                    ctypes.c_void_p(stream.cuda_stream))


def _relerr(a, b, n):
    a = a.reshape(n, -1)
    b = b.reshape(n, -1)
    return float(((a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-300)).max())


class _Leaves:
    """The first n leaves of a workload, as their own batch."""

    def __init__(self, w, n):
        self.m, self.kappa, self.n_leaves = w.m, w.kappa, n
        self.p = w.p[:n]
        self.box = np.ascontiguousarray(w.boxes()[:n])
        self.coefficients, self.body_load = w.coefficients, w.body_load

    def boxes(self):
        return self.box


@pytest.mark.parametrize("which", ["p12_8x8", "p20_bench_leaves", "psi_p14_4x4"])
def test_noalloc_matches_plan_path_two_calls(which):
    lib = hps.load_library()
    if which == "p12_8x8":
        w = WL.bumps(p=12, nx=8, ny=8, kappa=60.0, seed=13, m=1)
    elif which == "psi_p14_4x4":   # mixed term c12 != 0: the corner weights of the scratch tables
        w = WL.psi_curved(p=14, nx=4, ny=4, kappa=10.0, m=1)
    else:   # 40 leaves of the 64 x 64, p = 20, kappa = 200 workload
        w = _Leaves(WL.bumps_p20(), 40)
    p = int(w.p[0])
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    ref = plan.condense(coef, f, m=1, prec="fp64")
    box = torch.from_numpy(np.ascontiguousarray(w.boxes())).cuda()
    stream = torch.cuda.current_stream()
    n = w.n_leaves
    for call in range(2):
        out = {k: torch.full_like(v, float("nan") if v.dtype == torch.float64 else -7) for k, v in ref.items()}
        st = _noalloc(lib, n, p, w.kappa, box, coef, f, 1, out, stream)
        assert st == hps.HPS_OK, lib.hps_last_error(None)
        torch.cuda.synchronize()
        assert (out["info"] == 0).all()
        for k in ("S", "T", "h", "W"):
            err = _relerr(out[k], ref[k], n)
            assert err <= TOL, (call, k, err)


def test_noalloc_rejects_oversized_call():
    lib = hps.load_library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = {"S": None, "T": dummy, "h": dummy, "W": None, "info": info}
    stream = torch.cuda.current_stream()
    # 800k leaves of tables alone exceed the 32 MiB scratch: rejected before any launch
    st = _noalloc(lib, 800_000, 10, 1.0, dummy, dummy, None, 0, out, stream)
    assert st == hps.HPS_ERR_ARG
    assert b"scratch" in lib.hps_last_error(None)
    # p = 42 with many body loads: one leaf's workspace alone is too large
    st = _noalloc(lib, 1, 42, 1.0, dummy, dummy, dummy, 1000, out, stream)
    assert st == hps.HPS_ERR_ARG
