"""hps_condense_host: the condensation with host buffers, copies overlapped
with the launches in chunks, must give exactly what hps_condense gives on
device buffers (each leaf is condensed by the same code in one CTA)."""

import numpy as np
import pytest
import torch

from gpu_cases import gpu_inputs
from paper_2211_14969_b300 import hps
from paper_2211_14969_b300 import workloads as WL

pytestmark = pytest.mark.gpu


def device_reference(plan, coef, f, m, prec):
    out = plan.condense(coef, f, m=m, prec=prec, tol=1e-12, kmax=6)
    torch.cuda.synchronize()
    return {k: v.cpu() for k, v in out.items()}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("chunks", [1, 3, 8])
def test_host_call_equals_device_call(prec, chunks):
    """Mixed orders (12..32) on a 16 x 8 tiling, two loads: bit-identical
    S, T, h, W and info for 1, 3 and 8 chunks."""
    w = WL.uneven(nx=16, ny=8, m=2)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    ref = device_reference(plan, coef, f, 2, prec)
    out = plan.condense_host(coef.cpu().pin_memory(), f.cpu().pin_memory(), m=2, prec=prec, tol=1e-12, kmax=6,
                             chunks=chunks)
    torch.cuda.synchronize()
    for k in ("S", "T", "h", "W", "info"):
        assert torch.equal(out[k], ref[k]), k
    plan.close()


def test_repeated_calls_pageable_buffers_and_no_S():
    """Two calls in a row on one plan (the staging buffers are reused),
    pageable host memory, S not stored."""
    w = WL.bumps(p=14, nx=8, ny=8, kappa=40.0, seed=3, m=1)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    ref = device_reference(plan, coef, f, 1, "fp32")
    coef_h, f_h = coef.cpu(), f.cpu()
    for _ in range(2):
        out = plan.condense_host(coef_h, f_h, m=1, prec="fp32", tol=1e-12, kmax=6, store_S=False, chunks=5)
        torch.cuda.synchronize()
        assert "S" not in out
        for k in ("T", "h", "W", "info"):
            assert torch.equal(out[k], ref[k]), k
    plan.close()


def test_host_call_argument_errors():
    w = WL.bumps(p=8, nx=2, ny=2, kappa=5.0, seed=1, m=1)
    plan = hps.Plan(w.p, w.boxes(), w.kappa)
    coef, f, _ = gpu_inputs(w, plan)
    with pytest.raises(hps.HpsError):
        plan.condense_host(coef.cpu(), f.cpu(), m=1, chunks=65)
    with pytest.raises(hps.HpsError):
        plan.condense_host(coef.cpu(), f.cpu(), m=1, chunks=-1)
    with pytest.raises(ValueError):
        plan.condense_host(coef, f, m=1)          # device tensors
    plan.close()
