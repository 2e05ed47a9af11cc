"""sg_apply_H_noalloc: the apply for callers that may not allocate device memory.

Such a caller (one whose device memory is all held by another allocator, or a
loop that cannot take a cudaMalloc's synchronisation) gets the same y = H_S x
as sg_apply_H, with the scratch taken from a fixed array in the library.  Each
case calls the no-alloc entry point twice in a row, with different inputs, and
compares both results with sg_apply_H's at the tolerances of the parity tests.
This file is collected last so that a run stopping at its first failure has
run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from paper_2111_13655_gb300 import synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # relative, as in the FP64 parity tests
MIXED_TOL = 5e-6   # relative, as in the mixed-precision parity tests


def rel_err(a, b):
    return float((a - b).abs().max() / b.abs().max())


CASES = [
    ("fp64", synth.workload_C2(), 8, FP64_TOL),
    ("mixed", synth.workload_C2(), 8, MIXED_TOL),
    ("fp64", synth.workload_C3(L=5), 8, FP64_TOL),
    ("mixed", synth.workload_C3(L=5), 3, MIXED_TOL),
]


@pytest.mark.parametrize("prec,p,nvec,tol", CASES, ids=[f"{c[0]}-D{c[1].D}L{c[1].L}-nvec{c[2]}" for c in CASES])
def test_noalloc_matches_sg_apply_H_on_two_calls(prec, p, nvec, tol):
    with sg.sg_create(p, prec) as ctx:
        for call, seed in enumerate((11, 12)):
            x = torch.from_numpy(synth.random_vectors(ctx.n_cs, nvec, seed)).cuda().contiguous().view(-1)
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            sg.sg_apply_H(ctx, x, y_ref, nvec)
            sg.sg_apply_H_noalloc(ctx, x, y, nvec)
            torch.cuda.synchronize()
            assert sg.sg_device_error(ctx) == 0
            assert torch.isfinite(y).all(), f"call {call}"
            assert rel_err(y, y_ref) <= tol, f"call {call}: {rel_err(y, y_ref)}"


def test_noalloc_rejects_requests_beyond_its_scratch():
    p = synth.workload_C3(L=7)  # N_cs = 50388
    with sg.sg_create(p, "mixed") as ctx:
        assert ctx.n_cs == 50388
        x = torch.zeros(11 * ctx.n_cs, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(sg.SgError) as ei:  # 11 * 50388 > 524272 elements
            sg.sg_apply_H_noalloc(ctx, x, y, 11)
        assert ei.value.status == sg.SG_EUNSUPPORTED and "524272" in str(ei.value)
    with sg.sg_create(synth.workload_C1(), "fp64") as ctx:
        x = torch.zeros(65 * ctx.n_cs, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(sg.SgError) as ei:  # more than 64 vectors
            sg.sg_apply_H_noalloc(ctx, x, y, 65)
        assert ei.value.status == sg.SG_EUNSUPPORTED
