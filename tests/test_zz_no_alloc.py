"""sg_apply_H_noalloc: the apply for callers that may not allocate device memory.

Such a caller (one whose device memory is all held by another allocator, or a
loop that cannot take a cudaMalloc's synchronisation) gets the same y = H_S x
as sg_apply_H, with the scratch taken from a fixed array in the library.  Each
case calls the no-alloc entry point twice in a row, with different inputs.  Both
entry points run the same kernels and the same exact fixed-point sum, so the
results must be bitwise equal: any stale accumulator word left by an
incomplete clear of the shared scratch would show.
This file is collected last so that a run stopping at its first failure has
run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from paper_2111_13655_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("fp64", synth.workload_C2(), 8),
    ("mixed", synth.workload_C2(), 8),
    ("fp64", synth.workload_C3(L=5), 8),
    ("mixed", synth.workload_C3(L=5), 3),
    # beyond the FP64 element limit, within the mixed one (one word per element)
    ("mixed", synth.workload_C3(L=7), 12),
]


@pytest.mark.parametrize("prec,p,nvec", CASES, ids=[f"{c[0]}-D{c[1].D}L{c[1].L}-nvec{c[2]}" for c in CASES])
def test_noalloc_equals_sg_apply_H_bitwise_on_two_calls(prec, p, nvec):
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
            assert torch.equal(y, y_ref), f"call {call}: max |diff| {float((y - y_ref).abs().max())}"


def test_noalloc_rejects_requests_beyond_its_scratch():
    p = synth.workload_C3(L=7)  # N_cs = 50388
    with sg.sg_create(p, "fp64") as ctx:
        assert ctx.n_cs == 50388
        x = torch.zeros(11 * ctx.n_cs, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(sg.SgError) as ei:  # FP64: 11 * 50388 > 524272 elements
            sg.sg_apply_H_noalloc(ctx, x, y, 11)
        assert ei.value.status == sg.SG_EUNSUPPORTED and "524272" in str(ei.value)
    with sg.sg_create(p, "mixed") as ctx:
        x = torch.zeros(42 * ctx.n_cs, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(sg.SgError) as ei:  # mixed: 42 * 50388 > 2097088 elements
            sg.sg_apply_H_noalloc(ctx, x, y, 42)
        assert ei.value.status == sg.SG_EUNSUPPORTED and "2097088" in str(ei.value)
    with sg.sg_create(synth.workload_C1(), "fp64") as ctx:
        x = torch.zeros(65 * ctx.n_cs, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(sg.SgError) as ei:  # more than 64 vectors
            sg.sg_apply_H_noalloc(ctx, x, y, 65)
        assert ei.value.status == sg.SG_EUNSUPPORTED
