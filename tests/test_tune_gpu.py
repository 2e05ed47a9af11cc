"""sg_tune: measured choice of the fast path's slicing target.

After tuning, the context must still compute H_S within the parity
tolerances (FP64 1e-12 norm-wise and element-wise against the oracles, mixed
as in tests/helpers.py), repeatably to the bit, and report which target it
kept."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from oracle import galerkin
from oracle import oracle as orc
from paper_2111_13655_gb300 import synth

from helpers import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["D=6 L=8 nq=l+1 (literal oracle)", "D=12 L=6 nq=l+2 (Galerkin)"])
def test_tuned_context_keeps_parity_and_determinism(prec, which):
    if which.startswith("D=6"):
        p = synth.workload_C2()
        ref_of = lambda x: orc.apply_H(p, x)
    else:
        p = synth.workload_C3(L=6)
        ref_of = lambda x: galerkin.apply_H(p, x)
    nvec = 4
    with sg.sg_create(p, prec) as ctx:
        xn = synth.random_vectors(ctx.n_cs, nvec, 5)
        x = torch.from_numpy(xn).cuda().contiguous().view(-1)
        vt, ms = sg.sg_tune(ctx, nvec)
        assert vt in (1, 2, 4) and ms > 0.0
        plan = sg.sg_tune_plan(ctx)
        assert plan["slice_vt"] == vt and plan["warp_vt"] in (1, 2, 4)
        assert plan["smem_kb"] in ((52, 70, 104) if prec == "mixed" else (70, 104))
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        sg.sg_apply_H(ctx, x, y1, nvec)
        sg.sg_apply_H(ctx, x, y2, nvec)
        torch.cuda.synchronize()
        assert sg.sg_device_error(ctx) == 0
        assert torch.equal(y1, y2)
        assert_parity(y1.view(nvec, -1).cpu().numpy(), ref_of(xn), prec, which)


def test_generic_path_has_nothing_to_tune():
    p = synth.polynomial_problem(3, 4, [0.9, 1.1, 1.0],
                                 [(0.05, [(0, 1), (1, 1), (2, 1)]), (0.2, [(0, 2), (1, 2)])])
    with sg.sg_create(p, "fp64") as ctx:
        assert sg.sg_tune(ctx, 2) == (0, 0.0)


def test_batch_made_before_tuning_refuses_until_recreated():
    p = synth.workload_C2()
    with sg.sg_create(p, "mixed") as ctx:
        x = torch.from_numpy(synth.random_vectors(ctx.n_cs, 2, 3)).cuda().contiguous().view(-1)
        y0, y1 = torch.empty_like(x), torch.empty_like(x)
        b = sg.sg_batch_create([ctx])
        sg.sg_tune(ctx, 2)
        with pytest.raises(sg.SgError) as ei:
            sg.sg_apply_H_batch(b, x, y0, 2)
        assert ei.value.status == sg.SG_EINVAL and "recreate" in str(ei.value)
        sg.sg_batch_destroy(b)
        b = sg.sg_batch_create([ctx])
        sg.sg_apply_H_batch(b, x, y0, 2)
        sg.sg_apply_H(ctx, x, y1, 2)
        torch.cuda.synchronize()
        assert torch.equal(y0, y1)
        sg.sg_batch_destroy(b)
