"""Term-sharded apply on one GPU: the parts of the term list (processing
positions p = part mod nparts) accumulated separately and summed as 64-bit
integers give bitwise the full sg_apply_H, for any number of parts (the
integer sum is associative).  This is the arithmetic a multi-GPU apply runs
with one part per GPU and one integer all-reduce (the MPI sum of Alg. 2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from paper_2111_13655_gb300 import sharded, synth

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "D=6 L=8 nq=l+1": synth.workload_C2(),
    "D=12 L=6 nq=l+2": synth.workload_C3(L=6),
    "general polynomial (generic kernel)": synth.polynomial_problem(
        3, 5, [0.9, 1.1, 1.0],
        [(0.3, [(0, 1)]), (0.2, [(0, 2), (1, 2)]), (0.05, [(0, 1), (1, 1), (2, 1)]), (0.7, [])],
        q0=[0.3, -0.2, 0.1], scale=[1.3, 0.8, 1.0]),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_parts_summed_as_integers_equal_the_full_apply_bitwise(prec, name):
    p = PROBLEMS[name]
    nvec = 3
    with sg.sg_create(p, prec) as ctx:
        x = torch.from_numpy(synth.random_vectors(ctx.n_cs, nvec, 21)).cuda().contiguous().view(-1)
        y_ref = torch.empty_like(x)
        sg.sg_apply_H(ctx, x, y_ref, nvec)
        for nparts in (2, 3):
            total = torch.zeros(sg.acc_words(ctx, nvec), dtype=torch.int64, device="cuda")
            for part in range(nparts):
                acc = torch.zeros_like(total)
                sg.sg_apply_H_part(ctx, x, acc, nvec, part, nparts)
                total += acc                      # 64-bit integer sum (wraps)
            y = torch.full_like(x, float("nan"))
            sg.sg_apply_H_finish(ctx, x, total, y, nvec)
            torch.cuda.synchronize()
            assert sg.sg_device_error(ctx) == 0
            assert torch.equal(y, y_ref), (name, prec, nparts)
            assert int(total.abs().max()) == 0    # the finish clears the accumulators


def test_single_rank_sharded_helper_equals_sg_apply_H():
    p = synth.workload_C2()
    with sg.sg_create(p, "mixed") as ctx:
        x = torch.from_numpy(synth.random_vectors(ctx.n_cs, 2, 5)).cuda().contiguous().view(-1)
        y, y_ref = torch.empty_like(x), torch.empty_like(x)
        sg.sg_apply_H(ctx, x, y_ref, 2)
        sharded.apply_H_sharded(ctx, x, y, 2)
        torch.cuda.synchronize()
        assert torch.equal(y, y_ref)
