"""Batched apply with a large member: a problem with enough block-form terms
to fill the GPU by itself runs as its own launches inside the batch's launch
sequence (its parameters in the kernel's parameter bank), beside the packed
launches of the small problems.  Results stay bitwise those of each problem's
own context.  (A file of its own, run last: it holds the D=12 L=10 tables.)
"""
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from paper_2111_13655_gb300 import synth

from test_batch_gpu import batched, per_context

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_large_member_runs_as_its_own_launches_bitwise(prec):
    """A problem with many block-form terms (the D=12 L=10 workload: over
    300,000 of its 646,646 terms run one per block) runs as its own launches
    inside the batch's sequence, beside packed small ones; every result is
    still bitwise that of the problem's own context, with the workspace grown
    and reused.  (At D=12 L=8 the block form holds too few terms for that.)"""
    probs = [synth.workload_C2(), synth.workload_C3(), synth.chained_henon_heiles(5, 4, synth.draw_omega(5, 8), 0.2)]
    ctxs = [sg.sg_create(p, prec) for p in probs]
    b = sg.sg_batch_create(ctxs)
    try:
        # max|x|, input copies, finalisation, at most two packed launches: more means
        # the large problem has launches of its own
        assert b.launches_per_apply >= 6, b.launches_per_apply
        for call, nvec in enumerate((2, 4, 2)):
            xs = [torch.from_numpy(synth.random_vectors(c.n_cs, nvec, 300 + 10 * call + j)).cuda().contiguous().view(-1)
                  for j, c in enumerate(ctxs)]
            ref = per_context(ctxs, xs, nvec)
            got = batched(b, xs, nvec)
            for j in range(len(ctxs)):
                assert torch.equal(got[j], ref[j]), f"call {call} problem {j} ({probs[j].name})"
        for c in ctxs:
            assert sg.sg_device_error(c) == 0
    finally:
        sg.sg_batch_destroy(b)
        for c in ctxs:
            sg.sg_destroy(c)
