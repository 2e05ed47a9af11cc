"""Batched apply: many independent problems per sg_apply_H_batch.

The batch runs the terms of all problems of one kernel variant in one launch,
ordered by cost over all problems.  Every problem's arithmetic is the same as
in its own sg_apply_H (same records, vector chunks and exact fixed-point
compress-add), so results must agree bitwise; FP64 results are also checked
against the literal CPU oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from oracle import oracle as orc
from paper_2111_13655_gb300 import synth

from helpers import assert_parity

pytestmark = pytest.mark.gpu


def mixed_bag():
    """Problems of several kernel variants, with a generic-path one among them."""
    return [
        synth.workload_C1(),
        synth.workload_C2(),
        synth.workload_C3(L=5),                                  # nb = l+1, nq = l+2
        synth.chained_henon_heiles(4, 5, synth.draw_omega(4, 9), 0.2, nb_rule=(1, 2), nq_rule=(1, 2)),
        synth.polynomial_problem(                                # three-mode monomial: generic kernel
            3, 5, [0.9, 1.1, 1.0],
            [(0.3, [(0, 1)]), (0.2, [(0, 2), (1, 2)]), (0.05, [(0, 1), (1, 1), (2, 1)]), (0.7, [])],
            q0=[0.3, -0.2, 0.1], scale=[1.3, 0.8, 1.0]),
        synth.chained_henon_heiles(5, 4, synth.draw_omega(5, 8), 0.2, q0=0.4, scale=1.2),
        synth.chained_henon_heiles(1, 9, [1.3], 0.0),
        synth.chained_henon_heiles(8, 6, synth.draw_omega(8, 5), synth.HH_LAMBDA),
    ]


def per_context(ctxs, xs, nvec):
    ys = []
    for c, x in zip(ctxs, xs):
        y = torch.empty_like(x)
        sg.sg_apply_H(c, x, y, nvec)
        ys.append(y)
    torch.cuda.synchronize()
    return ys


def batched(b, xs, nvec):
    x = torch.cat(xs)
    y = torch.full_like(x, float("nan"))
    sg.sg_apply_H_batch(b, x, y, nvec)
    torch.cuda.synchronize()
    return [y[nvec * int(b.offsets[j]):nvec * int(b.offsets[j + 1])] for j in range(len(xs))]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_each_problem_bitwise(prec):
    probs = mixed_bag()
    ctxs = [sg.sg_create(p, prec) for p in probs]
    b = sg.sg_batch_create(ctxs)
    try:
        assert b.n_cs_total == sum(c.n_cs for c in ctxs)
        for call, nvec in enumerate((3, 5, 2)):   # growing then shrinking the batch workspace
            xs = [torch.from_numpy(synth.random_vectors(c.n_cs, nvec, 100 * call + j)).cuda().contiguous().view(-1)
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


def test_batch_fp64_matches_oracle():
    probs = mixed_bag()[:2] + mixed_bag()[3:7]
    ctxs = [sg.sg_create(p, "fp64") for p in probs]
    b = sg.sg_batch_create(ctxs)
    try:
        nvec = 2
        xs_np = [synth.random_vectors(c.n_cs, nvec, 7 + j) for j, c in enumerate(ctxs)]
        got = batched(b, [torch.from_numpy(x).cuda().contiguous().view(-1) for x in xs_np], nvec)
        for j, p in enumerate(probs):
            ref = orc.apply_H(p, xs_np[j])
            g = got[j].view(nvec, -1).cpu().numpy()
            assert_parity(g, ref, "fp64", p.name)
    finally:
        sg.sg_batch_destroy(b)
        for c in ctxs:
            sg.sg_destroy(c)


def test_wavepacket_batch_of_the_batched_configuration_shape():
    """24 wavepackets drawn like the 256-instance configuration (smaller D and L),
    complex wavepackets as two real vectors each; mixed and FP64 side by side."""
    items = synth.workload_C4(n=24, seed=41, Ds=(4, 6, 8), Ls=(6, 7))
    for prec in ("mixed", "fp64"):
        ctxs = [sg.sg_create(p, prec) for p, _ in items]
        b = sg.sg_batch_create(ctxs)
        try:
            xs = []
            for (p, q0), c in zip(items, ctxs):
                psi = sg.sg_product_state(c, synth.coherent_factors(q0, p.L + 1))
                psi /= np.linalg.norm(psi)
                xs.append(torch.from_numpy(np.concatenate([psi, np.roll(psi, 1)])).cuda())
            ref = per_context(ctxs, xs, 2)
            got = batched(b, xs, 2)
            for j in range(len(items)):
                assert torch.equal(got[j], ref[j])
        finally:
            sg.sg_batch_destroy(b)
            for c in ctxs:
                sg.sg_destroy(c)


def test_batch_rejects_mixed_precisions():
    a = sg.sg_create(synth.workload_C1(), "fp64")
    c = sg.sg_create(synth.workload_C1(), "mixed")
    try:
        with pytest.raises(sg.SgError):
            sg.sg_batch_create([a, c])
    finally:
        sg.sg_destroy(a)
        sg.sg_destroy(c)


def test_graph_replays_on_a_stream_stay_bitwise_per_context():
    """On a non-default stream the batched apply captures its launch sequence
    once per (x, y, nvec, stream) and replays it: new input values, new
    buffers and a new block size must all give each context's own result."""
    probs = [synth.workload_C2(), synth.workload_C3(L=5), synth.chained_henon_heiles(5, 4, synth.draw_omega(5, 8), 0.2)]
    for prec in ("mixed", "fp64"):
        ctxs = [sg.sg_create(p, prec) for p in probs]
        b = sg.sg_batch_create(ctxs)
        s = torch.cuda.Stream()
        try:
            for call, nvec in enumerate((2, 2, 2, 3, 3)):
                xs = [torch.from_numpy(synth.random_vectors(c.n_cs, nvec, 500 + 10 * call + j)).cuda().contiguous().view(-1)
                      for j, c in enumerate(ctxs)]
                x = torch.cat(xs)
                if call == 2:
                    x = x.clone()                  # new buffers at call 2
                y = torch.full_like(x, float("nan"))
                torch.cuda.synchronize()
                with torch.cuda.stream(s):
                    sg.sg_apply_H_batch(b, x, y, nvec, s)
                s.synchronize()
                ref = per_context(ctxs, xs, nvec)
                for j in range(len(ctxs)):
                    got = y[nvec * int(b.offsets[j]):nvec * int(b.offsets[j + 1])]
                    assert torch.equal(got, ref[j]), (prec, call, j)
        finally:
            sg.sg_batch_destroy(b)
            for c in ctxs:
                sg.sg_destroy(c)
