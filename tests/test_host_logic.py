"""Host logic of the CUDA library, checked on the CPU against the oracle.

sg_plan builds the terms, the compact ranking and the 1D tables without a GPU;
these tests compare them with the oracle's independent routes (Golub-Welsch vs
bracketed Newton nodes, Christoffel vs classical weights, ladder vs ODE second
derivatives, combinatorial ranking vs sorted-list search).
"""
import numpy as np
import pytest

import paper_2111_13655_gb300 as sg
from oracle import oracle as orc
from paper_2111_13655_gb300 import synth

CASES = [
    synth.chained_henon_heiles(2, 3, [1.0, 1.0], 0.1),
    synth.workload_C1(),
    synth.chained_henon_heiles(4, 5, synth.draw_omega(4, 1), 0.2, nq_rule=(2, 1)),
    synth.chained_henon_heiles(3, 4, synth.draw_omega(3, 2), 0.2, nb_rule=(1, 2), nq_rule=(1, 2)),
    synth.chained_henon_heiles(5, 3, synth.draw_omega(5, 3), 0.2, nb_rule=(2, 1), nq_rule=(3, 1)),
    synth.workload_C2(),
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def planned(request):
    p = CASES[request.param]
    ctx = sg.sg_plan(p, "fp64")
    yield p, ctx
    sg.sg_destroy(ctx)


def test_sizes_match_oracle_counts(planned):
    p, ctx = planned
    nt, ns, ncs = orc.counts(p.D, p.L, p.nb_A, p.nb_B)
    s = sg.sg_size(ctx)
    assert (s["n_terms"], s["n_s"], s["n_cs"]) == (nt, ns, ncs)


def test_terms_in_table2_order_with_coefficients(planned):
    p, ctx = planned
    lv, c = sg.sg_term_levels(ctx)
    lo, co = orc.enumerate_terms(p.D, p.L)
    assert np.array_equal(lv, lo)
    assert np.array_equal(c.astype(np.int64), co)


def test_compact_rank_is_bit_exact(planned):
    p, ctx = planned
    K = orc.enumerate_compact(p.D, p.L, p.nb_A, p.nb_B)
    r = sg.sg_compact_rank(ctx, K)
    assert np.array_equal(r, np.arange(K.shape[0]))
    # indices outside the compact basis are rejected
    bad = K[-1:].copy()
    bad[0, 0] += p.L + 5
    assert sg.sg_compact_rank(ctx, bad)[0] == -1


def test_mode_tables_match_oracle(planned):
    p, ctx = planned
    for i in range(p.D):
        for l in range(p.L + 1):
            t = sg.sg_mode_tables(ctx, i, l)
            B, D2, W, Q = orc.mode_tables(t["nb"], t["nq"], float(p.q0[i]), float(p.scale[i]))
            assert np.abs(t["B"] - B).max() < 1e-13
            assert np.abs(t["BW"] - (B * W[:, None]).T).max() < 1e-12 * max(1, W.max())
            assert np.abs(t["Q"] - Q).max() < 1e-13
            Kref = -0.5 * p.omega[i] * (B.T * W[None, :]) @ D2
            assert np.abs(t["K"] - Kref).max() < 1e-11 * max(1.0, np.abs(Kref).max())


def test_plan_limits_and_errors():
    p = synth.chained_henon_heiles(3, 40, [1.0] * 3, 0.1)       # nq(L) = 41 > 32
    with pytest.raises(sg.SgError) as e:
        sg.sg_plan(p)
    assert e.value.status == sg.SG_EUNSUPPORTED
    p = synth.chained_henon_heiles(3, 4, [1.0] * 3, 0.1, nb_rule=(2, 1), nq_rule=(1, 1))  # nq < nb
    with pytest.raises(sg.SgError) as e:
        sg.sg_plan(p)
    assert e.value.status == sg.SG_EINVAL


def test_plan_context_has_no_device_state():
    ctx = sg.sg_plan(synth.workload_C1())
    # the device-state check comes before any pointer is used
    assert sg.lib().sg_apply_H(ctx.ptr, 8, 4096, 1, None) == sg.SG_EINVAL
    assert "sg_plan" in sg.sg_last_error(ctx)
    sg.sg_destroy(ctx)


def test_c3_plan_sizes():
    """D=12 L=10 nb=l+1 nq=l+2: 646,646 terms and compact functions, N_s = 131,128,140."""
    p = synth.workload_C3()
    ctx = sg.sg_plan(p, "mixed")
    s = sg.sg_size(ctx)
    assert s["n_terms"] == 646646 and s["n_cs"] == 646646 and s["n_s"] == 131128140
    assert s["n_grid"] == 68292740824
    sg.sg_destroy(ctx)


def inner_block_table_elements(levels, u):
    """Elements of the inner-block tables at nb = l+1, nq = l+2 (chained
    coupling): per term with two neighbouring transformed modes, the upper
    triangle of an NBI x NBI block (NBI = 2^R, R = min(3, its level-1 modes))
    in 16-byte units (one element when NBI = 1) at every outer grid point,
    padded to 16 bytes per term."""
    total = 0
    for l in levels:
        act = [v > 0 for v in l]
        if not any(act[i] and act[i + 1] for i in range(len(l) - 1)):
            continue
        R = min(3, sum(1 for v in l if v == 1))
        nbi = 2 ** R
        ngo = 1
        n1 = 0
        for v in l[::-1]:
            if v == 1 and n1 < R:
                n1 += 1
            elif v > 0:
                ngo *= v + 2
        ue = 1 if nbi == 1 else u
        per = -(-(nbi * (nbi + 1) // 2) // ue) * ue
        total += -(-(per * ngo) // u) * u
    return total


def test_plan_reports_the_device_bytes_of_sg_create():
    """A planned context holds no device memory but reports what sg_create would
    allocate.  At D=12 L=10 that includes M^B (N_s int32) and the inner-block
    tables of the terms with a grid, in the context's precision, so FP64 needs
    more."""
    from oracle import oracle as orc
    lv, _ = orc.enumerate_terms(12, 10)
    p = synth.workload_C3()
    sizes = {}
    for prec, rb in (("mixed", 4), ("fp64", 8)):
        ctx = sg.sg_plan(p, prec)
        b = sg.sg_size(ctx)["bytes_device"]
        sg.sg_destroy(ctx)
        lower = 131128140 * 4 + inner_block_table_elements(lv.tolist(), 16 // rb) * rb
        assert lower <= b <= lower + 3 * 10 ** 9, (prec, b, lower)
        sizes[prec] = b
    assert sizes["fp64"] > sizes["mixed"]
    # the double-float mode holds its tables as (hi, lo) FP32 pairs: the FP64 sizes
    ctx = sg.sg_plan(p, "df64")
    assert sg.sg_size(ctx)["bytes_device"] == sizes["fp64"]
    sg.sg_destroy(ctx)
