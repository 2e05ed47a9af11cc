"""The double-float contraction mode (SG_DF64) through the C ABI.

Parity with the oracle at the tolerances of tests/helpers.py (norm-wise as
FP64, element-wise DF64_ELEM_TOL), on the literal oracle's cases and on the
benchmark workload at full size against the exact closed form; bitwise
repeatability and the bitwise identity of every entry point (vectors one by
one or together, the no-allocation apply); the contexts the mode refuses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from oracle import galerkin
from oracle import oracle as orc
from paper_2111_13655_gb300 import synth

from helpers import DF64_ELEM_TOL, DF64_TOL, assert_parity, elem_rel, norm_rel

pytestmark = pytest.mark.gpu

CASES = {
    "C1 D=2 L=6 nq=l+1": (synth.workload_C1(), 4),
    "C2 D=6 L=8 nq=l+1": (synth.workload_C2(), 2),
    "D=12 L=5 nq=l+2": (synth.workload_C3(L=5), 2),
    "D=8 L=8 nq=l+2": (synth.workload_C3(L=8, D=8), 1),
    "D=5 L=4 nb=2+l nq=3+l": (synth.chained_henon_heiles(5, 4, synth.draw_omega(5, 8), 0.2,
                                                        nb_rule=(2, 1), nq_rule=(3, 1)), 2),
}


def apply(ctx, x, nvec=None):
    x = np.atleast_2d(x)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.full_like(xd, float("nan"))
    sg.sg_apply_H(ctx, xd, yd, x.shape[0] if nvec is None else nvec)
    torch.cuda.synchronize()
    assert sg.sg_device_error(ctx) == 0
    return yd.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_df64_matches_oracle(name):
    p, nvec = CASES[name]
    x = synth.random_vectors(orc.n_compact(p), nvec, 4321)
    with sg.sg_create(p, "df64") as ctx:
        y = apply(ctx, x)
    if not galerkin.exactness_violations(p):
        n, e = assert_parity(y, galerkin.apply_H(p, x), "df64", name + " (masked Galerkin)")
    else:
        # the literal oracle's own floating-point compress-add adds u * sum |D_l| element-wise
        y_ref = orc.apply_H(p, x)
        n, e = norm_rel(y, y_ref), elem_rel(y, y_ref)
        _, c = orc.enumerate_terms(p.D, p.L)
        own = 2.0 ** -53 * float(np.abs(np.asarray(c, float)).sum())
        assert n <= DF64_TOL and e <= DF64_ELEM_TOL + own, (name, n, e)
    print(f"df64 {name}: norm-wise {n:.3e}, element-wise {e:.3e}")


def test_df64_c3_full_size_matches_masked_galerkin():
    """The benchmark workload, D=12 L=10 nq=l+2, 8 vectors as the benchmark
    times them, against the exact closed form."""
    p = synth.workload_C3()
    x = synth.random_vectors(646646, 8, 17)
    y_ref = galerkin.apply_H(p, x)
    with sg.sg_create(p, "df64") as ctx:
        y = apply(ctx, x)
    n, e = assert_parity(y, y_ref, "df64", "D=12 L=10")
    print(f"df64 D=12 L=10: norm-wise {n:.3e}, element-wise {e:.3e}")


def test_df64_entry_points_bitwise():
    """Exact fixed-point sum: repeats, vectors one at a time, and the
    no-allocation apply (which gathers from x instead of the staged copy)
    give the same bits."""
    p = synth.workload_C3(L=6)
    n = orc.n_compact(p)
    x = synth.random_vectors(n, 3, 99)
    with sg.sg_create(p, "df64") as ctx:
        y = apply(ctx, x)
        assert np.array_equal(apply(ctx, x), y)
        for v in range(3):
            assert np.array_equal(apply(ctx, x[v:v + 1])[0], y[v])
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        yd = torch.empty_like(xd)
        sg.sg_apply_H_noalloc(ctx, xd, yd, 3)
        torch.cuda.synchronize()
        assert np.array_equal(yd.cpu().numpy(), y)


def test_df64_eigenvalues_match_the_oracle_spectrum():
    p = synth.workload_C1()
    from helpers import dense_oracle
    ref = np.linalg.eigvalsh(dense_oracle(p))[:6]
    with sg.sg_create(p, "df64") as ctx:
        ev, _, _, ok = sg.sg_eigs(ctx, 6, "davidson", block=4, tol=1e-9, max_it=300)
    assert ok
    assert np.max(np.abs(ev - ref)) <= 1e-10


def test_df64_tuned_plan_keeps_parity():
    """sg_tune re-plans a double-float context (slicing, split, budget); the
    tuned applies stay within the tolerances and repeat bitwise."""
    p = synth.workload_C3(L=6)
    x = synth.random_vectors(orc.n_compact(p), 4, 31)
    y_ref = galerkin.apply_H(p, x)
    with sg.sg_create(p, "df64") as ctx:
        sg.sg_tune(ctx, 4)
        y = apply(ctx, x)
        assert np.array_equal(apply(ctx, x), y)
    assert_parity(y, y_ref, "df64", "D=12 L=6 tuned")


def test_df64_refusals():
    """Problems off the fast path (a monomial of three modes) and batches are
    refused with SG_EUNSUPPORTED, a double-float server with SG_EINVAL."""
    p3 = synth.polynomial_problem(3, 3, [1.0, 1.0, 1.0], [(0.1, [(0, 1), (1, 1), (2, 1)])])
    with pytest.raises(sg.SgError) as ei:
        sg.sg_create(p3, "df64")
    assert ei.value.status == sg.SG_EUNSUPPORTED
    with sg.sg_create(synth.workload_C1(), "df64") as ctx:
        with pytest.raises(sg.SgError) as ei:
            sg.sg_batch_create([ctx])
        assert ei.value.status == sg.SG_EUNSUPPORTED
    with pytest.raises(sg.SgError) as ei:
        sg.Server("df64")
    assert ei.value.status == sg.SG_EINVAL
