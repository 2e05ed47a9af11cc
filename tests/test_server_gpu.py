"""Propagation server: continuous batching of Chebyshev propagation requests.

Checks: the closed-form phases at zero coupling; agreement with sg_propagate
on the same problem; every request's result bitwise the same alone and in a
mix whose membership changes while it runs (FP64 and mixed), also behind an
eigen request that holds several batch slots; admission by the
device-memory budget; requests without steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_13655_gb300 as sg
from oracle import oracle as orc
from paper_2111_13655_gb300 import synth

from helpers import dense_oracle

pytestmark = pytest.mark.gpu


def packet(p, q0=1.5):
    kw = int(max(p.nb_A + p.nb_B * p.L))
    q = np.zeros(p.D)
    q[0] = q0
    return synth.coherent_factors(q, kw)


def normalised_state(p, q0=1.5):
    with sg.sg_plan(p, "fp64") as c:
        psi = sg.sg_product_state(c, packet(p, q0))
    return psi / np.linalg.norm(psi)


def test_uncoupled_request_matches_closed_form_phases():
    om = synth.draw_omega(4, 12)
    p = synth.chained_henon_heiles(4, 6, om, 0.0)
    E = (orc.enumerate_compact(4, 6) + 0.5) @ om
    psi0 = normalised_state(p)
    with sg.Server("fp64") as srv:
        rid = srv.submit(p, 0.1, 15, psi0=psi0.astype(complex))
        srv.run()
        psi, nl, el, _ = srv.result(rid)
    assert np.max(np.abs(psi - psi0 * np.exp(-1j * E * 1.5))) < 1e-10
    assert np.max(np.abs(nl - 1.0)) < 1e-12
    assert np.max(np.abs(el - el[0])) < 1e-11


def test_server_matches_sg_propagate():
    p = synth.chained_henon_heiles(6, 6, synth.draw_omega(6, 2), synth.HH_LAMBDA)
    psi0 = normalised_state(p, 2.0)
    with sg.sg_create(p, "fp64") as ctx:
        d = torch.from_numpy(np.concatenate([psi0, np.zeros_like(psi0)])).cuda()
        nl_ref, el_ref = sg.sg_propagate(ctx, d, 0.1, 12, order=64)
        ref = d.cpu().numpy()
    ref = ref[:len(psi0)] + 1j * ref[len(psi0):]
    with sg.Server("fp64") as srv:
        rid = srv.submit(p, 0.1, 12, psi0=psi0.astype(complex))
        srv.run()
        psi, nl, el, _ = srv.result(rid)
    assert np.max(np.abs(psi - ref)) < 1e-11
    assert np.max(np.abs(nl - nl_ref)) < 1e-12
    assert np.max(np.abs(el - el_ref)) < 1e-11


# mixed: measured 3.8e-7 on GB300 (FP32 contractions through 50 steps of
# order-64 Chebyshev); the bound keeps a margin above ten
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 5e-6)])
def test_request_matches_exact_propagator_of_the_oracle(prec, tol):
    """A D=6 L=8 coupled request (the 6D propagation configuration, 50 steps of
    0.1) against psi(t) = exp(-i H_S t) psi(0) from the literal oracle's dense
    H_S, element by element; the mixed server's error is printed."""
    p = synth.workload_C2()
    w, U = np.linalg.eigh(dense_oracle(p))
    psi0 = normalised_state(p, 2.0)
    exact = U @ (np.exp(-1j * w * 5.0) * (U.T @ psi0))
    with sg.Server(prec) as srv:
        rid = srv.submit(p, 0.1, 50, psi0=psi0.astype(complex))
        srv.run()
        psi, nl, el, _ = srv.result(rid)
    err = np.max(np.abs(psi - exact))
    print(f"server {prec}, D=6 L=8, t = 5: max |psi - psi_exact| = {err:.2e}")
    assert err <= tol


def mix_problems():
    return {
        "R": synth.chained_henon_heiles(6, 6, synth.draw_omega(6, 21), synth.HH_LAMBDA),
        "A": synth.chained_henon_heiles(4, 7, synth.draw_omega(4, 22), synth.HH_LAMBDA),
        "B": synth.chained_henon_heiles(8, 5, synth.draw_omega(8, 23), synth.HH_LAMBDA),
        "C": synth.workload_C3(L=4),
    }


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_results_identical_alone_and_in_a_changing_mix(prec):
    P = mix_problems()
    steps = {"R": 6, "A": 3, "B": 8, "C": 2}
    alone = {}
    for name, p in P.items():
        with sg.Server(prec) as srv:
            rid = srv.submit(p, 0.1, steps[name], order=48, factors=packet(p))
            srv.run()
            alone[name] = srv.result(rid)[:3]
    with sg.Server(prec) as srv:
        ids = {"A": srv.submit(P["A"], 0.1, steps["A"], order=48, factors=packet(P["A"]))}
        srv.progress(5)                       # A runs alone for a while
        ids["R"] = srv.submit(P["R"], 0.1, steps["R"], order=48, factors=packet(P["R"]))
        srv.progress(7)                       # R joins mid-step of A
        ids["B"] = srv.submit(P["B"], 0.1, steps["B"], order=48, factors=packet(P["B"]))
        ids["C"] = srv.submit(P["C"], 0.1, steps["C"], order=48, factors=packet(P["C"]))
        seen = set()
        while True:
            a, q = srv.progress(3)
            seen.add(a)
            if a == 0 and q == 0:
                break
        assert max(seen) >= 3                 # the requests did overlap
        for name, rid in ids.items():
            psi, nl, el, _ = srv.result(rid)
            assert np.array_equal(psi, alone[name][0]), name
            assert np.array_equal(nl, alone[name][1]) and np.array_equal(el, alone[name][2]), name
        assert srv.stats()["bytes_in_use"] == 0


def test_admission_by_device_memory_budget():
    P = mix_problems()
    with sg.Server("fp64") as big:
        rid = big.submit(P["B"], 0.1, 2, order=32, factors=packet(P["B"]))
        big.progress(1)
        need = big.stats()["bytes_in_use"]   # planned bytes of B while active
        big.run()
        ref = big.result(rid)[0]
    assert need > 0
    with sg.Server("fp64", hbm_budget_bytes=int(need * 1.5)) as srv:
        ids = [srv.submit(P["B"], 0.1, 2, order=32, factors=packet(P["B"])) for _ in range(3)]
        while True:
            a, q = srv.progress(1)
            assert a <= 1                     # only one fits the budget at a time
            assert srv.stats()["bytes_in_use"] <= int(need * 1.5)
            if a == 0 and q == 0:
                break
        for rid in ids:
            assert np.array_equal(srv.result(rid)[0], ref)
    with sg.Server("fp64", hbm_budget_bytes=need // 4) as srv:
        with pytest.raises(sg.SgError) as ei:
            srv.submit(P["B"], 0.1, 2, order=32, factors=packet(P["B"]))
        assert ei.value.status == sg.SG_EBUDGET


def test_request_without_steps_returns_its_initial_state():
    p = mix_problems()["A"]
    psi0 = normalised_state(p) * np.exp(0.3j)
    with sg.Server("mixed") as srv:
        rid = srv.submit(p, 0.1, 0, psi0=psi0)
        srv.run()
        psi, nl, el, _ = srv.result(rid)
    assert np.array_equal(psi, psi0) and nl.size == 0 and el.size == 0


# --- eigen requests -------------------------------------------------------

def test_eigen_request_equals_sg_eigs_bitwise():
    """An eigen request runs the block Davidson of sg_eigs with its block
    applications batched by the engine; batched applies are bitwise those of
    the request's own context, so the eigenpairs are bitwise those of sg_eigs."""
    p = synth.workload_C2()
    with sg.sg_create(p, "fp64") as ctx:
        ev, rs, vec, ok = sg.sg_eigs(ctx, 6, "davidson", block=4, tol=1e-9, max_it=300, vectors=True)
    assert ok
    with sg.Server("fp64") as srv:
        rid = srv.submit_eigs(p, 6, block=4, tol=1e-9, max_it=300, vectors=True)
        srv.run()
        ev2, rs2, vec2, _, nconv = srv.eig_result(rid, vectors=True)
    assert nconv == 6
    assert np.array_equal(ev2, ev) and np.array_equal(rs2, rs)
    assert np.array_equal(vec2, vec.cpu().numpy())


def test_eigen_request_matches_the_oracle_spectrum():
    """D=2 L=6 Henon-Heiles: the 10 lowest eigenvalues against the literal
    oracle's dense H_S, FP64 server and mixed-precision server (the mixed
    result carries the FP32 contractions' error, reported per eigenvalue)."""
    p = synth.workload_C1()
    ref = np.linalg.eigvalsh(dense_oracle(p))[:10]
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        with sg.Server(prec) as srv:
            rid = srv.submit_eigs(p, 10, block=4, tol=1e-10 if prec == "fp64" else 1e-6, max_it=300)
            srv.run()
            ev, rs, _, _, nconv = srv.eig_result(rid)
        err = np.abs(ev - ref)
        print(f"server {prec} eigen request D=2 L=6: max |E - E_oracle| = {err.max():.2e}")
        assert err.max() <= tol, (prec, err)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eigen_and_propagation_requests_identical_alone_and_in_a_mix(prec):
    P = mix_problems()
    alone = {}
    with sg.Server(prec) as srv:
        rid = srv.submit_eigs(P["A"], 4, block=2, tol=1e-7, max_it=200)
        srv.run()
        alone["eA"] = srv.eig_result(rid)[:2]
    with sg.Server(prec) as srv:
        rid = srv.submit_eigs(P["B"], 3, block=3, tol=1e-7, max_it=200)
        srv.run()
        alone["eB"] = srv.eig_result(rid)[:2]
    for name in ("R", "C"):
        with sg.Server(prec) as srv:
            rid = srv.submit(P[name], 0.1, 3, order=32, factors=packet(P[name]))
            srv.run()
            alone[name] = srv.result(rid)[:3]
    with sg.Server(prec) as srv:
        ids = {"R": srv.submit(P["R"], 0.1, 3, order=32, factors=packet(P["R"]))}
        srv.progress(4)                                    # R runs alone first
        ids["eA"] = srv.submit_eigs(P["A"], 4, block=2, tol=1e-7, max_it=200)
        srv.progress(3)                                    # eA joins R
        # eB holds two batch slots; C comes after it in slot order
        ids["eB"] = srv.submit_eigs(P["B"], 3, block=3, tol=1e-7, max_it=200)
        ids["C"] = srv.submit(P["C"], 0.1, 3, order=32, factors=packet(P["C"]))
        seen = set()
        while True:
            a, q = srv.progress(2)
            seen.add(a)
            if a == 0 and q == 0:
                break
        assert max(seen) >= 3
        for name, rid in ids.items():
            if name.startswith("e"):
                ev, rs = srv.eig_result(rid)[:2]
                assert np.array_equal(ev, alone[name][0]) and np.array_equal(rs, alone[name][1]), name
            else:
                psi, nl, el, _ = srv.result(rid)
                assert np.array_equal(psi, alone[name][0]), name
                assert np.array_equal(nl, alone[name][1]) and np.array_equal(el, alone[name][2]), name
        assert srv.stats()["bytes_in_use"] == 0


def test_eigen_request_over_the_budget_is_refused():
    with sg.Server("fp64", hbm_budget_bytes=1 << 20) as srv:
        with pytest.raises(sg.SgError) as ei:
            srv.submit_eigs(mix_problems()["B"], 4, block=4)
        assert ei.value.status == sg.SG_EBUDGET
