#!/usr/bin/env python
"""Benchmark: Smolyak H|psi> applications/s on the D=12 L=10 workload.

Workload: chained Henon-Heiles, D=12, L=10, nb(l)=l+1, nq(l)=l+2, omega_i ~
U[0.8,1.2] (seeded), lambda = 0.111803; N_cs = 646,646 compact functions,
646,646 Smolyak terms.  One step = one sg_apply_H on a block of `nvec` real
vectors (the block of the block-Davidson solver); one application = one real
vector.  Mixed precision (FP32 contractions, FP64 accumulation) is the headline;
FP64 mode is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs an independent replica (independent
problems, no collective on the data path); value = all ranks' applications /
the slowest rank's time ("scaling": "weak").  --sharding terms instead splits
one problem's terms over the ranks with one integer all-reduce per apply
("scaling": "strong").
--impl reference: the CPU oracle (the literal Alg. 1 in C) timed as it stands
on the host cores, each step a random sample of the workload's terms.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Smolyak H|psi> applications/s and % roofline at D=12 L=10; mixed vs FP64; p50/p99"
UNIT = "applications/s"
WORKLOAD = "chained Henon-Heiles D=12 L=10 nb=l+1 nq=l+2 (N_cs=646646, 646646 terms)"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the term kernel
# k_apply_fast per apply (its block-form and warp-form launches) at the
# benchmark workload with the plan sg_tune keeps, per precision, from the
# one-pass ncu capture of the full workload summarised in profiles/; None when
# the kernel has changed since.
TRAFFIC_BYTES = {"mixed": 8_849_153_280, "fp64": 23_382_741_248, "df64": 23_298_306_560}
# FP32 instructions of one double-float multiply-add (csrc/sg_df.cuh df_fma:
# one multiply, three FMAs, two_sum 6, two additions): the double-float arm's
# roofline counts these against the FP32 issue rate
DF_INSTR_PER_FMA = 12
# FP32 lanes per SM (the unit count of the derived FP32 peak)
FP32_LANES_PER_SM = 128
# kernels of one sg_apply_H at this workload: k_maxabs, k_stage_x (entry-major
# input copy), k_apply_fast (block form over the large terms), k_apply_fast
# (warp form over the small terms), k_finalize
LAUNCHES_PER_APPLY = 5


def algorithmic_flops_per_vector(levels: np.ndarray, nbA=1, nbB=1, nqA=2, nqB=1, rmax=None) -> int:
    """FLOPs of one real-vector apply of the chained Henon-Heiles operator by
    the route the fast kernel takes, 2 flops per multiply-add.  Per term:
      - a term has a grid when two neighbouring modes (a coupled pair) both
        have nb > 1; then its last `rmax` level-1 modes (mode order) are inner
        positions (rmax = 3 for nb(1) = 2, 2 for nb(1) = 3, else 0);
      - forward one-mode contractions over the other (outer) modes with
        nb > 1, in the planned order (ascending 1/nb - 1/nq, ties in mode
        order), each on NBI = prod(inner nb) values per site, and the mirrored
        backward chain (the same count);
      - at every outer grid point the NBI x NBI inner block;
      - the single-mode matrices of the outer modes (and the constant c0 of a
        term without a grid), one multiply-add per basis entry and function;
      - the weighted compress-add, 2 flops per basis entry."""
    l = np.asarray(levels).astype(np.int64)
    n_t, D = l.shape
    nb_all = nbA + nbB * l
    nq_all = nqA + nqB * l
    act = nb_all > 1
    if rmax is None:
        rmax = 3 if nbA + nbB == 2 else 2 if nbA + nbB == 3 else 0
    grid = (act[:, :-1] & act[:, 1:]).any(axis=1) if D > 1 else np.zeros(n_t, bool)
    l1 = (l == 1) & act
    # rank of each level-1 mode counted from the last mode: inner if <= R
    from_right = np.cumsum(l1[:, ::-1], axis=1)[:, ::-1]
    inner = l1 & (from_right <= rmax) & grid[:, None]
    outer = act & ~inner
    NBI = np.where(inner, nb_all, 1).prod(axis=1)
    key = np.where(outer, 1.0 / nb_all - 1.0 / nq_all, np.inf)
    idx = np.argsort(key, axis=1, kind="stable")
    ob = np.take_along_axis(np.where(outer, nb_all, 1), idx, axis=1)
    oq = np.take_along_axis(np.where(outer, nq_all, 1), idx, axis=1)
    om = np.take_along_axis(outer, idx, axis=1)
    # prefix product of nq over earlier outer positions, suffix product of nb over later ones
    pre = np.cumprod(np.concatenate([np.ones((n_t, 1), np.int64), oq[:, :-1]], axis=1), axis=1)
    suf = np.ones_like(ob)
    for i in range(D - 2, -1, -1):
        suf[:, i] = suf[:, i + 1] * ob[:, i + 1]
    fwd = (np.where(om, ob * oq, 0) * pre * suf).sum(axis=1) * NBI
    NB = np.where(act, nb_all, 1).prod(axis=1)
    NGo = oq.prod(axis=1)
    reg = np.where(grid, NGo * NBI * NBI, 0)
    basis = NB * (np.where(outer, nb_all, 0).sum(axis=1) + np.where(grid, 0, 1))
    return int((2 * (2 * fwd + reg + basis) + 2 * NB).sum())


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_rate(problem, n_terms: int, seconds: float, seed: int, threads: int = 0):
    """Time the literal oracle on a random sample of terms sized to ~`seconds`;
    returns (applications/s estimate, sample description, threads used)."""
    from oracle import oracle as orc
    rng = np.random.default_rng(seed)
    x = np.random.default_rng(seed).standard_normal((1, orc.n_compact(problem)))
    pilot = rng.choice(n_terms, 64, replace=False)
    t0 = time.perf_counter()
    orc.apply_H(problem, x, pilot, threads)
    tp = max(time.perf_counter() - t0, 1e-3)
    n = int(min(n_terms, max(64, 64 * seconds / tp)))
    sub = rng.choice(n_terms, n, replace=False)
    t0 = time.perf_counter()
    orc.apply_H(problem, x, sub, threads)
    dt = time.perf_counter() - t0
    est_apply_s = dt * n_terms / n
    used = threads if threads > 0 else orc.max_threads()
    return 1.0 / est_apply_s, f"{n} of {n_terms} terms drawn uniformly (1 vector), {dt:.1f} s; " \
        f"full apply estimated as sample time x {n_terms}/{n}", used


def bench_config(args, world: int) -> dict:
    """The `config` of the JSON line; the same for both arms."""
    par = f"terms sharded x{world}" if getattr(args, "sharding", "replicas") == "terms" and world > 1 \
        else f"replicas x{world}"
    return {"workload": workload_name(args.L), "precision": "mixed (FP32 contractions, FP64 accumulation)",
            "vectors_per_step": args.nvec, "parallelism": par,
            "l2": "flushed between timed steps (256 MB write)"}


def workload_name(L: int) -> str:
    if L == 10:
        return WORKLOAD
    return f"chained Henon-Heiles D=12 L={L} nb=l+1 nq=l+2 (reduced size)"


def measure_peaks(sg, torch, seconds: float) -> dict:
    """Roofline denominators measured on this GPU: FP32 (the larger of the scalar
    and the packed two-lane fma loops) and FP64 fma throughput from
    sg_measure_peak, with the SM clock sampled meanwhile.  Beside them the
    derived FP32 figure: SM count (read from the device) x 128 lanes x 2 flops
    x the maximum SM clock."""
    with ClockSampler(torch.cuda.current_device()) as clk:
        f32, sms = sg.sg_measure_peak("fp32", seconds)
        f32x2, _ = sg.sg_measure_peak("fp32x2", seconds)
        f64, _ = sg.sg_measure_peak("fp64", seconds)
    c = clk.summary()
    mx = c.get("sm_max_mhz") or 2070.0
    clock = f"SM clock median {c.get('sm_mhz')} MHz of max {mx} MHz, reasons {c.get('reasons')}"
    return {"fp32": max(f32, f32x2) / 1e12, "fp64": f64 / 1e12, "sms": sms,
            "fp32_scalar": f32 / 1e12, "fp32_packed": f32x2 / 1e12,
            "derived_fp32": sms * FP32_LANES_PER_SM * 2 * mx * 1e6 / 1e12,
            "note_fp32": f"measured FP32 fma loop on {sms} SMs (scalar {f32 / 1e12:.1f}, packed f32x2 "
                         f"{f32x2 / 1e12:.1f} TFLOP/s; the larger); {clock}",
            "note_fp64": f"measured FP64 fma loop on {sms} SMs; {clock}",
            "clocks": c}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2111_13655_gb300 import synth
    from oracle import oracle as orc
    orc.build()
    p = synth.workload_C3()
    n_terms = orc.counts(12, 10)[0]
    rates = []
    desc = ""
    cores = 0
    for i in range(args.warmup + args.steps):
        r, desc, cores = oracle_sample_rate(p, n_terms, args.ref_seconds, 1000 + i)
        if i >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: " + desc + " (the FP64 CPU oracle, one vector)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class Replicas:
    """N > 1: one independent replica per rank (no collective on the data path);
    only the timing is combined: a barrier around each timed region and the
    maximum of the ranks' times.  `backend` "nccl" on GPUs, "gloo" on CPU."""

    def __init__(self, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.dist = None
        self.device = "cuda" if backend == "nccl" else "cpu"
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None

    def max_over_ranks(self, value: float) -> float:
        if self.dist is None:
            return float(value)
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def replica_throughput(world: int, units_per_rank: int, slowest_seconds: float) -> float:
    """Whole-job rate: every rank's units over the slowest rank's time."""
    return world * units_per_rank / slowest_seconds


def run_stream(sg, prec, items, factors, rate, eig_every, eig_args, seed=55):
    """One Poisson stream through a server of precision `prec`: propagation
    requests, and every eig_every-th request an eigen request of the same
    problem instead.  Returns (results by request index, makespan s, stats)."""
    arrivals = np.cumsum(np.random.Generator(np.random.PCG64(seed)).exponential(1.0 / rate, len(items)))
    srv = sg.Server(prec, hbm_budget_bytes=150 * 10**9)
    ids = []
    t0 = time.perf_counter()
    i = 0
    while True:
        now = time.perf_counter() - t0
        while i < len(items) and arrivals[i] <= now:
            p, q0, ns = items[i]
            if eig_every and i % eig_every == eig_every - 1:
                ids.append(("eig", srv.submit_eigs(p, **eig_args[prec])))
            else:
                ids.append(("prop", srv.submit(p, 0.1, ns, order=64, factors=factors[i])))
            i += 1
        a, q = srv.progress(16)
        if a == 0 and q == 0:
            if i == len(items):
                break
            time.sleep(max(0.0, arrivals[i] - (time.perf_counter() - t0)))
    makespan = time.perf_counter() - t0
    res = []
    for kind, rid in ids:
        try:
            if kind == "eig":
                ev, rs, _, tm, nconv = srv.eig_result(rid)
                res.append({"kind": "eig", "evals": ev, "latency": tm[1], "converged": nconv})
            else:
                psi, nl, el, tm = srv.result(rid)
                res.append({"kind": "prop", "psi": psi, "energy": el, "latency": tm[1]})
        except sg.SgError as e:  # a refused or failed request is reported, not fatal
            res.append({"kind": kind, "failed": str(e), "latency": None})
    stats = srv.stats()
    srv.close()
    return res, makespan, stats


def run_serving(args, sg, synth, torch):
    """Streams of propagation and eigen requests (the serving configuration's
    distribution) through the server: mixed precision at every arrival rate,
    FP64 at the highest; the same propagation requests one at a time by
    sg_propagate in FP64 and in mixed precision (separating the effect of
    batching from that of precision); per-request errors of the mixed server's
    results against the FP64 server's."""
    items = synth.workload_C5(args.serve_requests, seed=5, Ds=tuple(range(6, args.serve_dmax + 1)),
                              Ls=tuple(range(4, args.serve_lmax + 1)), steps=(20, args.serve_steps_max))
    factors = [synth.coherent_factors(q0, p.L + 1) for p, q0, _ in items]
    # "rate" or "rate:n" (a stream of the first n requests at that rate)
    rates = [(float(r.split(":")[0]), min(len(items), int(r.split(":")[1])) if ":" in r else len(items))
             for r in args.serve_rates.split(",")]
    eig_args = {"mixed": dict(nev=4, block=4, tol=1e-5, max_it=300),
                "fp64": dict(nev=4, block=4, tol=1e-9, max_it=300)}
    E = args.serve_eig_every
    sweep = []
    mixed_res = None
    for rate, nreq in rates:
        res, makespan, st = run_stream(sg, "mixed", items[:nreq], factors[:nreq], rate, E, eig_args)
        lat = np.array([r["latency"] for r in res if "failed" not in r])
        sweep.append({"rate_req_s": rate, "requests": nreq, "failed": sum("failed" in r for r in res),
                      "applications_per_s": st["applications"] / makespan,
                      "requests_per_s": nreq / makespan, "makespan_s": makespan,
                      "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}})
        print("serving mixed:", json.dumps(sweep[-1]), file=sys.stderr, flush=True)
        if mixed_res is None or len(res) > len(mixed_res):
            mixed_res = res
    arms = set(args.serve_arms.split(","))
    top = max(r for r, _ in rates)
    fp64_server, res64 = None, None
    n64 = min(len(items), args.serve_fp64_requests) if args.serve_fp64_requests > 0 else len(items)
    if "fp64" in arms:
        res64, makespan64, st64 = run_stream(sg, "fp64", items[:n64], factors[:n64], top, E, eig_args)
        lat64 = np.array([r["latency"] for r in res64 if "failed" not in r])
        fp64_server = {"rate_req_s": top, "requests": n64, "failed": sum("failed" in r for r in res64),
                       "applications_per_s": st64["applications"] / makespan64,
                       "requests_per_s": n64 / makespan64, "makespan_s": makespan64,
                       "latency_s": {"p50": float(np.percentile(lat64, 50)), "p99": float(np.percentile(lat64, 99))}}
        print("serving fp64:", json.dumps(fp64_server), file=sys.stderr, flush=True)
    # per-request accuracy of the mixed server against the FP64 server (the
    # requests both ran: the FP64 stream is the mixed one's first n64)
    psi_err, drift_m, drift_64, eig_err = [], [], [], []
    for rm, r64 in zip(mixed_res, res64 or []):
        if "failed" in rm or "failed" in r64:
            continue
        if rm["kind"] == "prop":
            psi_err.append(float(np.linalg.norm(rm["psi"] - r64["psi"])))
            if len(rm["energy"]):
                drift_m.append(float(np.max(np.abs(rm["energy"] - rm["energy"][0]))))
                drift_64.append(float(np.max(np.abs(r64["energy"] - r64["energy"][0]))))
        else:
            eig_err.append(float(np.max(np.abs(rm["evals"] - r64["evals"]))))
    # the propagation requests one at a time, sg_propagate, each precision
    prop = [(it, f) for j, (it, f) in enumerate(zip(items[:n64], factors[:n64])) if not (E and j % E == E - 1)]
    per_request = {}
    for prec in (("fp64", "mixed") if "per_request" in arms else ()):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        apps = 0
        for (p, q0, ns), f in prop:
            with sg.sg_create(p, prec) as ctx:
                psi = sg.sg_product_state(ctx, f)
                d = torch.from_numpy(np.concatenate([psi, np.zeros_like(psi)])).cuda()
                sg.sg_propagate(ctx, d, 0.1, ns, order=64)
        torch.cuda.synchronize()
        per_request[prec] = {"seconds": time.perf_counter() - t1, "requests": len(prop)}
    n_eig = sum(1 for r in mixed_res if r["kind"] == "eig")
    desc = (f"{len(items)} requests, chained Henon-Heiles, D uniform in 6..{args.serve_dmax}, "
            f"L uniform in 4..{args.serve_lmax}, nb=nq=l+1; {len(items) - n_eig} propagation requests "
            f"(steps uniform in 20..{args.serve_steps_max}, order 64, dt 0.1, Gaussian displaced by 2.0) "
            f"and {n_eig} eigen requests (4 lowest, block Davidson, block 4); Poisson arrivals; budget 150 GB")
    head = max(sweep, key=lambda r: r["applications_per_s"])
    q = lambda a: {"max": float(np.max(a)), "median": float(np.median(a))} if len(a) else None
    return {"workload": desc, "precision": "mixed (server, continuous batching)",
            "applications_per_s": head["applications_per_s"], "rate_req_s": head["rate_req_s"],
            "latency_s": head["latency_s"], "sweep": sweep, "fp64_server": fp64_server,
            "per_request": ({
                "fp64": dict(per_request["fp64"], requests_per_s=per_request["fp64"]["requests"] /
                             per_request["fp64"]["seconds"]),
                "mixed": dict(per_request["mixed"], requests_per_s=per_request["mixed"]["requests"] /
                              per_request["mixed"]["seconds"]),
                "note": "propagation requests in arrival order, sg_propagate, one at a time"}
                if per_request else None),
            "accuracy_mixed_vs_fp64_server": {
                "psi_l2_error": q(psi_err), "energy_drift_mixed": q(drift_m), "energy_drift_fp64": q(drift_64),
                "eigenvalue_error": q(eig_err)}}


def run_batched(args, sg, synth, torch):
    """Many independent wavepacket problems per apply (sg_apply_H_batch) against
    the same problems applied one after another (sg_apply_H each), mixed and
    FP64.  Complex wavepackets: two real vectors per instance."""
    import concurrent.futures as cf
    items = synth.workload_C4(n=args.batch_instances, seed=4)
    nvec = 2
    out = {"workload": f"{len(items)} chained Henon-Heiles wavepackets, D uniform in {{4,6,8,10,12}}, "
                       f"L uniform in 6..10, nb=nq=l+1, Gaussian centres q0 ~ U[0,2] per mode, "
                       f"complex (2 real vectors) each",
           "unit": UNIT}
    stream = torch.cuda.current_stream()
    dev = torch.cuda.current_device()
    for prec in ("mixed", "fp64"):
        def make(it):
            torch.cuda.set_device(dev)
            return sg.sg_create(it[0], prec)
        with cf.ThreadPoolExecutor(8) as ex:
            ctxs = list(ex.map(make, items))
        b = sg.sg_batch_create(ctxs)
        xs = []
        for (p, q0), c in zip(items, ctxs):
            psi = sg.sg_product_state(c, synth.coherent_factors(q0, p.L + 1))
            psi /= np.linalg.norm(psi)
            xs.append(np.concatenate([psi, np.roll(psi, 1)]))
        x = torch.from_numpy(np.concatenate(xs)).cuda()
        y = torch.empty_like(x)
        offs = [nvec * int(o) for o in b.offsets]
        xv = [x[offs[j]:offs[j + 1]] for j in range(len(ctxs))]
        yv = [y[offs[j]:offs[j + 1]] for j in range(len(ctxs))]
        res = {}
        for mode in ("batched", "per_instance"):
            def step():
                if mode == "batched":
                    sg.sg_apply_H_batch(b, x, y, nvec, stream)
                else:
                    for c, a, o in zip(ctxs, xv, yv):
                        sg.sg_apply_H(c, a, o, nvec, stream)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.batch_steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.batch_steps
            res[mode] = {"value": len(ctxs) * nvec / (ms * 1e-3), "ms_per_apply": ms}
        res["launches_per_apply"] = b.launches_per_apply
        for c in ctxs:
            if sg.sg_device_error(c):
                raise RuntimeError(f"device error in the batched {prec} apply")
        sg.sg_batch_destroy(b)
        for c in ctxs:
            sg.sg_destroy(c)
        del x, y, xv, yv
        torch.cuda.empty_cache()
        out[prec] = res
    return out


def time_device(ctx, xd, yd, nvec, steps, warmup, flush, torch, sg, sharded_terms=False):
    """Per-step CUDA-event times of sg_apply_H (or, with sharded_terms, of this
    rank's share of the terms, the integer all-reduce and the finish)."""
    stream = torch.cuda.current_stream()
    acc = None
    if sharded_terms:
        from paper_2111_13655_gb300 import sharded
        acc = torch.zeros(sg.acc_words(ctx, nvec), dtype=torch.int64, device="cuda")
        apply = lambda: sharded.apply_H_sharded(ctx, xd, yd, nvec, acc=acc, stream=stream)
    else:
        apply = lambda: sg.sg_apply_H(ctx, xd, yd, nvec, stream)
    for _ in range(warmup):
        apply()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()                       # L2 flush, outside the timed interval
        ev[i][0].record(stream)
        apply()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nvec", type=int, default=8)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu1-seconds", type=float, default=5.0)
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-eig-every", type=int, default=8, help="every n-th request is an eigen request (0: none)")
    ap.add_argument("--serve-arms", default="mixed,fp64,per_request",
                    help="serving arms: mixed (server at every rate), fp64 (server at the top rate), per_request")
    ap.add_argument("--serve-rates", default="10,100,1000")
    ap.add_argument("--serve-fp64-requests", type=int, default=0,
                    help="FP64 server and one-at-a-time arms on the stream's first n requests (0: all)")
    ap.add_argument("--serve-dmax", type=int, default=20)
    ap.add_argument("--serve-lmax", type=int, default=6)
    ap.add_argument("--serve-steps-max", type=int, default=200)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-only", action="store_true", help="only the serving leg (its JSON line alone)")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--L", type=int, default=10, help="Smolyak level of the D=12 workload (10: the benchmark)")
    ap.add_argument("--precisions", default="mixed,fp64,df64")
    ap.add_argument("--tune", action=argparse.BooleanOptionalAction, default=True,
                    help="run sg_tune on each arm's context before timing (--no-tune: the default plan)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--peak-seconds", type=float, default=1.0, help="0: skip the peak measurement")
    ap.add_argument("--sharding", default="replicas", choices=["replicas", "terms"],
                    help="N > 1: independent replicas (weak scaling) or one problem's terms split over the "
                         "ranks with one integer all-reduce per apply (strong scaling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2111_13655_gb300 as sg
    from paper_2111_13655_gb300 import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.serving_only:
        # the serving leg alone (used for the longer streams of the serving configuration)
        print(json.dumps({"metric": METRIC, "serving": run_serving(args, sg, synth, torch)}), flush=True)
        return 0
    rep = Replicas("nccl")
    world, rank = rep.world, rep.rank
    barrier = rep.barrier

    # CPU baseline before any GPU work on rank 0 (the oracle's OpenMP pool
    # starts in this process; no fork happens after CUDA initialisation).
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as orc
        orc.build()
        r, desc, cores = oracle_sample_rate(synth.workload_C3(), 646646, args.cpu_seconds, 7)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        if args.cpu1_seconds > 0:  # the same oracle on one host thread
            r1, desc1, _ = oracle_sample_rate(synth.workload_C3(), 646646, args.cpu1_seconds, 8, threads=1)
            cpu["single_thread"] = {"value": r1, "unit": UNIT, "cores": 1, "sample": desc1}

    peaks = None
    if args.peak_seconds > 0:
        peaks = measure_peaks(sg, torch, args.peak_seconds)
    else:
        peaks = {"fp32": None, "fp64": None, "note_fp32": "not measured", "note_fp64": "not measured",
                 "derived_fp32": None}
    p = synth.workload_C3(L=args.L)
    nvec = args.nvec
    results = {}
    for prec in args.precisions.split(","):
        ctx = sg.sg_create(p, prec)
        tuned = args.tune and not (args.sharding == "terms" and world > 1)
        if tuned:
            # the library's own autotuner picks the schedule for these applies
            # (slicing target, block/warp split, shared-memory budget) by timing
            sg.sg_tune(ctx, nvec)
        plan = dict(sg.sg_tune_plan(ctx), tuned=bool(tuned))
        n = ctx.n_cs
        # replicas: independent inputs per rank; term sharding: one problem, the same x everywhere
        x = synth.random_vectors(n, nvec, 11 + (0 if args.sharding == "terms" else rank))
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
        steps = args.steps if prec == "mixed" else args.fp64_steps
        warm = max(3, args.warmup if prec == "mixed" else 3)
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            times = time_device(ctx, xd, yd, nvec, steps, warm, flush, torch, sg,
                                sharded_terms=args.sharding == "terms" and world > 1)
        barrier()
        torch.cuda.synchronize()
        total_ms = rep.max_over_ranks(sum(times))
        derr = sg.sg_device_error(ctx)
        if derr:
            raise RuntimeError(f"device error code {derr} in the {prec} apply")
        lv, _ = sg.sg_term_levels(ctx)
        f_alg = algorithmic_flops_per_vector(lv) * nvec
        ms = total_ms / steps
        units = nvec * steps if args.sharding == "terms" and world > 1 else None
        if prec == "df64":
            # double-float: F_alg / 2 multiply-adds of DF_INSTR_PER_FMA FP32
            # instructions each, against the FP32 issue rate (fma rate / 2)
            instr = f_alg / 2 * DF_INSTR_PER_FMA
            peak = peaks["fp32"] / 2 if peaks["fp32"] else None
            achieved = instr / (statistics.mean(times) * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32-instructions/s",
                    "frac": achieved / peak if peak else None, "traffic": TRAFFIC_BYTES[prec],
                    "flops_per_launch": f_alg, "fp32_instructions_per_launch": instr,
                    "peak_source": "measured",
                    "peak_note": "half the measured FP32 fma rate (one instruction per lane per cycle); "
                                 + str(peaks["note_fp32"])}
        else:
            peak = peaks["fp32"] if prec == "mixed" else peaks["fp64"]
            achieved = f_alg / (statistics.mean(times) * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if peak else None,
                    "traffic": TRAFFIC_BYTES[prec],
                    "flops_per_launch": f_alg,
                    "peak_source": "measured",
                    "peak_note": peaks["note_fp32" if prec == "mixed" else "note_fp64"],
                    "peak_derived": peaks["derived_fp32"] if prec == "mixed" else None}
        results[prec] = {
            "value": (units / (total_ms * 1e-3) if units else replica_throughput(world, nvec * steps, total_ms * 1e-3)),
            "ms_per_step": ms, "steps": steps,
            "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
            "roofline": roof,
            "clocks": clk.summary(),
            "plan": plan,
        }
        if prec == "mixed" and not args.no_e2e:
            # end to end through the host-buffer entry point: H2D + apply + D2H per step
            xh = torch.from_numpy(x).pin_memory()
            yh = torch.empty_like(xh).pin_memory()
            for _ in range(2):
                sg.sg_apply_H_host(ctx, xh, yh, nvec)
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                sg.sg_apply_H_host(ctx, xh, yh, nvec)
            e2e_s = rep.max_over_ranks(time.perf_counter() - t0)
            results[prec]["e2e"] = {"value": replica_throughput(world, nvec * args.steps, e2e_s), "unit": UNIT,
                                    "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(x.nbytes)}
        sg.sg_destroy(ctx)
        del xd, yd, flush
        torch.cuda.empty_cache()

    serving = None
    # single-GPU legs: at N > 1 they would hold the other GPUs idle
    if world == 1 and not args.no_serving:
        serving = run_serving(args, sg, synth, torch)
    batched = None
    if world == 1 and not args.no_batched:
        batched = run_batched(args, sg, synth, torch)

    if rank == 0:
        m = results.get("mixed") or next(iter(results.values()))
        f = results.get("fp64")
        d = results.get("df64")
        line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": m["steps"],
                "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
                "scaling": "strong" if args.sharding == "terms" and world > 1 else "weak", "vs_baseline": None,
                "dtype": "f32" if "mixed" in results else "f64",
                "data": "synthetic", "config": bench_config(args, world),
                "latency_ms": m["latency_ms"], "roofline": m["roofline"], "clocks": m["clocks"],
                "e2e": m.get("e2e"), "gpu_launches": LAUNCHES_PER_APPLY * m["steps"], "plan": m.get("plan"),
                "fp64": ({"value": f["value"], "unit": UNIT, "ms_per_step": f["ms_per_step"], "steps": f["steps"],
                          "latency_ms": f["latency_ms"], "roofline": f["roofline"], "clocks": f["clocks"],
                          "plan": f.get("plan")}
                         if f else None),
                "df64": ({"value": d["value"], "unit": UNIT, "ms_per_step": d["ms_per_step"], "steps": d["steps"],
                          "precision": "double-float contractions (pairs of FP32, ~48 bits), FP64 accumulation",
                          "latency_ms": d["latency_ms"], "roofline": d["roofline"], "clocks": d["clocks"],
                          "plan": d.get("plan")}
                         if d else None),
                "peaks": {k: v for k, v in peaks.items() if k != "clocks"} if peaks else None,
                "cpu_baseline": cpu, "batched": batched, "serving": serving}
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
