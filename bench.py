#!/usr/bin/env python3
"""Benchmark: trimmed mass-matrix nnz formed per second on GB300.

Workload (the paper's "plain FP64" shape, Sect. 4): twelve trimmed patches --
degrees p = 3, 4, 5 x 128^2 and 512^2 elements x hybrid Gauss and
discontinuous weighted quadrature -- each a perturbed bilinear geometry
(c = det J) with a seeded 12-point cubic B-spline hole of radius 0.3 +- 0.05.
One step forms all twelve from their host descriptors: every table kernel
(WQ points and weights, classification, cut-element rules, DWQ rules, CSR
pattern) and the formation kernels, writing FP64 CSR into resident buffers.
value = nnz of the twelve matrices / step time.

The --impl reference arm times the CPU oracle (single thread) on a bounded
sample of the same workload: full set-up of each patch plus a seeded sample
of rows, extrapolated to the whole matrix.

Besides the step, the JSON line carries: e2e (the same step with the CSRs
copied to pinned host memory), the roofline of the interior-row kernel, the
formation-only rates of the three precisions, the 512-patch batched run, the
density-gradient workload (256^2, p = 3), the 1024^2 precision study with its
L2 projections, and the extended B-spline projection at 512^2, p = 4; each
section can be skipped with its --no-* flag.

Multi-GPU: the path has no exchange step; each rank forms its own copy of the
workload (weak scaling, replicas), timings are max-reduced over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = [(p, nel, m) for nel in (128, 512) for p in (3, 4, 5) for m in ("hybrid", "dwq")]
METRIC = "trimmed mass-matrix nnz formed/sec"
UNIT = "nnz/s"


def specs():
    return [synth.config2(p=p, nel=nel, method=m) for (p, nel, m) in WORKLOAD]


def select_case(case):
    """--case p,nel,method restricts the workload to one patch of the sweep
    (used as the profiling driver)."""
    global WORKLOAD
    p, nel, m = case.split(",")
    WORKLOAD = [(int(p), int(nel), m)]


def workload_name():
    return ("config-2 sweep: p in {3,4,5} x {128^2, 512^2} elements x {hybrid Gauss, DWQ}; "
            "perturbed bilinear geometry (c = det J), seeded 12-point cubic B-spline hole "
            "r = 0.3 +- 0.05; FP64 CSR")


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# algorithmic work of the interior-row kernel (for the roofline)


def _points_per_element(p, nel):
    npe = np.full(nel, 2, dtype=np.int64)
    npe[0] = npe[-1] = p + 1
    return npe


def _overlap_points(p, nel):
    """ov[i, r] = WQ points in supp B_i cap supp B_j, j = i - p + r."""
    n = nel + p
    npe = _points_per_element(p, nel)
    cs = np.concatenate([[0], np.cumsum(npe)])
    ov = np.zeros((n, 2 * p + 1), dtype=np.int64)
    for i in range(n):
        for r in range(2 * p + 1):
            j = i - p + r
            if j < 0 or j >= n:
                continue
            lo = max(max(0, i - p), max(0, j - p))
            hi = min(min(nel - 1, i), min(nel - 1, j))
            if hi >= lo:
                ov[i, r] = cs[hi + 1] - cs[lo]
    return ov, cs


def interior_flops(p, nel, fstate):
    """FP64 flops the sum-factorised WQ contraction of the interior rows needs:
    stage 2, one FMA per point of supp B_i cap supp B_j in direction 1 for
    every output; stage 1, one FMA per point of the same overlap in direction
    2 for every (i2, j2, k1) with k1 a point some interior row of i2 uses."""
    n = nel + p
    ov, cs = _overlap_points(p, nel)
    fs = fstate.reshape(n, n)  # [i2, i1]
    interior = fs == 1
    valid = np.zeros((n, 2 * p + 1), dtype=bool)
    for r in range(2 * p + 1):
        j = np.arange(n) - p + r
        valid[:, r] = (j >= 0) & (j < n)
    s1 = (2 * ov * valid).sum(axis=1)         # per i1: sum_r1 2 ov1
    nr = valid.sum(axis=1)                    # valid r per i
    stage2 = float(np.sum(interior * (nr[:, None] * s1[None, :])))
    qlo = np.array([cs[max(0, i - p)] for i in range(n)])
    qhi = np.array([cs[min(nel - 1, i) + 1] for i in range(n)])
    stage1 = 0.0
    s2 = (2 * ov * valid).sum(axis=1)
    for i2 in range(n):
        rows = np.where(interior[i2])[0]
        if len(rows) == 0:
            continue
        mask = np.zeros(cs[-1], dtype=bool)
        for i1 in rows:
            mask[qlo[i1]:qhi[i1]] = True
        stage1 += float(s2[i2] * mask.sum())
    return stage1 + stage2


# ---------------------------------------------------------------------------


def minnorm_flops(m, N):
    """FP64 operations of the minimum-norm solution of an m x N system (m <= N)
    by Householder reflectors applied from the right (reading R2): per reflector
    k the norm of its part of row k (2 (N - k)), its application to the m - k - 1
    rows below (a dot product and an update, 4 (N - k) each) and its step of the
    back transformation (4 (N - k)); then the forward substitution (m^2)."""
    return sum(2 * (N - k) + 4 * (m - k - 1) * (N - k) + 4 * (N - k) for k in range(m)) + m * m


def wq_points_per_element(p, nel, nested=()):
    """Reading R1 (and R5 for the elements next to a disc): p + 1 points in the
    two end elements and in the elements listed in `nested`, 2 elsewhere."""
    return [p + 1 if e in (0, nel - 1) or e in nested else 2 for e in range(nel)]


def setup_minnorm_flops(p, nel1, nel2, ndisc):
    """Algorithmic FP64 operations of the set-up's min-norm solves: the WQ
    weights of every test function of both directions (Eq. 5) and, per disc
    knot, the 2p refined systems of the DWQ rule (Sect. 3.3: t inserted p times,
    nested points next to it; counted for a disc away from the patch's ends)."""
    total = 0
    for nel in (nel1, nel2):
        n = nel + p
        cnt = wq_points_per_element(p, nel)
        for i in range(n):
            lo, hi = max(0, i - p), min(i, nel - 1)
            N = sum(cnt[lo:hi + 1])
            m = min(n - 1, i + p) - max(0, i - p) + 1
            total += minnorm_flops(m, N)
    # one interior disc of direction 1: refined knots with t of multiplicity p + 1
    nel = nel1
    s = nel // 2
    U = synth.open_uniform_knots(p, nel)
    t = U[p + s]
    R = np.concatenate([U[:p + s + 1], [t] * p, U[p + s + 1:]])
    cnt = wq_points_per_element(p, nel, nested=(s - 1, s))
    bp = U[p:p + nel + 1]
    nref = len(R) - p - 1

    def supp(l):
        return R[l], R[l + p + 1]

    per_disc = 0
    for l in range(s, s + 2 * p):
        a, b = supp(l)
        m = sum(1 for k in range(max(0, l - p), min(nref, l + p + 1))
                if min(b, supp(k)[1]) > max(a, supp(k)[0]))
        N = sum(cnt[e] for e in range(nel) if bp[e] >= a and bp[e + 1] <= b)
        per_disc += minnorm_flops(m, N)
    return total + ndisc * per_disc


def fp64_peak_gflops():
    """FP64 peak of a GB300 from its unit counts and clock: 152 SMs x 2 DFMA
    per clock x 2 flop x 2.07 GHz (a DFMA-loop probe measured 1 255.6 GFLOP/s)."""
    return 152 * 2 * 2 * 2.07


# DRAM bytes per k_interior launch over the timed step (dram__bytes_read.sum +
# dram__bytes_write.sum of its 12 launches / 12, one ncu capture kept under
# profiles/), valid only for the kernel sources it was taken with
INTERIOR_TRAFFIC = {
    "bytes_per_launch": 69440533,
    "sources_sha256": {
        "paper_2101_08053_gb300/csrc/tw_interior.cuh":
            "9b0b894c99a4c477aefd4f279970588eec901791beef3fc5015b0c6ba72d578f",
    },
}


def interior_traffic():
    import hashlib
    for rel, h in INTERIOR_TRAFFIC["sources_sha256"].items():
        with open(os.path.join(ROOT, rel), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != h:
                return None
    return INTERIOR_TRAFFIC["bytes_per_launch"]


def max_over_ranks(x, world, device):
    """The largest per-rank value (a step time) over all ranks; the identity
    on one rank.  The job's time is the slowest rank's."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: every rank processes units_per_rank units (weak
    scaling, replicas) in the slowest rank's ms."""
    return world * units_per_rank / (ms * 1e-3)


def pin_spec(spec, torch, keep):
    """The spec with its host arrays (knots, control nets, curve control
    points) moved to pinned host memory, so the library's copies of the
    descriptors are DMA transfers; `keep` holds the pinned buffers."""
    def pin(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
        keep.append(t)
        return t.numpy()

    s = dict(spec)
    s["knots"] = [pin(u) for u in spec["knots"]]
    s["trim"] = dict(spec["trim"])
    if spec["trim"].get("ctrl") is not None:
        s["trim"]["ctrl"] = pin(spec["trim"]["ctrl"])
    s["geom"] = dict(spec["geom"])
    if spec["geom"].get("ctrl") is not None:
        s["geom"]["ctrl"] = pin(spec["geom"]["ctrl"])
    return s


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2101_08053_gb300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    api.load()
    stream = torch.cuda.current_stream()
    pinned = []
    sp = [pin_spec(s_, torch, pinned) for s_ in specs()]
    # one build per spec to size the resident outputs
    outs, infos = [], []
    for s in sp:
        P = api.Patch(s)
        outs.append(P.alloc_csr("fp64"))
        infos.append((P.n_rows, P.nnz, P.n_cut_fns, P.n_cut_elems, P.n_dwq_rows, P.n_discs))
        P.close()
    nnz_step = sum(i[1] for i in infos)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the patches are independent: each is one job of tw_run_jobs (created and
    # formed on its own stream by the library's native thread pool), largest
    # first; `--streams` native threads take the jobs
    order = sorted(range(len(sp)), key=lambda k: -infos[k][1])
    jstreams = [torch.cuda.Stream(device=dev) for _ in order]
    jobs = api.Jobs([sp[k] for k in order], jstreams, outs=[outs[k] for k in order],
                    nthreads=max(1, args.streams))
    ns = max(1, min(args.streams, len(sp)))
    streams = jstreams

    def step(tag=None):
        start = torch.cuda.Event()
        start.record(stream)
        for s_ in jstreams:
            s_.wait_event(start)
        jobs.run()
        jobs.destroy()  # each destroy waits for its patch's stream
        for s_ in jstreams:
            stream.wait_stream(s_)

    def form_one(idx):
        P = api.Patch(sp[idx])
        P.form_mass("fp64", out=outs[idx])
        P.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local_rank) if rank == 0 else None
    if clk:
        clk.start()
        time.sleep(0.4)
    launches0 = api.launch_count()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step("timed_step")
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = api.launch_count() - launches0
    clocks = clk.stop() if clk else None
    # stage times of the overlapped step, from extra (untimed) steps with the
    # stage profiler on: its events are not part of the timed region
    api.profile_enable(True)
    for st in api.STAGES:
        api.profile_read(st)
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        step()
        torch.cuda.synchronize()
    api.profile_enable(False)
    stage_batched = {k: api.profile_read(k) for k in api.STAGES}
    # kernels of different patches overlap in the batched step, so the
    # per-kernel roofline is timed over a second pass of the same steps on one
    # stream (events on the launching stream, L2 flushed between steps)
    api.profile_enable(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        for idx in range(len(sp)):
            form_one(idx)
        torch.cuda.synchronize()
    api.profile_enable(False)
    stage = {k: api.profile_read(k) for k in api.STAGES}
    ms = max_over_ranks(float(np.mean(times)), world, dev)
    value = job_rate(world, nnz_step, ms)

    # end to end through the C-ABI with host buffers: descriptors from host
    # memory, CSR copied back to pinned host buffers, inside the timed region
    host = [(torch.empty(o[0].numel(), dtype=torch.int64, pin_memory=True),
             torch.empty(o[1].numel(), dtype=torch.int32, pin_memory=True),
             torch.empty(o[2].numel(), dtype=torch.float64, pin_memory=True)) for o in outs]
    h2d = 0
    for s in sp:
        h2d += sum(np.asarray(u).nbytes for u in s["knots"]) + np.asarray(s["trim"]["ctrl"]).nbytes
        h2d += np.asarray(s["geom"]["ctrl"]).nbytes
    d2h = sum(o[0].numel() * 8 + o[1].numel() * 4 + o[2].numel() * 8 for o in outs)

    e2e_jobs = api.Jobs([sp[k] for k in order], jstreams, outs=[outs[k] for k in order],
                        host=[host[k] for k in order], nthreads=max(1, args.streams))

    def e2e_step():
        start = torch.cuda.Event()
        start.record(stream)
        for s_ in jstreams:
            s_.wait_event(start)
        e2e_jobs.run()
        e2e_jobs.destroy()
        torch.cuda.synchronize()

    e2e_step()
    et = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        et.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(float(np.mean(et)) * 1e3, world, dev)

    # the reduced-precision forms against the plain FP64 GPU form: formation
    # only (patch tables resident), serialised, relative Frobenius error
    modes = {}
    patches = [api.Patch(s_) for s_ in sp]
    ref = []
    for P, o in zip(patches, outs):
        P.form_mass("fp64", out=o)
        ref.append(o[2][:P.nnz].clone())
    for mode in ("fp64", "fp32x2", "fp32"):
        mo = [P.alloc_csr(mode) for P in patches]
        for P, o in zip(patches, mo):
            P.form_mass(mode, out=o)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for P, o in zip(patches, mo):
                P.form_mass(mode, out=o)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        num = sum(float(torch.linalg.norm(o[2][:P.nnz].double() - r_) ** 2)
                  for P, o, r_ in zip(patches, mo, ref))
        den = sum(float(torch.linalg.norm(r_) ** 2) for r_ in ref)
        ms_ = float(np.mean(ts))
        modes[mode] = {"form_nnz_per_s": nnz_step / (ms_ * 1e-3), "form_ms": round(ms_, 3),
                       "rel_frobenius_vs_fp64_gpu": math.sqrt(num / den)}
        del mo
    for P in patches:
        P.close()

    # batched variant (config 4): 512 patches of seeded degree 2..6, 16..256
    # elements per direction, ellipse or 8-point spline holes; tables built on
    # the streams, then every matrix formed by one persistent launch replayed
    # from a CUDA graph (tiles by the autotuner), FP64 and FP32
    remark1 = None if args.no_remark1 else run_remark1(api, torch, args, stream, flush)
    batched = None
    if not args.no_batched:
        batched = run_batched(api, torch, args, stream, streams, dev)
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(api, torch, args, stream)
    precision = None
    if not args.no_precision:
        precision = run_precision(api, torch, args, stream, flush)
    extension = None
    if not args.no_extension:
        extension = run_extension(api, torch, args, stream)

    # roofline of the dominant kernel (interior rows, FP64 DFMA-bound)
    flops = 0.0
    for s in sp:
        P = api.Patch(s)
        _, fs, _ = P.states()
        flops += interior_flops(s["p"], s["nel"][0], fs.cpu().numpy())
        P.close()
    int_ms, int_n = stage["interior"]
    launches_per_step = int_n / max(1, args.steps)
    avg_launch_ms = int_ms / max(1, int_n)
    flops_per_launch = flops / max(1, launches_per_step)
    achieved = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12
    peak = fp64_peak_gflops() / 1e3
    # the set-up's min-norm solves (WQ weights, DWQ rules), timed in the same
    # serialised pass by their profiler stages
    su_flops = sum(setup_minnorm_flops(s_["p"], s_["nel"][0], s_["nel"][1], info[5])
                   for s_, info in zip(sp, infos))
    su_ms = (stage["wq_weights"][0] + stage["dwq"][0]) / max(1, args.steps)
    su_achieved = su_flops / (su_ms * 1e-3) / 1e12 if su_ms > 0 else 0.0
    stage_ms = {k: round(v[0] / max(1, args.steps), 3) for k, v in stage.items() if v[1]}
    stage_ms_batched = {k: round(v[0] / max(1, args.steps), 3) for k, v in stage_batched.items()
                        if v[1]}
    return {
        "value": value, "ms": ms, "nnz_step": nnz_step, "infos": infos, "launches": launches,
        "clocks": clocks, "e2e_ms": e2e_ms, "h2d": h2d, "d2h": d2h, "stage_ms": stage_ms,
        "stage_ms_batched": stage_ms_batched, "modes": modes, "batched": batched,
        "remark1": remark1,
        "adjoint": adjoint, "precision": precision, "extension": extension,
        "roofline": {"bound": "alu", "kernel": "k_interior (interior rows, WQ + sum factorisation)",
                     "achieved": round(achieved, 4), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4), "traffic": interior_traffic(),
                     "flops_per_launch": flops_per_launch, "avg_launch_ms": avg_launch_ms,
                     "timing": "events on the launching stream over a serialised pass of the "
                               "same steps (the batched step overlaps kernels of different "
                               "patches)",
                     "peak_source": "GB300 unit counts x max clock (152 SMs x 2 DFMA/clk x "
                                    "2.07 GHz); a DFMA probe measured 1.2556 TFLOP/s"},
        "roofline_setup": {"bound": "alu",
                           "kernel": "k_wq_weights + k_dwq_build (the set-up's min-norm solves, "
                                     "Eq. 5 and Sect. 3.3)",
                           "achieved": round(su_achieved, 5), "peak": peak, "unit": "TFLOP/s",
                           "frac": round(su_achieved / peak, 5), "traffic": None,
                           "flops_per_step": su_flops, "ms_per_step": round(su_ms, 4),
                           "timing": "stage events around the two kernels in the serialised pass",
                           "flops": "Householder LQ per system: reflector norms, application "
                                    "to the rows below, back transformation, forward "
                                    "substitution (bench.minnorm_flops)"},
    }


def run_batched(api, torch, args, stream, streams, dev):
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    specs4 = [synth.config4_patch(rng, method="hybrid") for _ in range(args.batched_patches)]
    patches = [None] * len(specs4)
    ns = len(streams)

    def build(k):
        torch.cuda.set_device(dev)
        with torch.cuda.stream(streams[k]):
            for idx in range(k, len(specs4), ns):
                patches[idx] = api.Patch(specs4[idx])

    t0 = time.perf_counter()
    th = [threading.Thread(target=build, args=(k,)) for k in range(ns)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    nnz = sum(P.nnz for P in patches)
    res = {"patches": len(patches), "nnz": nnz, "setup_s_4_streams": round(setup_s, 3),
           "p_hist": {str(p): sum(1 for P in patches if P.p == p) for p in range(2, 7)}}
    for mode in ("fp64", "fp32"):
        outs = [P.alloc_csr(mode) for P in patches]
        t0 = time.perf_counter()
        B = api.Batch(patches, outs, mode)
        create_s = time.perf_counter() - t0
        B.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.run()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.mean(ts))

        # the same patches formed one tw_form_mass call per patch, serially on
        # one stream and spread over the streams, into the same buffers
        def per_patch(nstreams):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sts = [stream] if nstreams == 1 else streams[:nstreams]
            for st in sts:
                st.wait_event(e0)
            for k, P in enumerate(patches):
                P.form_mass(mode, out=outs[k], stream=sts[k % len(sts)])
            for st in sts:
                ev = torch.cuda.Event()
                ev.record(st)
                stream.wait_event(ev)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        per = {}
        for nst in (1, len(streams)):
            per_patch(nst)
            t = float(np.mean([per_patch(nst) for _ in range(max(1, args.steps))]))
            per["streams_%d" % nst] = {"form_ms": round(t, 3), "form_nnz_per_s": nnz / (t * 1e-3)}
        best = min(v["form_ms"] for v in per.values())
        res[mode] = {"form_nnz_per_s": nnz / (ms * 1e-3), "form_ms": round(ms, 3),
                     "batch_create_s": round(create_s, 3), "items": B.items,
                     "persistent_blocks": B.blocks,
                     "tiles": {str(p): t for p, t in B.tiles.items() if any(P.p == p for P in patches)},
                     "per_patch_launches": per,
                     "vs_per_patch": round(best / ms, 3)}
        B.close()
        del outs
    for P in patches:
        P.close()
    return res


def run_remark1(api, torch, args, stream, flush):
    """The cut rows' Gauss part two ways, config-2 geometry and hole at 512^2,
    hybrid Gauss, p = 3..6: element matrices of the regular elements near the
    curve (formed in set-up) gathered by the cut rows, against Remark 1's
    row-level sum factorisation (Sect. 3.2).  Device times from the stage
    profiler (events on the launching stream), L2 flushed before each pass."""
    out = {}
    for p in (3, 4, 5, 6):
        spec = synth.config2(p=p, nel=512, method="hybrid")
        api.profile_enable(True)
        for st in api.STAGES:
            api.profile_read(st)
        gm, cr_e, cr_s = [], [], []
        P = None
        for rep in range(max(2, args.steps)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if P is not None:
                P.close()
            P = api.Patch(spec)
            torch.cuda.synchronize()
            gm.append(api.profile_read("gaussmat")[0])
            api.profile_read("setup")
            csr = P.alloc_csr("fp64")
            for rowsf, acc in ((False, cr_e), (True, cr_s)):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                api.profile_read("cutrows")
                P.form_mass("fp64", out=csr, rowsf=rowsf)
                torch.cuda.synchronize()
                acc.append(api.profile_read("cutrows")[0])
            api.profile_read("interior")
        api.profile_enable(False)
        e_ms = float(np.mean(gm[1:])) + float(np.mean(cr_e[1:]))
        s_ms = float(np.mean(cr_s[1:]))
        out["p%d" % p] = {"cut_rows": P.n_cut_fns, "element_matrices_ms": round(float(np.mean(gm[1:])), 4),
                          "gather_ms": round(float(np.mean(cr_e[1:])), 4),
                          "element_form_ms": round(e_ms, 4), "remark1_ms": round(s_ms, 4),
                          "remark1_over_element": round(s_ms / e_ms, 3)}
        P.close()
    return out


def run_precision(api, torch, args, stream, flush):
    """Precision variant: p = 4 and p = 6, 1024^2 elements, perturbed geometry
    (c = det J), circular hole r = 0.3, hybrid Gauss.  Per mode: formation time
    (patch tables resident), the interior-row kernel's share and its CSR write
    rate, the relative Frobenius error of M against the FP64 GPU form, and the
    L2 projection of f = sin(pi x) sin(pi y) with that matrix (CG in FP64 on the
    matrix widened to FP64): its L2 error and its L2 distance from the FP64
    projection (coefficient vectors are not compared: the cut functions with
    tiny visible support make them ill-determined)."""
    f = synth.func_sinsin()
    out = {}
    for p in (4, 6):
        spec = synth.config3(p=p)
        P = api.Patch(spec)
        res = {"n_rows": P.n_rows, "nnz": P.nnz, "interior_rows": P.n_interior}
        _, _, act = P.states()
        act = act.long()
        ref = None
        g64 = None
        n64 = None
        for mode in ("fp64", "fp32x2", "fp32"):
            csr = P.form_mass(mode)
            torch.cuda.synchronize()
            api.profile_enable(True)
            for st in ("interior", "cutrows"):
                api.profile_read(st)
            ts = []
            for _ in range(max(1, args.steps)):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.form_mass(mode, out=(csr[0], csr[1], csr[2]))
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            im, ic = api.profile_read("interior")
            cm, cc = api.profile_read("cutrows")
            api.profile_enable(False)
            ms = float(np.mean(ts))
            vb = 4 if mode == "fp32" else 8
            r = {"form_ms": round(ms, 3), "form_nnz_per_s": P.nnz / (ms * 1e-3),
                 "interior_kernel_ms": round(im / max(1, ic), 4),
                 "cutrows_ms": round(cm / max(1, cc), 4)}
            val = csr[2][:P.nnz].double()
            if ref is None:
                ref = val.clone()
            r["rel_frobenius_vs_fp64_gpu"] = float(torch.linalg.norm(val - ref) /
                                                   torch.linalg.norm(ref))
            u, it, rel = P.l2_project(f, (csr[0], csr[1], val), tol=1e-10, maxit=4000,
                                      check=False)
            L, _ = P.loss(u, f)
            r["l2_error"] = math.sqrt(max(float(L.item()), 0.0))
            r["cg_iterations"] = it
            r["cg_relres"] = rel
            if g64 is None:
                # the FP64 projection as a spline of the patch's own space
                coef = torch.zeros(P.n1 * P.n2, dtype=torch.float64, device=u.device)
                on = act >= 0
                coef[on] = u[act[on]]
                g64 = {"kind": "spline", "p": spec["p"], "knots": spec["knots"],
                       "coef": coef.view(P.n2, P.n1).cpu().numpy()}
                n64 = math.sqrt(float(P.loss(torch.zeros_like(u), g64)[0].item()))
            r["l2_rel_diff_vs_fp64_projection"] = math.sqrt(
                max(float(P.loss(u, g64)[0].item()), 0.0)) / n64
            r["csr_write_bytes_per_nnz"] = vb + 4
            res[mode] = r
            del csr, val
        out["p%d" % p] = res
        P.close()
    return out


def run_adjoint(api, torch, args, stream):
    """Differentiation workload: 256^2 elements, p = 3, circular hole, density
    spline of degree 2 with 32 x 32 coefficients (c = rho); loss of projecting
    a Gaussian bump g onto the trimmed space, gradient w.r.t. the 1024 density
    coefficients.  Forward = patch set-up + formation + CG + loss; backward =
    adjoint CG + gradient kernels."""
    spec = synth.config5()
    g = synth.func_gauss(8.0, 0.3, 0.7)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0, e1 = ev(), ev()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    api.profile_enable(True)
    for _ in range(max(1, args.warmup)):
        P = api.Patch(spec)
        csr = P.form_mass("fp64")
        u, _, _ = P.l2_project(g, csr, tol=1e-12)
        L, dl = P.loss(u, g)
        P.l2_project_adjoint(g, csr, dl, u, tol=1e-12)
        P.close()
    torch.cuda.synchronize()
    for st in ("loss", "adjoint", "cg"):
        api.profile_read(st)
    acc = {"setup_form": [], "project": [], "loss": [], "adjoint": []}
    its = []
    for _ in range(args.steps):
        def mk():
            Q = api.Patch(spec)
            return Q, Q.form_mass("fp64")
        (P, csr), t_sf = timed(mk)
        (u, it, _), t_pr = timed(lambda: P.l2_project(g, csr, tol=1e-12))
        (L, dl), t_lo = timed(lambda: P.loss(u, g))
        (gr, lam, it2, _), t_ad = timed(lambda: P.l2_project_adjoint(g, csr, dl, u, tol=1e-12))
        its.append((it, it2))
        for k, t in zip(acc, (t_sf, t_pr, t_lo, t_ad)):
            acc[k].append(t)
        P.close()
    cg_ms, cg_n = api.profile_read("cg")
    gr_ms, gr_n = api.profile_read("adjoint")
    lo_ms, lo_n = api.profile_read("loss")
    api.profile_enable(False)
    n = max(1, args.steps)
    res = {k: round(float(np.mean(v)), 3) for k, v in acc.items()}
    return {"workload": "256x256 elements, p = 3, circle r = 0.25, density q = 2, 32 x 32 "
                        "coefficients; g = Gaussian bump",
            "ms": res, "forward_ms": round(res["setup_form"] + res["project"] + res["loss"], 3),
            "backward_ms": res["adjoint"],
            "gradient_kernels_ms": round(gr_ms / n, 3), "loss_kernels_ms": round(lo_ms / n, 3),
            "cg_ms_forward_plus_adjoint": round(cg_ms / n, 3),
            "cg_iterations_forward_adjoint": list(its[-1]), "n_coefficients": 1024}


def run_extension(api, torch, args, stream):
    """Extended B-splines on the 512^2, p = 4 patch of the sweep (spline
    geometry, c = det J, 12-point B-spline hole): build of the extension
    tables, formation of E^T M E, and the L2 projection of sin(2x) cos(3y)
    with and without the extension (CG iterations, time, largest coefficient,
    relative L2 error from tw_loss)."""
    spec = synth.config2(p=4, nel=512)
    f = synth.func_sincos(2.0, 3.0)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    acc = {"build": [], "form_extended": [], "project_extended": [], "project_plain": []}
    for step in range(max(1, args.warmup) + max(1, args.steps)):
        P = api.Patch(spec)
        csr = P.form_mass("fp64")
        info, t_b = timed(P.extension)
        xcsr, t_x = timed(lambda: P.form_mass_extended(csr))
        (ue, it_e, rel_e), t_pe = timed(lambda: P.l2_project_extended(f, xcsr, tol=1e-12,
                                                                      check=False))
        (u0, it_0, rel_0), t_p0 = timed(lambda: P.l2_project(f, csr, tol=1e-12, check=False))
        if step >= max(1, args.warmup):
            for k, t in zip(acc, (t_b, t_x, t_pe, t_p0)):
                acc[k].append(t)
        if step == max(1, args.warmup) + max(1, args.steps) - 1:
            zero = torch.zeros_like(ue)
            fn2 = P.loss(zero, f)[0].item()
            err_e = (P.loss(ue, f)[0].item() / fn2) ** 0.5
            err_0 = (P.loss(u0, f)[0].item() / fn2) ** 0.5
            umax_e = torch.max(torch.abs(ue)).item()
            umax_0 = torch.max(torch.abs(u0)).item()
            n_rows, nnz = P.n_rows, P.nnz
        P.close()
    ms = {k: round(float(np.mean(v)), 3) for k, v in acc.items()}
    n_inner, n_outer, nnz_e, nnz_x = info
    return {"workload": "512x512 elements, p = 4, perturbed spline geometry (c = det J), "
                        "12-point cubic B-spline hole; f = sin(2x) cos(3y)",
            "ms": ms, "rows": n_rows, "inner": n_inner, "outer": n_outer, "nnz": nnz,
            "nnz_extended": nnz_x,
            "form_extended_nnz_per_s": round(nnz_x / (ms["form_extended"] * 1e-3), 1),
            "cg_iterations": {"extended": it_e, "plain": it_0},
            "cg_relres": {"extended": rel_e, "plain": rel_0},
            "max_abs_coefficient": {"extended": umax_e, "plain": umax_0},
            "rel_l2_error": {"extended": err_e, "plain": err_0}}


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_count": os.cpu_count(), "model": model, "machine": platform.machine()}


def oracle_sample(rows_per_patch=300, seed=0, omp=False):
    """Oracle time for the whole workload: full set-up of every patch plus a
    seeded sample of rows per patch formed in C (or_form_rows), the row time
    extrapolated to all rows.  omp=False: the single-thread oracle; omp=True:
    the same code built with OpenMP, on all host cores.  Returns (nnz/s,
    extrapolated seconds, process CPU seconds, threads, nnz)."""
    import oracle

    rng = np.random.default_rng(seed)
    t_full = 0.0
    nnz = 0
    cpu0 = time.process_time()
    for s in specs():
        t0 = time.perf_counter()
        O = oracle.Patch(s, omp=omp)
        t_setup = time.perf_counter() - t0
        rows = rng.integers(0, O.n_rows, rows_per_patch)
        t0 = time.perf_counter()
        O.form_rows(rows)
        t_rows = time.perf_counter() - t0
        t_full += t_setup + t_rows * O.n_rows / rows_per_patch
        nnz += O.nnz
    cpu = time.process_time() - cpu0
    return nnz / t_full, t_full, cpu, oracle.threads(omp), nnz


def cpu_baseline_block(rows_single=300, rows_omp=3000, seed=0):
    """The oracle on the host cores: the all-cores build as the baseline, the
    single-thread one beside it."""
    import oracle

    v1, t1, c1, _, _ = oracle_sample(rows_single, seed, omp=False)
    host = host_cpu()
    out = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "full set-up of all 12 patches + %d seeded rows per patch, time "
                     "extrapolated per row to the whole matrices (%.1f s of CPU), one thread"
                     % (rows_single, c1),
           "host": host}
    if oracle.lib(True) is not None:
        vn, tn, cn, th, _ = oracle_sample(rows_omp, seed, omp=True)
        out = {"value": vn, "unit": UNIT, "cores": th, "kind": "oracle",
               "sample": "full set-up of all 12 patches + %d seeded rows per patch, time "
                         "extrapolated per row to the whole matrices (%.1f s of CPU), the "
                         "oracle built with OpenMP (row-parallel, the same loops) on %d threads"
                         % (rows_omp, cn, th),
               "host": host,
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample": "%d seeded rows per patch" % rows_single}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default=None, help="p,nel,method: one patch of the sweep only")
    ap.add_argument("--streams", type=int, default=12,
                    help="concurrent streams (and host threads) for the step; 12 = one per patch")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-patch batched variant")
    ap.add_argument("--batched-patches", type=int, default=512)
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the density-gradient (adjoint) section")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 1024^2 precision-variant section")
    ap.add_argument("--no-extension", action="store_true",
                    help="skip the extended B-spline section")
    ap.add_argument("--no-remark1", action="store_true",
                    help="skip the comparison of the cut rows' two Gauss forms")
    args = ap.parse_args()
    if args.case:
        select_case(args.case)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    config = {"workload": workload_name() if not args.case else "single patch " + args.case,
              "patches": len(WORKLOAD), "p": [3, 4, 5],
              "elements": ["128x128", "512x512"], "methods": ["hybrid", "dwq"],
              "l2": "flushed between timed steps (256 MB write); outputs > L2",
              "streams": args.streams}

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        omp = oracle.lib(True) is not None
        rows = 1000 if omp else 100
        for _ in range(args.warmup):
            oracle_sample(rows_per_patch=rows, omp=omp)
        vals, walls, cpus = [], [], []
        nnz, th = 0, 1
        for k in range(args.steps):
            v, t, c, th, nnz = oracle_sample(rows_per_patch=rows, seed=k, omp=omp)
            vals.append(v)
            walls.append(t)
            cpus.append(c)
        value = float(np.mean(vals))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(config, nnz_per_step=int(nnz), parallelism="single"),
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                                 "sample": "full set-up of all 12 patches + %d seeded rows per "
                                           "patch, extrapolated per row%s; ms_per_step is that "
                                           "extrapolated time" % (
                                               rows, ", OpenMP build on %d threads" % th
                                               if omp else ", one thread"),
                                 "host": host_cpu()},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    r = run_ours(args, rank, world, local_rank)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline_block()
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(config, nnz_per_step=r["nnz_step"],
                                                    parallelism="replicas" if world > 1 else "single"),
                "e2e": {"value": job_rate(world, r["nnz_step"], r["e2e_ms"]), "unit": UNIT,
                        "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
                "gpu_launches": r["launches"], "clocks": r["clocks"], "roofline": r["roofline"],
                "roofline_setup": r["roofline_setup"],
                "cpu_baseline": cpu, "stage_ms_per_step_serial": r["stage_ms"],
                "stage_ms_per_step_batched": r["stage_ms_batched"],
                "precision_modes_formation_only": r["modes"],
                "batched_config4": r["batched"], "adjoint_config5": r["adjoint"],
                "precision_config3": r["precision"], "extension_config2": r["extension"],
                "remark1_config2": r["remark1"]}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
