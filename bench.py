#!/usr/bin/env python
"""Throughput of the SIPG DG operator apply on GB300 (DoFs/s).

Workload: 32^3 = 32768 hexahedra of the unit cube mapped by
x_i + 0.1 sin(pi x) sin(pi y) sin(pi z), full per-quadrature-point Jacobians
(geometry variant G3), kappa = 1 + 0.5 sin(2 pi x), Dirichlet boundary,
degree 4 (125 dofs per cell, 4,096,000 dofs), FP64 arithmetic.  One step is
one operator evaluation y = A u (cell and face integrals, one kernel launch).
Inputs (vector and geometry, > 500 MB) stay resident in HBM and exceed the
129 MB L2, so no flush is needed between steps.

The JSON line also carries the same workload in FP32, the upwind advection
operator, one fused CG iteration, the roofline of the apply kernel, the
end-to-end rate through the C ABI with host buffers, and the FP64 oracle
timed on the host cores on a bounded sample of cells.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--degree P] [--impl gb300|reference]

Under torchrun every rank runs an independent replica (the operator needs no
exchange on one GPU); rank 0 prints the line, value = all ranks' dofs / the
slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import dg_inputs  # noqa: E402

METRIC = "DoFs/s of SIPG dg_apply (FP64 vs FP32) and % HBM roofline; solves/s, p50/p99 latency"
UNIT = "DoFs/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "source": "fallback"}
# FP64 vector-ALU peak from the unit counts and clock: 152 SMs x 4 FP64 flop/clk/SM
# (2 DFMA) x 2.07 GHz = 1.26 TFLOP/s, the nominal 1.25 TFLOP/s of the part.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def even_odd_ops(k, anti):
    """Operations of one 1D kernel on a line of k values in even-odd form
    (Sec. 4.1): k - (k mod 2) sums/differences, h = k // 2 output pairs
    from (k+1)//2 even and h odd products plus their sum and difference, and
    the middle output for odd k."""
    h, h2 = k // 2, (k + 1) // 2
    return 2 * h + h * (h2 + h + 2) + ((h if anti else h2) if k % 2 else 0)


def kernel_flops_per_cell(k, op, geom, even_odd=False, folded=False):
    """Floating-point work of one cell in the apply kernels as implemented,
    counted as 2 per arithmetic instruction (an FMA, or an add or multiply
    that takes an FMA slot of the pipe): tensor-product sweeps on the cell,
    the neighbour's face-normal and in-face interpolation, the own-side face
    traces and flux at every face point, the quadrature-point operation and
    the injection of the face coefficients.  even_odd: the cell sweeps in
    even-odd form (the binary64 kernel for k >= 5).  folded: binary64
    storage with the weights folded into the stored vectors (full Jacobians:
    three instructions fewer per quadrature point; faces with per-point
    geometry: two fewer per face point and side)."""
    k2, k3, k4 = k * k, k ** 3, k ** 4
    if op == "sipg":
        if even_odd:   # 3 S + 3 S^T (centrosymmetric), 3 D + 3 D^T (anti), D^T accumulated
            sweeps = 2 * k2 * (6 * even_odd_ops(k, False) + 6 * even_odd_ops(k, True) + 3 * k)
        else:
            sweeps = 24 * k4                   # 12 sweeps (3 S, 3 D^co, 3 D^T, 3 S^T), k^4 FMA each
        nb = 6 * 2 * (k3 + 4 * k3)        # 6 faces: D_f (k^3 FMA) + 2 fields x 2 in-face sweeps
        flux = 6 * k2 * (2 * 6 * k + 20 - (4 if folded and geom != "cartesian" else 0))  # traces + flux
        qop = {"full": 39 - (6 if folded else 0), "merged": 15, "cartesian": 8}[geom] + 48  # + 24 FMA injection
        return sweeps + nb + flux + qop * k3
    if even_odd:
        sweeps = 2 * k2 * (6 * even_odd_ops(k, False) + 3 * even_odd_ops(k, True) + 3 * k)
    else:
        sweeps = 18 * k4                       # 3 S, 3 D^T, 3 S^T
    nb = 6 * 2 * (2 * k3)                  # value layer, 2 in-face sweeps
    flux = 6 * k2 * (2 * k + 8)
    qop = {"full": 24, "merged": 3, "cartesian": 3}[geom] + 3 + 12
    return sweeps + nb + flux + qop * k3


def kernel_flops_per_cell_loop(k, op, geom, even_odd=False, folded=False):
    """Floating-point work of one cell in the face-loop FP64 apply (two
    launches), counted like kernel_flops_per_cell: the forward sweeps, the
    own traces on six faces (E_s extrapolation of u and the reference
    gradient), the q-point operation; then the flux on the six faces tested
    on this cell's side, the injection of their test coefficients and the
    backward sweeps."""
    k2, k3 = k * k, k ** 3
    c, a = even_odd_ops(k, False), even_odd_ops(k, True)
    if op == "sipg":
        if even_odd:
            sweeps = 2 * k2 * (3 * c + 3 * a) + 2 * k2 * (3 * c + 3 * a + 3 * k)
        else:
            sweeps = 24 * k ** 4
        traces = (6 * 4 - 2) * k2 * 2 * k  # the x faces' value traces are end layers (no arithmetic)
        qop = {"full": 39 - (6 if folded else 0), "merged": 15, "cartesian": 8}[geom] * k3
        face = 6 * k2 * (24 - (4 if folded and geom != "cartesian" else 0))
        return sweeps + traces + qop + face + 48 * k3
    if even_odd:
        sweeps = 2 * k2 * (3 * c) + 2 * k2 * (3 * a + 3 * c + 3 * k)
    else:
        sweeps = 18 * k ** 4
    traces = (6 - 2) * k2 * 2 * k
    qop = ({"full": 24, "merged": 3, "cartesian": 3}[geom] + 3) * k3
    return sweeps + traces + qop + 6 * k2 * 8 + 12 * k3


def eo_flops(k, anti):
    """Flops of one 1D kernel on a line of k values in even-odd form (Sec.
    4.1), each addition, subtraction or multiplication 1 and each FMA 2: the
    k - (k mod 2) input sums and differences, per output pair an even and an
    odd dot product (first term a multiplication) and their sum and
    difference, and the middle output for odd k."""
    h, h2 = k // 2, (k + 1) // 2
    mid = (2 * h - 1 if anti else 2 * h2 - 1) if k % 2 else 0
    return 2 * h + 2 * k * h + mid


def algorithmic_flops_per_cell_loop(k, op, geom, even_odd, folded, boundary_fraction=0.0):
    """Flops of one cell in the face-loop apply counted as the paper does
    (Sec. 4.1: each FMA 2, each other addition or multiplication 1; the
    first term of a dot product is a multiplication): the forward S and D^co
    sweeps, the own traces (E_s extrapolation, 4 fields for SIPG) on six
    faces, the q-point operation; the flux on six faces tested on this side
    (boundary_fraction of the face sides on the domain boundary take the
    boundary flux), the injection of the face test coefficients, the
    D^co^T sweeps accumulated into the value field and the S^T sweeps."""
    k2, k3 = k * k, k ** 3
    direct = k * (2 * k - 1)                       # one line, direct form
    s_line = eo_flops(k, False) if even_odd else direct
    d_line = eo_flops(k, True) if even_odd else direct
    bf = boundary_fraction
    if op == "sipg":
        fwd = 3 * k2 * s_line + 3 * k2 * d_line
        traces = (6 * 4 - 2) * k2 * (2 * k - 1)  # x faces' value traces: end layers
        qop = {"full": 30 if folded else 33, "merged": 15, "cartesian": 13}[geom] * k3
        flux_int = {"cartesian": 18}.get(geom, 19)
        flux_bdy = {"cartesian": 12}.get(geom, 11)
        flux = 6 * k2 * ((1 - bf) * flux_int + bf * flux_bdy)
        inject = (4 * 11 + 3) * k3
        bwd = 3 * k2 * (d_line + k) + 3 * k2 * s_line
        return fwd + traces + qop + flux + inject + bwd
    fwd = 3 * k2 * s_line
    traces = (6 - 2) * k2 * (2 * k - 1)
    qop = {"full": 21, "merged": 3, "cartesian": 12}[geom] * k3
    flux = 6 * k2 * ((1 - bf) * 7 + bf * 1)
    inject = 11 * k3
    bwd = 3 * k2 * (d_line + k) + 3 * k2 * s_line
    return fwd + traces + qop + flux + inject + bwd


def bytes_per_dof(k, s, op, geom):
    """Algorithmic bytes per dof of one apply: src read and dst write, the
    cell geometry per point, the face geometry per face point (3 faces per
    cell, k^2 points each) and the penalty per face.  SIPG cell arrays with
    full Jacobians: sqrt(kappa JxW) J^{-1} (9 values) in binary64, J^{-1} and
    kappa JxW (10) in binary32; G2: the position and kappa (4 values).  SIPG face arrays: both sides' J^{-T} n and
    kappa da w (7 values) in binary64; in binary32 one J^{-T} e_d (the two
    sides' vectors differ only in sign) and kappa da w (4 values)."""
    vec = 2 * s
    if geom == "cartesian":
        return vec
    cell = {("sipg", "full"): 9 if s == 8 else 10, ("advection", "full"): 10, ("sipg", "merged"): 6,
            ("advection", "merged"): 3, ("sipg", "positions"): 4, ("advection", "positions"): 3}[(op, geom)] * s
    nfa = (4 if s == 4 else 7) if op == "sipg" else 1
    face = nfa * s * 3 / k + (3 * s / k ** 3 if op == "sipg" else 0)
    return vec + cell + face


# DRAM traffic per apply (ncu dram__bytes_read.sum + dram__bytes_write.sum,
# one capture each, all launches of the apply) of the 32^3 deformed p = 4 G3
# SIPG workload, keyed by (arithmetic, face mode, degree, cells per block);
# reported only for exactly that launch configuration, and to be re-taken
# whenever the kernel changes.
MEASURED_TRAFFIC = {
    ("fp64", "loop", 4, 5): 962.1e6,
    ("fp32", "element", 4, 8): 232.4e6,
}


# FP64-pipe warp instructions per apply (ncu sass__inst_executed_per_opcode:
# DFMA + DADD + DMUL of both launches) of the same workload and launch
# configuration; to be re-taken whenever the kernels change.
MEASURED_FP64_WARP_INSTR = {
    ("fp64", "loop", 4, 5): 17.904845e6,
}


def measured_traffic(prec, face_mode, degree, cpb, workload):
    if workload != "deformed_dirichlet_32^3_p%d" % degree:
        return None
    return MEASURED_TRAFFIC.get((prec, face_mode, degree, cpb))


def probe_alu_peaks(dgp):
    """FP64 and FP32 FMA throughput measured on this GPU by the library's
    FMA-chain kernel (dg_peak_probe); the derived unit-count figures are the
    fallback if the probe fails."""
    out = {}
    for key, kind, derived in (("fp64_tflops", 0, FP64_PEAK_TFLOPS), ("fp32_tflops", 1, FP32_PEAK_TFLOPS)):
        try:
            out[key] = dgp.dg_peak_probe(kind)
            out[key + "_source"] = "measured in this run: dg_peak_probe(%d), FMA chains, best of 4 launches" % kind
        except Exception as e:  # noqa: BLE001
            out[key] = derived
            out[key + "_source"] = "derived from unit counts and the 2.07 GHz clock (probe failed: %s)" % e
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        d["source"] = "measured"
        return d
    except Exception:
        return dict(PEAKS_FALLBACK)


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms in the background."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        return rows


def summarize_clocks(rows, t0, t1):
    import datetime
    sel = []
    for r in rows if isinstance(rows, list) else []:
        try:
            ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except Exception:
            continue
        if t0 - 0.05 <= ts <= t1 + 0.05:
            sel.append(r)
    if not sel:
        sel = rows[-3:] if isinstance(rows, list) else []
    if not sel:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    sm = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
    mx = [float(r[3]) for r in sel if r[3].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in sel for i in range(4) if r[6 + i].lower() == "active"})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(sel),
            "power_w_max": max(float(r[4]) for r in sel if r[4].replace(".", "").isdigit()) if sel else None}


def aggregate_ranks(torch, dist, total_ms, steps, units_per_step, world, device):
    """Whole-job throughput over independent replicas: the slowest rank's
    time (all-reduce MAX) and all ranks' units over it.  Returns
    (max total ms, units per second)."""
    t_max = total_ms
    if dist is not None and world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * units_per_step * steps / (t_max / 1e3)


def time_applies(torch, op, src, dst, steps, per_launch=False):
    """Device time of `steps` back-to-back applies on the operator's stream
    (CUDA events around the whole region), and the average duration of one
    apply: total / steps, or (per_launch) the mean of per-apply event pairs,
    which add a few microseconds of event overhead to the region."""
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for i in range(steps):
        if per_launch:
            evs[i][0].record(stream)
        op.apply(src, dst)
        if per_launch:
            evs[i][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    total_ms = start.elapsed_time(end)
    launch_ms = float(np.mean([a.elapsed_time(b) for a, b in evs])) if per_launch else total_ms / steps
    return total_ms, launch_ms


def solve_metrics(torch, dgp, args, n=16, p=3, rtol=1e-10, repeats=20):
    """Poisson -div(kappa grad u) = f (manufactured u = sin sin sin, Dirichlet)
    on the n^3 sine-deformed mesh, degree p, G3 geometry: time to a relative
    residual of rtol with plain FP64 CG and with the mixed-precision solver
    (binary32 CG with residual replacement by the FP64 residual), then the
    latency distribution of repeated mixed solves from a zero initial guess."""
    kw = dict(geom="full", periodic=False, mapping=1, amplitude=0.1, coeff=1)
    o64 = dgp.Operator(n, p, prec="fp64", **kw)
    o64.set_face_mode(args.face_mode)
    o32 = dgp.Operator(n, p, prec="fp32", **kw)
    rhs = o64.rhs(1)
    torch.cuda.synchronize()
    x = torch.zeros_like(rhs)
    o64.cg(rhs, x, rtol=1e-2, max_it=50, raise_on_error=False)  # warm-up
    x.zero_()
    t = time.perf_counter()
    _, it64, rr64, st64 = o64.cg(rhs, x, rtol=rtol, max_it=50000, raise_on_error=False)
    t64 = time.perf_counter() - t
    lat = []
    outer = inner = 0
    rrm = None
    for i in range(repeats + 1):
        x.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, outer, inner, rrm = dgp.dg_cg_solve_mixed(o64.handle, o32.handle, rhs.data_ptr(), x.data_ptr(), rtol,
                                                      raise_on_error=False)
        if i:
            lat.append(time.perf_counter() - t)
    o64.close()
    o32.close()
    lat = np.array(lat)
    return {"workload": "deformed_dirichlet_%d^3_p%d manufactured Poisson, kappa variable, G3" % (n, p),
            "dofs": n ** 3 * (p + 1) ** 3, "rtol": rtol,
            "fp64_cg": {"seconds": t64, "iterations": it64, "rel_residual": rr64, "status": st64},
            "mixed": {"seconds_p50": float(np.median(lat)), "outer": outer, "inner_fp32_iterations": inner,
                      "rel_residual": rrm},
            "speedup_mixed_vs_fp64": t64 / float(np.median(lat)),
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
                           "samples": len(lat)},
            "solves_per_s": 1.0 / float(np.mean(lat))}


def batch_metrics(torch, dgp, args, count=64, prec_list=("fp64", "fp32"), budget_gb=120.0, seed=4, n_lo=8,
                  n_hi=48):
    """Many independent operators in one graph launch: count deformed-cube
    meshes with n^3 cells, n log-uniform in [n_lo, n_hi], degrees uniform in
    1..7 (G3 geometry, kappa variable, Dirichlet).  Compares one
    dg_batch_launch (fused launches per kernel group, per-group autotuned
    tile shapes, 8 graph branches) with the same applies issued one by one on
    a stream, each operator at its own autotuned tile shape; FP64 operators
    in the bench's face mode.  Meshes beyond the device-memory budget are
    dropped (their count is reported)."""
    rng = np.random.default_rng(seed)
    ns = np.round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count))).astype(int)
    ps = rng.integers(1, 8, count)
    out = {"workload": "%d meshes, n^3 cells with n log-uniform in [%d, %d], degree uniform in 1..7, G3" % (
        count, n_lo, n_hi)}
    for prec in prec_list:
        s = 4 if prec == "fp32" else 8
        ops, srcs, dsts, used = [], [], [], 0.0
        skipped = 0
        for n, p in zip(ns, ps):
            k = int(p) + 1
            dofs = int(n) ** 3 * k ** 3
            loop = prec == "fp64" and args.face_mode == "loop"
            work = (24.0 / k + 3.0) * 8 if loop else 0.0  # face-loop traces and gradient-test fields
            need = dofs * (bytes_per_dof(k, s, "sipg", "full") + 2 * s + work) / 1e9
            if used + need > budget_gb:
                skipped += 1
                continue
            used += need
            op = dgp.Operator(int(n), int(p), geom="full", prec=prec, mapping=1, amplitude=0.1, coeff=1)
            if loop:
                op.set_face_mode("loop")
            ops.append(op)
            srcs.append(torch.tensor(dg_inputs.src_vector(op.n_dofs, int(n) * 31 + int(p)), dtype=op.dtype,
                                     device="cuda"))
            dsts.append(torch.empty_like(srcs[-1]))
        total = sum(o.n_dofs for o in ops)
        # the one-by-one reference: each operator at its own autotuned tile shape
        for o in ops:
            o.autotune()
        stream = torch.cuda.current_stream()
        for _ in range(2):
            for o, x, y in zip(ops, srcs, dsts):
                o.apply(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            for o, x, y in zip(ops, srcs, dsts):
                o.apply(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        t_seq = e0.elapsed_time(e1) / reps
        b = dgp.dg_batch_create([o.handle for o in ops], [x.data_ptr() for x in srcs], [x.data_ptr() for x in dsts],
                                autotune=True, branches=8, stream=torch.cuda.current_stream().cuda_stream)
        groups, launches = dgp.dg_batch_info(b)
        for _ in range(3):
            dgp.dg_batch_launch(b)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            dgp.dg_batch_launch(b)
        e1.record(stream)
        torch.cuda.synchronize()
        t_batch = e0.elapsed_time(e1) / reps
        dgp.dg_batch_destroy(b)
        out[prec] = {"operators": len(ops), "skipped_for_memory": skipped, "dofs": total,
                     "kernel_groups": groups, "launches_per_batch": launches,
                     "launches_sequential": len(ops) * (2 if prec == "fp64" and args.face_mode == "loop" else 1),
                     "face_mode": "loop" if prec == "fp64" and args.face_mode == "loop" else "element",
                     "ms_per_batch_launch": t_batch, "dofs_per_s": total / (t_batch / 1e3),
                     "ms_sequential_applies": t_seq, "speedup_vs_sequential": t_seq / t_batch,
                     "cells_per_block_by_degree": {
                         str(d): sorted({o.info()["cells_per_block"] for o in ops if o.degree == d})
                         for d in sorted({o.degree for o in ops})}}
        for o in ops:
            o.close()
        del srcs, dsts
        torch.cuda.empty_cache()
    return out


def serve_requests(dgp, count, seed, dof_lo=1e4, dof_hi=2e7, rtol=1e-8):
    """Request mix: dofs lognormal over [dof_lo, dof_hi] (the interval is
    +-2 standard deviations, clipped), degree uniform in 2..6, every other
    request on a Cartesian mesh (kappa = 1) and the others on the sine-mapped
    mesh with G3 geometry and kappa = 1 + 0.5 sin(2 pi x)."""
    rng = np.random.default_rng(seed)
    mu, sig = 0.5 * (np.log(dof_lo) + np.log(dof_hi)), (np.log(dof_hi) - np.log(dof_lo)) / 4
    reqs = []
    for i in range(count):
        dofs = float(np.clip(np.exp(rng.normal(mu, sig)), dof_lo, dof_hi))
        p = int(rng.integers(2, 7))
        n = max(2, int(round((dofs / (p + 1) ** 3) ** (1.0 / 3.0))))
        reqs.append(dgp.make_request(n, p, mapping=i % 2, rtol=rtol))
    return reqs


def serve_metrics(dgp, count=48, seed=5, dof_hi=2e6, budget_gb=120, slots=8, rates=(0.5, 0.9), progress=None,
                  policies=(0,), max_age_s=2.0):
    """Continuous-batching solve server under Poisson arrivals: first all
    requests at once (capacity in solves/s, FIFO), then Poisson arrivals at
    given fractions of that capacity, for each admission policy (0 FIFO, 1
    shortest job first with aging max_age_s); p50/p99 latency (submit to
    done) per rate.  progress: optional callable given the partial result
    after each run."""
    budget = int(budget_gb * (1 << 30))
    reqs = serve_requests(dgp, count, seed, dof_hi=dof_hi)
    out = {"requests": count, "slots": slots, "budget_gb": budget_gb,
           "mix": "dofs lognormal over [1e4, %.0e], degree 2..6, half Cartesian / half deformed G3, "
                  "mixed-precision CG to 1e-8" % dof_hi,
           "total_dofs": int(sum(dgp.dg_request_device_bytes(r) * 0 + r.n[0] * r.n[1] * r.n[2] *
                                 (r.degree + 1) ** 3 for r in reqs))}
    res = dgp.serve_arrivals(reqs, [0.0] * count, budget, slots)
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    cap = count / span
    out["saturated"] = {"solves_per_s": cap, "seconds": span,
                        "all_converged": all(r["status"] == 0 and r["rel_res"] <= 1e-8 for r in res),
                        "p50_latency_ms": 1e3 * float(np.percentile([r["t_done"] - r["t_submit"] for r in res], 50))}
    if progress:
        progress(out)
    rng = np.random.default_rng(seed + 1)
    for frac in rates:
        lam = frac * cap
        arrivals = np.cumsum(rng.exponential(1.0 / lam, count))
        arrivals -= arrivals[0]
        for pol in policies:
            res = dgp.serve_arrivals(reqs, list(arrivals), budget, slots, policy=pol, max_age_s=max_age_s)
            lat = np.array([r["t_done"] - r["t_submit"] for r in res])
            svc = np.array([r["t_done"] - r["t_admit"] for r in res])  # service time (admitted to done)
            span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
            key = "rate_%.2f_of_capacity" % frac + ("" if pol == 0 else "_sjf")
            out[key] = {
                "arrival_rate_per_s": lam, "policy": "fifo" if pol == 0 else "sjf, aging %.1f s" % max_age_s,
                "p50_latency_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_latency_ms": 1e3 * float(np.percentile(lat, 99)),
                "p50_service_ms": 1e3 * float(np.percentile(svc, 50)),
                "p99_service_ms": 1e3 * float(np.percentile(svc, 99)),
                "p99_queueing_ms": 1e3 * float(np.percentile(lat - svc, 99)), "solves_per_s": count / span,
                "all_converged": all(r["status"] == 0 and r["rel_res"] <= 1e-8 for r in res)}
            if progress:
                progress(out)
    return out


def serve_slot_study(dgp, count=48, seed=5, dof_hi=2e6, budget_gb=120, frac=0.5, slot_list=(2, 4, 8, 16),
                     max_age_s=2.0):
    """p50/p99 latency against the slot count and the admission policy at one
    arrival rate (frac of the 8-slot FIFO capacity): the same request mix and
    arrival times for every run."""
    budget = int(budget_gb * (1 << 30))
    reqs = serve_requests(dgp, count, seed, dof_hi=dof_hi)
    res = dgp.serve_arrivals(reqs, [0.0] * count, budget, 8)
    cap = count / (max(r["t_done"] for r in res) - min(r["t_submit"] for r in res))
    rng = np.random.default_rng(seed + 7)
    arrivals = np.cumsum(rng.exponential(1.0 / (frac * cap), count))
    arrivals -= arrivals[0]
    rows = []
    for slots in slot_list:
        for pol in (0, 1):
            res = dgp.serve_arrivals(reqs, list(arrivals), budget, slots, policy=pol, max_age_s=max_age_s)
            lat = np.array([r["t_done"] - r["t_submit"] for r in res])
            rows.append({"slots": slots, "policy": "fifo" if pol == 0 else "sjf",
                         "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 2),
                         "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 2),
                         "all_converged": all(r["status"] == 0 for r in res)})
    return {"requests": count, "arrival_rate_per_s": frac * cap, "capacity_8_slots_per_s": cap,
            "aging_s": max_age_s, "rows": rows}


CONFIG3_CASES = (("cartesian_64^3_p3", 64, 3, 0), ("cartesian_64^3_p5", 64, 5, 0), ("deformed_48^3_p3", 48, 3, 1),
                 ("deformed_48^3_p5", 48, 5, 1))


def config3_metrics(torch, dgp, rtol=1e-10, cases=CONFIG3_CASES, face_mode="loop", emulated=True, emu_rtol=1e-9,
                    progress=None):
    """Mixed precision at full size: manufactured Poisson problems (64^3
    Cartesian and 48^3 deformed cells, degrees 3 and 5) solved to rtol by
    plain FP64 CG and by the mixed solver (binary32 CG with residual
    replacement by the FP64 residual; the FP64 operator in the given face
    mode); optionally also with the emulated-FP64 outer residual, to emu_rtol
    (double-float residuals floor near 2e-10 relative at p = 5, so that
    variant is run to 1e-9).  Wall time, iterations, L2 errors against the
    exact solution and the difference between the mixed and the FP64
    solutions."""
    out = {}
    for name, n, p, mapping in cases:
        kw = dict(geom="full" if mapping else "cartesian", mapping=mapping, amplitude=0.1, coeff=mapping)
        o64 = dgp.Operator(n, p, prec="fp64", **kw)
        o64.set_face_mode(face_mode)
        o32 = dgp.Operator(n, p, prec="fp32", **kw)
        oe = dgp.Operator(n, p, prec="fp64emu", **kw)
        oe.set_face_mode(face_mode)
        rhs = o64.rhs(mapping)
        res = {"dofs": o64.n_dofs, "rtol": rtol}
        x64 = torch.zeros_like(rhs)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, it, rr, st = o64.cg(rhs, x64, rtol=rtol, max_it=200000, raise_on_error=False)
        res["fp64_cg"] = {"seconds": time.perf_counter() - t, "iterations": it, "rel_res": rr, "status": st,
                          "l2_error": o64.l2_error(x64)}
        # the mixed solver with the inner arithmetic chosen by measurement (the
        # headline), each inner arithmetic forced, and (optionally) the
        # emulated-FP64 outer residual with a binary32 inner recursion
        variants = [("mixed_auto", o64, None, rtol), ("mixed_fp32_inner", o64, o32, rtol),
                    ("mixed_emulated_inner", o64, oe, rtol)]
        if emulated:
            variants.append(("mixed_emulated_fp64_outer", oe, o32, emu_rtol))
        for label, oh, ol, rt in variants:
            xm = torch.zeros_like(rhs)
            torch.cuda.synchronize()
            t = time.perf_counter()
            kind = None
            if ol is None:
                st, outer, inner, rr, kind = dgp.dg_cg_solve_mixed_auto(
                    oh.handle, oe.handle, o32.handle, rhs.data_ptr(), xm.data_ptr(), rt, max_outer=60,
                    inner_rtol=1e-2, max_inner=20000, raise_on_error=False)
            else:
                st, outer, inner, rr = dgp.dg_cg_solve_mixed(oh.handle, ol.handle, rhs.data_ptr(), xm.data_ptr(), rt,
                                                             max_outer=60, inner_rtol=1e-2, max_inner=20000,
                                                             raise_on_error=False)
            secs = time.perf_counter() - t
            res[label] = {"seconds": secs, "rtol": rt, "outer": outer, "inner_iterations": inner, "rel_res": rr,
                          "inner_arithmetic": kind or ("fp32" if ol is o32 else "fp64emu"),
                          "status": st, "l2_error": o64.l2_error(xm),
                          "rel_diff_to_fp64_solution": float((xm - x64).norm() / x64.norm()),
                          "speedup_vs_fp64_cg": res["fp64_cg"]["seconds"] / secs}
        out[name] = res
        if progress:
            progress(name, res)
        for o in (o64, o32, oe):
            if o is not None:
                o.close()
        torch.cuda.empty_cache()
    return out


def degree_sweep_metrics(torch, dgp, steps=30):
    """Apply throughput for p = 1..8 in FP64 and FP32 on the 32^3 mesh and on
    the paper's larger-than-cache size schedule (128^3 for p = 1-2, 64^3 for
    p = 3-5, 32^3 for p = 6-8), Cartesian, G3 (deformed, full Jacobians) and
    G4 (deformed, merged coefficients); FP64 element-centric and face loop;
    DoFs/s from the mean per-apply CUDA event time after warm-up, and the HBM
    fraction of the algorithmic bytes."""
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    rows = []
    for p in range(1, 9):
        for sched, n in (("32^3", 32), ("paper", dg_inputs.paper_size_schedule(p))):
            if sched == "paper" and n == 32:
                continue
            for geom, mapping in (("cartesian", 0), ("full", 1), ("merged", 1)):
                for prec in ("fp64", "fp64-loop", "fp32"):
                    o = dgp.Operator(n, p, geom=geom, prec=prec[:4], mapping=mapping, amplitude=0.1, coeff=1)
                    if prec == "fp64-loop":
                        o.set_face_mode("loop")
                    src = torch.tensor(dg_inputs.src_vector(o.n_dofs, 3), dtype=o.dtype, device="cuda")
                    dst = torch.empty_like(src)
                    for _ in range(3):
                        o.apply(src, dst)
                    _, ms = time_applies(torch, o, src, dst, steps)
                    s = 4 if prec == "fp32" else 8
                    bpd = bytes_per_dof(p + 1, s, "sipg", geom)
                    rows.append({"p": p, "mesh": "%d^3" % n, "schedule": sched, "geometry": geom, "prec": prec,
                                 "dofs": o.n_dofs, "us": round(ms * 1e3, 2),
                                 "gdofs_per_s": round(o.n_dofs / (ms / 1e3) / 1e9, 3),
                                 "hbm_frac": round(bpd * o.n_dofs / (ms / 1e3) / 1e9 / hbm, 4)})
                    o.close()
                    del src, dst
                    torch.cuda.empty_cache()
    return {"operator": "SIPG, kappa = 1 + 0.5 sin(2 pi x), Dirichlet", "hbm_peak_gbs": hbm, "rows": rows}


def fp32_degree_sweep(torch, dgp, steps=20, degrees=(2, 3, 4, 5, 6)):
    """The binary32 G3 SIPG apply (sine-deformed mesh, kappa variable,
    Dirichlet) for p = 2..6 on the paper's larger-than-cache size schedule
    (128^3 for p <= 2, 64^3 for p = 3-5, 32^3 for p >= 6): DoFs/s from the
    mean per-apply CUDA-event time, GB/s of the algorithmic bytes and the
    fraction of the measured HBM bandwidth."""
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    rows = []
    for p in degrees:
        n = dg_inputs.paper_size_schedule(p)
        o = dgp.Operator(n, p, geom="full", prec="fp32", mapping=1, amplitude=0.1, coeff=1)
        src = torch.tensor(dg_inputs.src_vector(o.n_dofs, 3), dtype=o.dtype, device="cuda")
        dst = torch.empty_like(src)
        for _ in range(3):
            o.apply(src, dst)
        _, ms = time_applies(torch, o, src, dst, steps)
        bpd = bytes_per_dof(p + 1, 4, "sipg", "full")
        gbs = bpd * o.n_dofs / (ms / 1e3) / 1e9
        rows.append({"p": p, "mesh": "%d^3" % n, "dofs": o.n_dofs, "us": round(ms * 1e3, 2),
                     "gdofs_per_s": round(o.n_dofs / (ms / 1e3) / 1e9, 3), "bytes_per_dof": round(bpd, 2),
                     "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                     # the same time against a byte count that moves both
                     # sides' face vectors (7 values per face point, not 4)
                     "hbm_frac_two_sided_face_bytes":
                         round((8 + 40 + 84 / (p + 1)) * o.n_dofs / (ms / 1e3) / 1e9 / hbm, 4)})
        o.close()
        del src, dst
        torch.cuda.empty_cache()
    return {"operator": "SIPG G3, kappa = 1 + 0.5 sin(2 pi x), Dirichlet, FP32", "hbm_peak_gbs": hbm, "rows": rows}


def cpu_baseline(workload, form, target_s=12.0):
    """The FP64 oracle (cell-by-cell brute-force quadrature, OpenMP on the
    host cores) on a seeded sample of cells of the same workload; DoFs/s =
    sampled dofs / time."""
    import oracle
    mesh, p = workload["mesh"], workload["degree"]
    n = oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=1)
    nc = oracle.n_cells(mesh)
    batch = 64
    done, t_used, seed = 0, 0.0, 0
    while t_used < target_s and done < nc:
        cells = dg_inputs.sample_cells(nc, batch, seed=1000 + seed)
        t = time.perf_counter()
        oracle.apply(mesh, p, form, u, cells=cells)
        t_used += time.perf_counter() - t
        done += len(cells)
        seed += 1
        batch = min(batch * 2, 4096)
    k3 = (p + 1) ** 3
    return {"value": done * k3 / t_used, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d sampled cells (%d dofs) of the same workload, %.1f s" % (done, done * k3, t_used)}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle as it stands, on the host cores,
    each step a bounded sample of cells of the same workload."""
    if rank != 0:
        return
    import oracle
    oracle.lib()
    wname = "deformed_dirichlet_32^3_p%d" % args.degree
    w = dg_inputs.workload(wname)
    mesh, p = w["mesh"], w["degree"]
    form = dict(op="sipg", coeff=w["coeff"])
    n = oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=1)
    nc = oracle.n_cells(mesh)
    per_step = max(16, int(256 * (5.0 / (p + 1)) ** 6))
    times = []
    for i in range(args.warmup + args.steps):
        cells = dg_inputs.sample_cells(nc, per_step, seed=5000 + i)
        t = time.perf_counter()
        oracle.apply(mesh, p, form, u, cells=cells)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
    k3 = (p + 1) ** 3
    total = sum(times)
    value = args.steps * per_step * k3 / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wname, "degree": p, "cells": nc, "dofs": n,
                                            "sample_cells_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d seeded cells per step (%d dofs)" % (per_step, per_step * k3)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "fp64emu"],
                    help="precision of the headline apply")
    ap.add_argument("--cells-per-block", type=int, default=0,
                    help="tile shape of the headline operator (0: the operator's default)")
    ap.add_argument("--face-mode", default="loop", choices=["loop", "element"],
                    help="FP64 / emulated-FP64 face evaluation: face loop (neighbour traces read, not recomputed; "
                         "faster on GB300) or element-centric")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--solve-config3", action="store_true",
                    help="only run the full-size mixed-precision solves and print their JSON")
    ap.add_argument("--degree-sweep", action="store_true",
                    help="only run the apply degree sweep (32^3 and the paper's size schedule) and print its JSON")
    ap.add_argument("--serve-config5", action="store_true",
                    help="only run the full serving stream (2000 requests, 1e4..2e7 dofs, swept arrival rates)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1711_03590_gb300 as dgp
    dgp.build()
    dgp.load_library()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    if args.serve_config5:
        # the full stream: 2000 requests, 1e4..2e7 dofs (mean about 2.7e6),
        # saturated, then at 90% of that capacity under FIFO and under
        # shortest-job-first admission; each run prints when done
        if rank == 0:
            serve_metrics(dgp, count=2000, seed=11, dof_hi=2e7, rates=(0.9,), policies=(0, 1), max_age_s=5.0,
                          progress=lambda r: print(json.dumps({"serve_config5": r}), flush=True))
        return
    if args.degree_sweep:
        if rank == 0:
            print(json.dumps({"degree_sweep": degree_sweep_metrics(torch, dgp)}), flush=True)
        return
    if args.solve_config3:
        if rank == 0:
            print(json.dumps({"solve_config3": config3_metrics(
                torch, dgp, face_mode=args.face_mode,
                progress=lambda nm, r: print(json.dumps({"case": nm, "result": r}), flush=True))}), flush=True)
        return

    wname = "deformed_dirichlet_32^3_p%d" % args.degree
    w = dg_inputs.workload(wname)
    mesh, p = w["mesh"], w["degree"]
    k = p + 1
    common = dict(periodic=mesh["periodic"], mapping=mesh["mapping"], amplitude=mesh["amplitude"])
    peaks = load_peaks()
    alu = probe_alu_peaks(dgp)

    op = dgp.Operator(mesh["n"], p, geom=w["geom"], op="sipg", prec=args.prec, coeff=w["coeff"], **common)
    loop = args.prec in ("fp64", "fp64emu") and args.face_mode == "loop"
    if loop:
        op.set_face_mode("loop")
    if args.cells_per_block:
        op.set_cells_per_block(args.cells_per_block)
    cpb_used = op.info()["cells_per_block"]
    n = op.n_dofs
    n_cells = op.info()["n_cells"]
    ssz = 4 if args.prec == "fp32" else 8
    src = torch.tensor(dg_inputs.src_vector(n, seed=1 + rank), dtype=op.dtype, device="cuda")
    dst = torch.empty_like(src)
    for _ in range(args.warmup):
        op.apply(src, dst)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local_rank)
    sampler.start()
    t0 = time.time()
    total_ms, launch_ms = time_applies(torch, op, src, dst, args.steps)
    t1 = time.time()
    if dist:
        dist.barrier()
    rows = sampler.stop()
    clocks = summarize_clocks(rows, t0, t1)
    torch.cuda.synchronize()
    t_max, value = aggregate_ranks(torch, dist, total_ms, args.steps, n, world, "cuda")
    ms_per_step = t_max / args.steps

    # roofline of the apply (one kernel; the face loop: its two launches)
    if loop:
        flops = kernel_flops_per_cell_loop(k, "sipg", w["geom"], even_odd=(args.prec == "fp64" and k >= 5),
                                           folded=args.prec != "fp32") * n_cells
    else:
        flops = kernel_flops_per_cell(k, "sipg", w["geom"], even_odd=(args.prec == "fp64" and k >= 5),
                                      folded=args.prec != "fp32") * n_cells
    achieved_tf = flops / (launch_ms / 1e3) / 1e12
    nx = mesh["n"]
    bfrac = 0.0 if mesh["periodic"] else 2.0 * (nx[0] * nx[1] + nx[1] * nx[2] + nx[0] * nx[2]) / (6.0 * n_cells)
    flops_alg = (algorithmic_flops_per_cell_loop(k, "sipg", w["geom"], even_odd=(args.prec == "fp64" and k >= 5),
                                                 folded=args.prec != "fp32", boundary_fraction=bfrac) * n_cells
                 if loop else None)
    bpd = bytes_per_dof(k, ssz, "sipg", w["geom"])
    achieved_gbs = bpd * n / (launch_ms / 1e3) / 1e9
    if args.prec == "fp32":
        kname = "apply_f32_kernel<%d,%d,FULL,SIPG>" % (k, op.info()["cells_per_block"])
    elif loop:
        kname = ("face-loop apply <%d,%s,FULL,SIPG>: split_cell_forward + split_cell_backward "
                 "(the roofline is per apply)" % (k, {"fp64": "double", "fp64emu": "df64"}[args.prec]))
    else:
        kname = "apply_kernel<%d,%s,FULL,SIPG>" % (k, {"fp64": "double", "fp64emu": "df64"}[args.prec])
    traffic = measured_traffic(args.prec, "loop" if loop else "element", p, op.info()["cells_per_block"], wname)
    tsrc = ("ncu capture of this launch configuration: dram__bytes_read.sum + dram__bytes_write.sum per apply"
            if traffic else None)
    hbm = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": achieved_gbs / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": tsrc, "kernel": kname,
           "bytes_per_dof": bpd, "algorithmic_bytes_per_launch": bpd * n, "peak_source": peaks.get("source")}
    if args.prec == "fp64":
        # achieved: the algorithmic flops (the paper's counting method) per
        # apply over its time; issue_slots: the kernels' own operation count
        # with every FP64 instruction charged as an FMA; fp64_pipe: the FP64
        # warp instructions ncu counted for this configuration against the
        # measured FMA rate (how full the FP64 pipe is)
        issue = {"flops_per_launch": flops, "achieved": achieved_tf, "frac": achieved_tf / alu["fp64_tflops"],
                 "counting": "2 per FP64 arithmetic instruction of the kernels' operation count"}
        winstr = MEASURED_FP64_WARP_INSTR.get((args.prec, "loop" if loop else "element", p,
                                               op.info()["cells_per_block"])) if wname == \
            "deformed_dirichlet_32^3_p%d" % p else None
        pipe = None if winstr is None else {
            "warp_instructions_per_launch": winstr,
            "frac": winstr * 32 * 2 / (launch_ms / 1e3) / 1e12 / alu["fp64_tflops"],
            "source": "ncu sass__inst_executed_per_opcode (DFMA + DADD + DMUL) of this launch configuration"}
        if flops_alg is not None:
            ach = flops_alg / (launch_ms / 1e3) / 1e12
            top = {"achieved": ach, "frac": ach / alu["fp64_tflops"], "flops_per_launch": flops_alg,
                   "flops_counting": "paper's method (Sec. 4.1): FMA 2, other add/mul 1, even-odd sweeps"}
        else:
            top = {"achieved": achieved_tf, "frac": achieved_tf / alu["fp64_tflops"], "flops_per_launch": flops,
                   "flops_counting": issue["counting"]}
        roofline = {"bound": "alu", "achieved": top["achieved"], "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                    "frac": top["frac"], "traffic": traffic, "traffic_source": tsrc,
                    "kernel": kname,
                    "flops_per_launch": top["flops_per_launch"],
                    "flops_counting": top["flops_counting"],
                    "issue_slots": issue,
                    "fp64_pipe": pipe,
                    "peak_source": alu["fp64_tflops_source"],
                    "peak_derived": FP64_PEAK_TFLOPS,
                    "hbm": hbm}
    else:
        roofline = dict(hbm, alu_tflops=achieved_tf, alu_peak_tflops=alu["fp32_tflops"])

    # end to end through the C ABI with pinned host buffers
    hsrc = torch.tensor(dg_inputs.src_vector(n, seed=1 + rank), dtype=op.dtype).pin_memory()
    hdst = torch.empty_like(hsrc).pin_memory()
    for _ in range(2):
        op.apply_host(hsrc, hdst)
    e2e_steps = max(3, min(args.steps, 50))
    te = time.perf_counter()
    for _ in range(e2e_steps):
        op.apply_host(hsrc, hdst)
    te = time.perf_counter() - te
    e2e = {"value": n / (te / e2e_steps), "unit": UNIT, "h2d_bytes_per_step": n * ssz, "d2h_bytes_per_step": n * ssz,
           "call": "dg_apply_host", "face_mode": "loop" if loop else "element"}
    op.close()

    fp64_element = None
    if loop and args.prec == "fp64":
        # the element-centric FP64 apply of the same workload: kernel-only,
        # and end to end; e2e reports the faster of the two public paths
        ope_ = dgp.Operator(mesh["n"], p, geom=w["geom"], op="sipg", prec="fp64", coeff=w["coeff"], **common)
        for _ in range(args.warmup):
            ope_.apply(src, dst)
        tot_el, _ = time_applies(torch, ope_, src, dst, args.steps)
        for _ in range(2):
            ope_.apply_host(hsrc, hdst)
        te2 = time.perf_counter()
        for _ in range(e2e_steps):
            ope_.apply_host(hsrc, hdst)
        te2 = time.perf_counter() - te2
        ope_.close()
        fp64_element = {"value": n / (tot_el / args.steps / 1e3), "unit": UNIT, "ms_per_step": tot_el / args.steps,
                        "e2e": n / (te2 / e2e_steps),
                        "speedup_of_face_loop": (tot_el / args.steps) / (total_ms / args.steps)}
        if n / (te2 / e2e_steps) > e2e["value"]:
            e2e.update({"value": n / (te2 / e2e_steps), "face_mode": "element"})

    extras = {}
    if fp64_element:
        extras["fp64_element"] = fp64_element
    if not args.no_extras and args.prec == "fp64":
        # FP32 arithmetic, same workload
        op32 = dgp.Operator(mesh["n"], p, geom=w["geom"], op="sipg", prec="fp32", coeff=w["coeff"], **common)
        s32, d32 = src.float(), torch.empty(n, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            op32.apply(s32, d32)
        tot32, l32 = time_applies(torch, op32, s32, d32, args.steps)
        b32 = bytes_per_dof(k, 4, "sipg", w["geom"])
        gbs = b32 * n / (l32 / 1e3) / 1e9
        tf32 = kernel_flops_per_cell(k, "sipg", w["geom"]) * n_cells / (l32 / 1e3) / 1e12
        extras["fp32"] = {"value": n / (tot32 / args.steps / 1e3), "unit": UNIT, "ms_per_step": tot32 / args.steps,
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": gbs / peaks["hbm_gbs"], "bytes_per_dof": b32,
                                       "traffic": measured_traffic("fp32", "element", p, op32.info()["cells_per_block"],
                                                                   wname),
                                       "kernel": "apply_f32_kernel<%d,%d,FULL,SIPG>" % (k, op32.info()["cells_per_block"]),
                                       "alu_tflops": tf32, "alu_peak_tflops": alu["fp32_tflops"]}}
        op32.close()
        # emulated FP64 (double-float on the FP32 pipe), same workload and vectors
        emu = {}
        for mode in (("element", "loop") if loop else ("element",)):
            ope = dgp.Operator(mesh["n"], p, geom=w["geom"], op="sipg", prec="fp64emu", coeff=w["coeff"], **common)
            ope.set_face_mode(mode)
            for _ in range(args.warmup):
                ope.apply(src, dst)
            emu[mode], _ = time_applies(torch, ope, src, dst, args.steps)
            ope.close()
        best = min(emu, key=emu.get)
        tote = emu[best]
        extras["fp64_emulated"] = {
            "value": n / (tote / args.steps / 1e3), "unit": UNIT, "ms_per_step": tote / args.steps,
            "face_mode": best,
            "ms_per_step_by_face_mode": {m: t / args.steps for m, t in emu.items()},
            "arithmetic": "double-float (pairs of binary32, error-free transformations) on the FP32 pipe; "
                          "FP64 vectors; parity with the FP64 oracle at 1e-12",
            "speedup_vs_fp64": (total_ms / args.steps) / (tote / args.steps),
            "hbm": {"achieved": bpd * n / (tote / args.steps / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}}
        # geometry variant G2 (positions stored, J computed in the kernel): the
        # same workload in FP64 (face loop) and FP32, bytes for arithmetic
        g2 = {}
        for prec in ("fp64", "fp32"):
            og = dgp.Operator(mesh["n"], p, geom="positions", op="sipg", prec=prec, coeff=w["coeff"], **common)
            sg = src if prec == "fp64" else src.float()
            dg_ = torch.empty_like(sg)
            for _ in range(args.warmup):
                og.apply(sg, dg_)
            totg, lg = time_applies(torch, og, sg, dg_, args.steps)
            bg = bytes_per_dof(k, 8 if prec == "fp64" else 4, "sipg", "positions")
            g2[prec] = {"value": n / (lg / 1e3), "unit": UNIT, "ms_per_step": lg, "bytes_per_dof": bg,
                        "hbm_frac": bg * n / (lg / 1e3) / 1e9 / peaks["hbm_gbs"],
                        "face_mode": "loop" if prec == "fp64" else "element",
                        "vs_g3": (total_ms / args.steps) / lg if prec == "fp64" else (l32 / lg)}
            og.close()
        extras["g2_positions"] = g2
        # the Hermite-like basis (Sec. 3.1): the same operator in another
        # basis; the binary32 kernel reads two layers of each neighbour instead
        # of k (slim face access)
        her = {}
        for prec in ("fp64", "fp32"):
            oh = dgp.Operator(mesh["n"], p, geom=w["geom"], op="sipg", prec=prec, coeff=w["coeff"], basis="hermite",
                              **common)
            if prec == "fp64" and loop:
                oh.set_face_mode("loop")
            sh = src if prec == "fp64" else src.float()
            dh = torch.empty_like(sh)
            for _ in range(args.warmup):
                oh.apply(sh, dh)
            _, lh = time_applies(torch, oh, sh, dh, args.steps)
            ref_ms = (total_ms / args.steps) if prec == "fp64" else l32
            her[prec] = {"value": n / (lh / 1e3), "unit": UNIT, "ms_per_step": lh,
                         "vs_lagrange": ref_ms / lh, "face_mode": "loop" if prec == "fp64" and loop else "element"}
            oh.close()
        extras["hermite_basis"] = her
        # advection, FP64
        opa = dgp.Operator(mesh["n"], p, geom=w["geom"], op="advection", prec="fp64", **common)
        if loop:
            opa.set_face_mode("loop")
        for _ in range(args.warmup):
            opa.apply(src, dst)
        tota, la = time_applies(torch, opa, src, dst, max(10, args.steps // 2))
        extras["advection_fp64"] = {"value": n / (tota / max(10, args.steps // 2) / 1e3), "unit": UNIT}
        opa.close()
        extras["fp32_degree_sweep"] = fp32_degree_sweep(torch, dgp)

    if not args.no_extras and args.prec == "fp64":
        extras["solve"] = solve_metrics(torch, dgp, args)
        # the mixed-precision workload at full size (64^3 Cartesian and 48^3
        # deformed, p = 3 and 5, to 1e-10): plain FP64 CG against the mixed solver
        extras["solve_config3"] = config3_metrics(torch, dgp, face_mode=args.face_mode, emulated=False)
        extras["batch"] = batch_metrics(torch, dgp, args)
        # many small meshes: where one launch per operator underfills the GPU
        extras["batch_small_meshes"] = batch_metrics(torch, dgp, args, count=64, seed=6, n_lo=3, n_hi=12)
        extras["serve"] = serve_metrics(dgp, policies=(0, 1))
        extras["serve_slots"] = serve_slot_study(dgp)
        # the serving stream's shape (dofs lognormal over 1e4..2e7, degrees
        # 2..6, half Cartesian / half deformed, mixed CG to 1e-8, 120 GB),
        # bounded to 160 requests: saturated, then 90% load with both policies
        extras["serve_config5_bounded"] = serve_metrics(dgp, count=160, seed=11, dof_hi=2e7, rates=(0.5, 0.9),
                                                        policies=(0, 1), max_age_s=5.0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, dict(op="sipg", coeff=w["coeff"]))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp64emu": "f64 (double-float arithmetic)"}[args.prec], "data": "synthetic",
                "config": {"workload": wname, "degree": p, "cells": n_cells,
                           "dofs": n, "geometry": "full per-point Jacobians (G3)", "operator": "SIPG",
                           "boundary": "Dirichlet", "coefficient": "1+0.5 sin(2 pi x)",
                           "l2_policy": "inputs larger than L2 (vector + geometry > 500 MB)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "cells_per_block": cpb_used,
                           "face_mode": ("face loop: two launches, neighbour traces read (dg_set_face_mode)"
                                         if loop else "element-centric fused kernel")},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * (2 if loop else 1),
                "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
