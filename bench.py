#!/usr/bin/env python
"""Benchmark of the F-COO hot path on GB300.

One step = SpMTTKRP on all three modes of the skewed 3-way workload
(12,000 x 9,000 x 28,000, 76M nonzeros, Zipf(1.1) per mode, R = 32 FP32
factors), each mode on its own mode-sorted F-COO copy resident in HBM.  The
headline value is effective GB/s: the algorithmic bytes of the three calls
(stream of Table II + segment map + factor rows read once + output written
once) divided by the device time of the step.

Also reported on the same line: the roofline fraction of the streaming kernel
against the measured HBM copy bandwidth, an end-to-end number through the C
ABI with host buffers (factor upload and result download inside the timed
region), the FP64 oracle timed on the host cores on a bounded sample, SpTTM on
the 4-way workload, CP-ALS (R = 64) seconds per sweep with BF16 and FP32
factors, and the sparse CP fit step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (under torchrun) every rank runs an independent replica of the
workload on its own GPU ("replicas only": the path has no exchange step);
value is the sum over ranks of the work divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import signal
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synth  # noqa: E402

METRIC = "SpMTTKRP/SpTTM effective GB/s (% HBM peak); CP-ALS s/iter, mixed vs FP32"
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 2 ** 20


# ---------------------------------------------------------------- helpers


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def mttkrp_alg_bytes(X, R: int, elem: int) -> int:
    """Compulsory bytes of one SpMTTKRP call: the Table II stream, the segment
    map, every factor row of the product modes read once, the output written once."""
    b = table2_read(X) + X.bytes["segmap"]
    b += sum(X.dims[k] * R * elem for k in X.prod_modes)
    b += X.dims[X.mode] * R * 4
    return int(b)


def table2_read(X) -> int:
    """Table II bytes the kernels read: with 16-bit product-mode indices once
    the handle is compressed (2 instead of 4 bytes per index)."""
    b = X.bytes["table2"]
    if X.bytes.get("pidx16"):
        b += X.bytes["pidx16"] - X.bytes["pidx"]
    return int(b)


def ttm_alg_bytes(X, R: int, elem: int) -> int:
    return int(table2_read(X) + X.dims[X.mode] * R * elem + X.nseg * R * 4)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            self.path = f"/tmp/fcoo_clocks_{os.getpid()}.csv"
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        loaded = [s for s, m, _ in rows if s > 0.5 * m] or [s for s, _, _ in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(m for _, m, _ in rows),
                "samples": len(rows), "reasons": reasons}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


def source_hash() -> str:
    """Hash of the streaming kernel's code (comments and blank lines removed),
    so that the recorded DRAM traffic is used only for the kernel it was
    measured on."""
    import re

    h = hashlib.sha256()
    for f in ("stream_kernel.cuh", "internal.cuh"):
        text = open(os.path.join(ROOT, "paper_1705_09905_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def profile_record():
    """The committed ncu record of the streaming kernel (SpMTTKRP mode 0 of the
    skewed workload), if it was taken on the current kernel source, else None."""
    p = os.path.join(ROOT, "profiles", "k_stream_skewed3_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return d if d.get("source_hash") == source_hash() else None


def traffic_from_profile():
    """dram bytes per launch of the streaming kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    d = profile_record()
    return (d.get("traffic_per_launch_full"), d.get("source_hash")) if d else (None, None)


def gather_roof(rec, nnz: int, t_mode: float, sm_mhz, sms: int):
    """The secondary roofs of the gather-bound streaming kernel, from the
    committed ncu record (counters per nonzero of one mode-0 launch) and the
    live per-mode time: the L1 data path (one 128-byte wavefront per SM clock,
    measured by the gather microbenchmark recorded beside it) and the L2 ->
    SM traffic against the L2 peak that the same capture implies."""
    if not rec or "l1_wavefronts" not in rec:
        return None
    n = rec["captured_nnz"]
    wf = rec["l1_wavefronts"] / n
    clk = (sm_mhz or 2070.0) * 1e6
    roof_s = wf * nnz / (sms * clk)
    l2 = rec["lts_bytes"] / n
    return {"bound": "l1_data_path", "unit": "wavefronts/clk/SM", "peak": 1.0,
            "wavefronts_per_nnz": wf, "achieved": wf * nnz / (sms * clk * t_mode), "frac": roof_s / t_mode,
            "l1_hit_rate": rec.get("l1_hit_rate"), "l2_bytes_per_nnz": l2,
            "l2_GBps": l2 * nnz / t_mode / 1e9, "l2_peak_GBps": rec.get("l2_peak_gbps"),
            "l2_frac": (l2 * nnz / t_mode / 1e9) / rec["l2_peak_gbps"] if rec.get("l2_peak_gbps") else None,
            "source": "ncu counters of profiles/k_stream_skewed3_traffic.json (same kernel source), live time"}


# ---------------------------------------------------------------- CPU oracle baseline


def cpu_baseline_rows(T_host, factors_host, nsample: int, runs: int = 5):
    """The oracle's SpMTTKRP loop in its multi-threaded build (gcc -O3
    -fopenmp, every output row summed by one thread; FP64 bitwise equal to
    the single-threaded oracle) on all host cores, FP64 and FP32 variants, all
    modes, over the first nsample nonzeros (a uniform random subset: the
    generator returns nonzeros in random order).  The nonzeros are grouped by
    row once per mode outside the timing, as the device's F-COO is built once.
    Returns {variant: (GB/s of the same algorithmic bytes as the device
    number, median seconds of `runs` runs)} and the thread count."""
    import oracle

    idx = [a[:nsample] for a in T_host["idx"]]
    val = T_host["val"][:nsample]
    dims = T_host["dims"]
    rows = [oracle.ModeRows(dims, idx, n) for n in range(3)]
    R = factors_host[0].shape[1]
    per_nnz = 2 * 4 + 4 + 1 / 8 + 1 / (8 * 8)
    out = {}
    for name, fp32 in (("fp64", False), ("fp32", True)):
        v = val.astype(np.float32) if fp32 else val
        F = [f.astype(np.float32) for f in factors_host] if fp32 else factors_host
        elem = 4 if fp32 else 8
        times = []
        for _ in range(runs):
            t0 = time.perf_counter()
            for n in range(3):
                oracle.mttkrp_rows(rows[n], v, F, fp32=fp32)
            times.append(time.perf_counter() - t0)
        dt = statistics.median(times)
        b = 3 * nsample * per_nnz + sum(3 * d * R * elem for d in dims)
        out[name] = (b / dt / 1e9, dt)
    return out, oracle.num_threads()


def oracle_sample_rate(T_host, factors_host, nsample: int):
    """FP64 oracle SpMTTKRP, all modes, on the first nsample nonzeros (a uniform
    random subset: the generator returns the nonzeros in random order)."""
    import oracle

    idx = [a[:nsample] for a in T_host["idx"]]
    val = T_host["val"][:nsample]
    t0 = time.perf_counter()
    for mode in range(3):
        oracle.mttkrp(T_host["dims"], idx, val, factors_host, mode)
    dt = time.perf_counter() - t0
    R = factors_host[0].shape[1]
    # the same per-nonzero algorithmic bytes as the device number, scaled to the sample
    per_nnz = 2 * 4 + 4 + 1 / 8 + 1 / (8 * 8)
    b = 3 * nsample * per_nnz + sum(3 * d * R * 4 for d in T_host["dims"])
    return b / dt / 1e9, dt


# ---------------------------------------------------------------- workloads


_HOST = {}


def host_tensor(T, cfg):
    """The workload tensor's COO on the host (uint32 indices, FP64 values), once."""
    if cfg.name not in _HOST:
        _HOST[cfg.name] = {"dims": cfg.dims, "idx": [a.cpu().numpy().astype(np.uint32) for a in T.idx],
                           "val": T.val.double().cpu().numpy()}
    return _HOST[cfg.name]


def build_workload(cfg, dev):
    import paper_1705_09905_gb300 as fc

    t0 = time.perf_counter()
    T = synth.make_tensor(cfg, device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
    t0 = time.perf_counter()
    Xs = [fc.FCOO.build(idx32, T.val, cfg.dims, n, "mttkrp", 8) for n in range(3)]
    t_build = time.perf_counter() - t0
    return T, Xs, t_gen, t_build


def time_spmttkrp(fc, Xs, F, outs, steps, warmup, stream):
    """Returns (total seconds for `steps` steps, per-mode mean call seconds)."""
    for _ in range(warmup):
        for n in range(3):
            fc.spmttkrp(Xs[n], F, out=outs[n], stream=stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps * 3)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for s in range(steps):
        for n in range(3):
            e = ev[s * 3 + n]
            e[0].record(stream)
            fc.spmttkrp(Xs[n], F, out=outs[n], stream=stream)
            e[1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    total = start.elapsed_time(end) / 1e3
    per_mode = [statistics.mean(ev[s * 3 + n][0].elapsed_time(ev[s * 3 + n][1]) for s in range(steps)) / 1e3
                for n in range(3)]
    return total, per_mode


def time_gather_bound(fc, Xs, F, steps, stream):
    """spmttkrp_gather_bound on each mode: the factor-row loads of spmttkrp
    alone (no products, reduction or output).  Returns (per-mode mean call
    seconds, rows loaded per mode)."""
    cnt = [torch.zeros(1, dtype=torch.int64, device=F[0].device) for _ in range(3)]
    for _ in range(3):
        for n in range(3):
            fc.spmttkrp_gather_bound(Xs[n], F, count=cnt[n], stream=stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps * 3)]
    for s in range(steps):
        for n in range(3):
            e = ev[s * 3 + n]
            e[0].record(stream)
            fc.spmttkrp_gather_bound(Xs[n], F, count=cnt[n], stream=stream)
            e[1].record(stream)
    torch.cuda.synchronize()
    per_mode = [statistics.mean(ev[s * 3 + n][0].elapsed_time(ev[s * 3 + n][1]) for s in range(steps)) / 1e3
                for n in range(3)]
    return per_mode, [int(c.item()) for c in cnt]


def gather_bound_record(fc, Xs, F, per_mode, nnz, sm_mhz, sms, stream, steps=20):
    """The gather-only bound beside the full kernel's per-mode times: the
    fraction of it that spmttkrp reaches, and both rates in factor rows per
    SM clock."""
    gb, rows = time_gather_bound(fc, Xs, F, steps, stream)
    clk = (sm_mhz or 2070.0) * 1e6
    return {"ms_per_mode": [t * 1e3 for t in gb], "kernel_ms_per_mode": [t * 1e3 for t in per_mode],
            "rows_per_mode": rows, "rows_per_nnz": [x / nnz for x in rows],
            "frac": sum(gb) / sum(per_mode), "frac_per_mode": [a / b for a, b in zip(gb, per_mode)],
            "rows_per_sm_clk_bound": [x / (t * sms * clk) for x, t in zip(rows, gb)],
            "rows_per_sm_clk_kernel": [x / (t * sms * clk) for x, t in zip(rows, per_mode)],
            "source": "spmttkrp_gather_bound: the factor-row loads of spmttkrp on the same handles and "
                      "factors (C row per nonzero, B row where the fibre or segment changes), same lane "
                      "layout, nothing else; CUDA events, mean of 20 calls per mode"}


def e2e_spmttkrp(fc, Xs, dims, R, steps, stream):
    """Through the public API with host buffers: upload the factors from pinned
    host memory, three SpMTTKRP calls, download the three results, per step."""
    dev = torch.device("cuda")
    g = torch.Generator().manual_seed(7)
    Fh = [torch.randn(d, R, generator=g).pin_memory() for d in dims]
    Oh = [torch.empty(d, R).pin_memory() for d in dims]
    Fd = [torch.empty(d, R, device=dev) for d in dims]
    Od = [torch.empty(d, R, device=dev) for d in dims]

    def step():
        for k in range(3):
            Fd[k].copy_(Fh[k], non_blocking=True)
        for n in range(3):
            fc.spmttkrp(Xs[n], Fd, out=Od[n], stream=stream)
        for n in range(3):
            Oh[n].copy_(Od[n], non_blocking=True)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
        torch.cuda.current_stream().synchronize()
    dt = time.perf_counter() - t0
    h2d = sum(f.numel() * 4 for f in Fh)
    d2h = sum(o.numel() * 4 for o in Oh)
    return dt / steps, h2d, d2h


def bench_spttm(fc, dev, quick, nnz=0):
    cfg = synth.CONFIGS["ttm4"]
    if quick:
        cfg = synth.scaled(cfg, 4_000_000, dims=(500, 400, 300, 50_000))
    if nnz:
        cfg = synth.scaled(cfg, nnz)
    T = synth.make_tensor(cfg, device=dev)
    idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
    X = fc.FCOO.build(idx32, T.val, cfg.dims, 3, "ttm", 8)
    del T, idx32
    U = synth.make_factors([cfg.dims[3]], 16, seed=1, device=dev)[0]
    out = torch.empty((X.nseg, 16), device=dev)
    for _ in range(3):
        fc.spttm(X, U, out=out)
    torch.cuda.synchronize()
    n = 20
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n):
        fc.spttm(X, U, out=out)
    b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3 / n
    byt = ttm_alg_bytes(X, 16, 4)
    res = {"workload": cfg.note, "nnz": X.nnz, "nfib": X.nseg, "R": 16, "ms": t * 1e3,
           "alg_bytes": byt, "GBps": byt / t / 1e9, "GFLOPs": 2 * 16 * X.nnz / t / 1e9}
    # the same with 16-bit indices (the product mode has 50,000 rows): its own,
    # smaller algorithmic bytes
    X.compress_indices()
    t16 = _time_calls(lambda: fc.spttm(X, U, out=out))
    b16 = ttm_alg_bytes(X, 16, 4)
    res["idx16"] = {"ms": t16 * 1e3, "alg_bytes": b16, "GBps": b16 / t16 / 1e9, "speedup": t / t16}
    return res


def ttmc_alg_bytes(X, R: int) -> int:
    """Compulsory bytes of one SpTTMc call: the Table II stream, the segment
    map, the product-mode factor rows read once, the R^(N-1)-wide output
    written once (FP32)."""
    b = X.bytes["table2"] + X.bytes["segmap"]
    b += sum(X.dims[k] * R * 4 for k in X.prod_modes)
    b += X.dims[X.mode] * R ** (X.nmodes - 1) * 4
    return int(b)


def fp32_alu_peak_tflops(dev, sm_mhz: float = 2070.0) -> float:
    """FP32 FMA peak: SMs x 128 FP32 lanes x 2 flops x the maximum SM clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def bench_spttmc(fc, Xs, dims, dev, T=None):
    """SpTTMc (Eq. 4) of every mode of the skewed 3-way workload at R = 8 and
    16 (output widths 64 and 256), FP32 factors, on the SpMTTKRP handles.
    Each nonzero costs R^2 FMAs: the kernel is bound by FP32 issue, not
    HBM, so the roofline is the FP32 FMA peak.  With the tensor T, also the
    by-fibre plan (SpTTM along the last product mode into fibre sums, then
    Eq. 4 over the fibres: R FMAs per nonzero plus R^2 per fibre); its
    "eq4_TFLOPs" counts the same 2 R^2 nnz as the direct kernel."""
    peak = fp32_alu_peak_tflops(dev)
    res = {"alu_peak_tflops": peak, "peak_source": "SMs x 128 FP32 lanes x 2 x 2070 MHz", "ranks": []}
    Xt = {}
    if T is not None:
        idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
        Xt = {b: fc.FCOO.build(idx32, T.val, dims, b, "ttm", 8) for b in (2, 1)}
        del idx32
    for R in (16, 8):
        F = [f.to(dev) for f in synth.make_factors(dims, R, seed=1)]
        Fb = [f.to(torch.bfloat16) for f in F]
        row = {"R": R, "width": R * R, "modes": []}
        for n in range(3):
            Y = torch.empty((dims[n], R * R), device=dev)
            t = _time_calls(lambda: fc.spttmc(Xs[n], F, out=Y))
            fl = 2 * R * R * Xs[n].nnz
            byt = ttmc_alg_bytes(Xs[n], R)
            m = {"mode": n, "ms": t * 1e3, "TFLOPs": fl / t / 1e12, "frac_alu": fl / t / 1e12 / peak,
                 "GBps": byt / t / 1e9, "pct_hbm": byt / t / 1e9 / peaks()[0]}
            tb = _time_calls(lambda: fc.spttmc(Xs[n], Fb, out=Y))
            m["bf16_factors"] = {"ms": tb * 1e3, "TFLOPs": fl / tb / 1e12}
            if Xt:
                plan = fc.SpTTMcPlan(Xt[1 if n == 2 else 2], n, R)
                tp = _time_calls(lambda: plan.run(F, out=Y))
                done = 2 * (R * Xs[n].nnz + R * R * plan.nfib)
                m["by_fibres"] = {"ms": tp * 1e3, "nfib": plan.nfib, "eq4_TFLOPs": fl / tp / 1e12,
                                  "TFLOPs": done / tp / 1e12, "frac_alu": done / tp / 1e12 / peak,
                                  "speedup_vs_direct": t / tp}
                plan.close()
            row["modes"].append(m)
            del Y
        res["ranks"].append(row)
    for X in Xt.values():
        X.close()
    return res


def bench_tucker(fc, Xs, dims, R=8, iters=5):
    """Tucker (HOOI around SpTTMc) on the skewed 3-way workload, rank
    (R, R, R): seconds per iteration over `iters` iterations after one
    untimed iteration from N(0,1) start factors."""
    g = torch.Generator().manual_seed(4)
    st = fc.TuckerState(dims, R, [torch.randn(d, R, generator=g) for d in dims])
    st.iterate(Xs, 1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    st.iterate(Xs, iters)
    b.record()
    torch.cuda.synchronize()
    s = st.stats()
    st.close()
    return {"R": R, "iters_timed": iters, "ms_per_iter": a.elapsed_time(b) / iters, "fit": s["fit"],
            "null_directions": s["null_directions"]}


def _time_calls(fn, n=20, warm=3):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / n


def bench_sweep(fc, dev, quick):
    """Mode, rank and threadlen sweep: SpTTM along every mode of the 4-way
    workload (R = 16), SpMTTKRP of every mode of the skewed 3-way workload at
    R = 8, 16, 32, 64 (FP32 factors), and SpMTTKRP mode 0 at R = 32 for
    threadlen 1..64.  GB/s of algorithmic bytes per call."""
    out = {"spttm_modes": [], "spmttkrp_ranks": []}
    cfg = synth.CONFIGS["ttm4"]
    if quick:
        cfg = synth.scaled(cfg, 4_000_000, dims=(500, 400, 300, 50_000))
    T = synth.make_tensor(cfg, device=dev)
    idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
    for n in range(len(cfg.dims)):
        X = fc.FCOO.build(idx32, T.val, cfg.dims, n, "ttm", 8)
        U = synth.make_factors([cfg.dims[n]], 16, seed=1, device=dev)[0]
        Y = torch.empty((X.nseg, 16), device=dev)
        t = _time_calls(lambda: fc.spttm(X, U, out=Y))
        byt = ttm_alg_bytes(X, 16, 4)
        out["spttm_modes"].append({"mode": n, "dim": cfg.dims[n], "nfib": X.nseg, "ms": t * 1e3,
                                   "GBps": byt / t / 1e9, "pct_hbm": byt / t / 1e9 / peaks()[0]})
        del Y, X
        torch.cuda.empty_cache()
    del T, idx32
    cfg = synth.CONFIGS["skewed3"] if not quick else synth.scaled(synth.CONFIGS["skewed3"], 4_000_000,
                                                                 dims=(1200, 900, 2800))
    T, Xs, _, _ = build_workload(cfg, dev)
    # threadlen (the partition length of the start-flags, tuned per tensor in
    # the paper's Table IV): SpMTTKRP mode 0 at R = 32 on handles built with
    # each value
    out["spmttkrp_threadlen"] = []
    idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
    F = [f.to(dev) for f in synth.make_factors(cfg.dims, 32, seed=1)]
    M = torch.empty((cfg.dims[0], 32), device=dev)
    for tl in (1, 4, 8, 16, 32, 64):
        X = fc.FCOO.build(idx32, T.val, cfg.dims, 0, "mttkrp", tl)
        t = _time_calls(lambda: fc.spmttkrp(X, F, out=M))
        byt = mttkrp_alg_bytes(X, 32, 4)
        out["spmttkrp_threadlen"].append({"threadlen": tl, "ms": t * 1e3, "GBps": byt / t / 1e9})
        X.close()
    del idx32, T, M
    for R in (8, 16, 32, 64):
        F = [f.to(dev) for f in synth.make_factors(cfg.dims, R, seed=1)]
        row = {"R": R, "modes": []}
        for n in range(3):
            M = torch.empty((cfg.dims[n], R), device=dev)
            t = _time_calls(lambda: fc.spmttkrp(Xs[n], F, out=M))
            byt = mttkrp_alg_bytes(Xs[n], R, 4)
            row["modes"].append({"mode": n, "ms": t * 1e3, "GBps": byt / t / 1e9,
                                 "pct_hbm": byt / t / 1e9 / peaks()[0]})
        out["spmttkrp_ranks"].append(row)
    return out


def ttm_handle(fc, T, dims, mode):
    """The SpTTM handle along `mode` of the workload tensor T (on the device)."""
    return fc.FCOO.build([a.to(torch.int32).contiguous() for a in T.idx], T.val, dims, mode, "ttm", 8)


def bench_mttkrp_bf16(fc, Xs, dims, R, steps=50):
    """The same three SpMTTKRP calls with BF16 factors (FP32 accumulation):
    half the gathered bytes per nonzero."""
    dev = torch.device("cuda")
    F = [f.to(dev).to(torch.bfloat16) for f in synth.make_factors(dims, R, seed=1)]
    outs = [torch.empty((dims[n], R), device=dev) for n in range(3)]
    total, per_mode = time_spmttkrp(fc, Xs, F, outs, steps, 5, torch.cuda.current_stream())
    alg = [mttkrp_alg_bytes(Xs[n], R, 2) for n in range(3)]
    gb, _ = time_gather_bound(fc, Xs, F, 20, torch.cuda.current_stream())
    return {"R": R, "factors": "bf16", "ms_per_step": total / steps * 1e3,
            "GBps": sum(alg) * steps / total / 1e9,
            "per_mode_ms": [t * 1e3 for t in per_mode],
            "gather_bound_ms_per_mode": [t * 1e3 for t in gb], "frac_of_gather_bound": sum(gb) / sum(per_mode)}


def host_cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (empty if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return ""


def bench_mttkrp_idx16(fc, Xs, dims, R, steps=50):
    """The headline's three SpMTTKRP calls after index compression (16-bit
    product-mode indices, every dimension <= 65,536), against the same calls
    on the same handles before it: ms per mode, and GB/s of each form's own
    algorithmic bytes (8.14 instead of 12.14 bytes of stream per nonzero)."""
    dev = torch.device("cuda")
    F = [f.to(dev) for f in synth.make_factors(dims, R, seed=1)]
    outs = [torch.empty((dims[n], R), device=dev) for n in range(3)]
    tot32, pm32 = time_spmttkrp(fc, Xs, F, outs, steps, 5, torch.cuda.current_stream())
    alg32 = [mttkrp_alg_bytes(Xs[n], R, 4) for n in range(3)]
    for X in Xs:
        X.compress_indices()
    tot16, pm16 = time_spmttkrp(fc, Xs, F, outs, steps, 5, torch.cuda.current_stream())
    alg16 = [mttkrp_alg_bytes(Xs[n], R, 4) for n in range(3)]
    return {"R": R, "per_mode_ms_idx32": [t * 1e3 for t in pm32], "per_mode_ms_idx16": [t * 1e3 for t in pm16],
            "GBps_idx32": sum(alg32) * steps / tot32 / 1e9, "GBps_idx16": sum(alg16) * steps / tot16 / 1e9,
            "alg_bytes_per_step_idx16": sum(alg16), "speedup": tot32 / tot16}


def bench_cp_als(fc, Xs, dims, sweeps, R=64, fp32_tail=2, Xttm=None, T_host=None):
    """CP-ALS, R = 64, `sweeps` sweeps from the same U(0,1) start: FP32 factor
    storage; BF16 storage throughout; and the mixed schedule, BF16 storage for
    all but the last `fp32_tail` sweeps, which run on FP32 storage
    (cp_state_set_dtype).  With Xttm (the SpTTM handle along mode 2), the
    same three again with modes 0 and 1 through the mode-2 fibre sums
    ("*_fibres").  Seconds per sweep over sweeps 2..`sweeps` (the first
    sweep, which also takes |X|^2, is outside the timing)."""
    init = synth.make_factors(dims, R, seed=0, kind="uniform")
    res = {}
    variants = [("fp32", torch.float32), ("bf16", torch.bfloat16), ("mixed", torch.bfloat16)]
    if Xttm is not None:
        variants += [(n + "_fibres", dt) for n, dt in variants]
    for name, dt in variants:
        st = fc.CPState(dims, R, init, dtype=dt)
        if name.endswith("_fibres"):
            st.use_fibres(Xttm)
        st.iterate(Xs)  # first sweep outside the timing (computes |X|^2 once)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if name.startswith("mixed"):
            st.iterate(Xs, sweeps=sweeps - 1 - fp32_tail)
            st.set_dtype(torch.float32)
            st.iterate(Xs, sweeps=fp32_tail)
        else:
            st.iterate(Xs, sweeps=sweeps - 1)
        b.record()
        torch.cuda.synchronize()
        s = st.stats()
        res[name] = {"s_per_iter": a.elapsed_time(b) / 1e3 / (sweeps - 1), "fit": s["fit"], "iters": s["iters"],
                     "pinv_solves": s["npinv"], "factors": [st.factor(k).float().cpu() for k in range(3)]}
        st.close()
    out = {"R": R, "sweeps": sweeps, "mixed_schedule": f"BF16 storage for sweeps 1-{sweeps - fp32_tail}, "
                                                        f"FP32 for the last {fp32_tail}"}
    names = [n for n, _ in variants]
    for name in names:
        out[name] = {k: v for k, v in res[name].items() if k != "factors"}
    if T_host is not None:
        # Algorithm 1 in FP64 by the oracle (multi-threaded SpMTTKRP loop) from
        # the same start: the reference the equal-fit reading compares with
        import oracle

        t0 = time.perf_counter()
        F, _, fits, npinv = oracle.cp_als_rows(dims, T_host["idx"], T_host["val"],
                                               [f.double().numpy() for f in init], sweeps)
        out["oracle_fp64"] = {"fit": float(fits[-1]), "pinv_solves": npinv, "seconds": time.perf_counter() - t0,
                              "threads": oracle.num_threads()}
        for name in names:
            out[name]["fit_diff_vs_oracle"] = abs(res[name]["fit"] - float(fits[-1]))
            out[name]["factor_rel_vs_oracle"] = [
                float(np.linalg.norm(res[name]["factors"][k].double().numpy() - F[k]) / np.linalg.norm(F[k]))
                for k in range(3)]
    for name in names[1:]:
        out[name]["fit_diff_vs_fp32"] = abs(res[name]["fit"] - res["fp32"]["fit"])
        out[name]["factor_rel_vs_fp32"] = [
            float(torch.linalg.norm(res[name]["factors"][k] - res["fp32"]["factors"][k]) /
                  torch.linalg.norm(res["fp32"]["factors"][k])) for k in range(3)]
        out[name]["speedup_vs_fp32"] = res["fp32"]["s_per_iter"] / res[name]["s_per_iter"]
    return out


def bench_sparse_fit(fc, dev, quick, steps=200, with_oracle=False):
    cfg = synth.CONFIGS["fit3"]
    if quick:
        cfg = synth.scaled(cfg, 1_000_000, dims=(5000, 4000, 3000))
    T = synth.make_tensor(cfg, device=dev)
    idx32 = [a.to(torch.int32).contiguous() for a in T.idx]
    Xs = [fc.FCOO.build(idx32, T.val, cfg.dims, n, "mttkrp", 8) for n in range(3)]
    R = cfg.R
    g = torch.Generator(device=dev).manual_seed(1)
    F = [(torch.randn(d, R, generator=g, device=dev) * R ** (-1 / 6)).requires_grad_(True) for d in cfg.dims]
    opt = torch.optim.Adam(F, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    losses = []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for s in range(steps):
        if s == 5:
            a.record()
        opt.zero_grad()
        loss = fc.SparseCPLoss.apply(Xs, *F)
        loss.backward()
        opt.step()
        if s in (0, steps - 1):
            losses.append(float(loss.item()))
    b.record()
    torch.cuda.synchronize()
    out = {"workload": cfg.note, "steps": steps, "ms_per_step": a.elapsed_time(b) / (steps - 5),
           "loss_first": losses[0], "loss_last": losses[-1], "optimizer": "Adam lr=1e-2",
           "noise_floor": 0.5 * cfg.nnz * cfg.noise_std ** 2,
           "rel_residual_last": (2.0 * losses[-1] / float(T.val.double().pow(2).sum())) ** 0.5}
    if with_oracle:
        # the device's loss at the final factors against the FP64 oracle's
        import oracle

        with torch.no_grad():
            loss_dev = float(fc.SparseCPLoss.apply(Xs, *F).item())
        idx = [a.cpu().numpy().astype(np.uint32) for a in T.idx]
        loss_orc, _, _ = oracle.sparse_fit(cfg.dims, idx, T.val.double().cpu().numpy(),
                                           [f.detach().double().cpu().numpy() for f in F],
                                           want_dfactors=False, want_dvals=False)
        out["loss_final_device"] = loss_dev
        out["loss_final_oracle"] = loss_orc
        out["loss_rel_diff_vs_oracle"] = abs(loss_dev - loss_orc) / loss_orc
    return out


# ---------------------------------------------------------------- arms


def workload_config(args):
    """The skewed 3-way workload; --quick or --nnz scale it (same recipe)."""
    cfg = synth.CONFIGS["skewed3"]
    if args.quick:
        cfg = synth.scaled(cfg, 4_000_000, dims=(1200, 900, 2800))
    if args.nnz:
        cfg = synth.scaled(cfg, args.nnz)
    if args.rank:
        cfg = synth.scaled(cfg, cfg.nnz, R=args.rank)
    return cfg


def run_ours(args):
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1705_09905_gb300 as fc

    cfg = workload_config(args)
    R = cfg.R
    T, Xs, t_gen, t_build = build_workload(cfg, dev)
    F = [f.to(dev) for f in synth.make_factors(cfg.dims, R, seed=1)]
    outs = [torch.empty((cfg.dims[n], R), device=dev) for n in range(3)]
    stream = torch.cuda.current_stream()
    alg = [mttkrp_alg_bytes(Xs[n], R, 4) for n in range(3)]
    step_bytes = sum(alg)
    flops = 3 * 3 * R * cfg.nnz

    barrier(pg)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        total, per_mode = time_spmttkrp(fc, Xs, F, outs, args.steps, args.warmup, stream)
    barrier(pg)
    total = max_over_ranks(pg, total)
    clocks = clk.summary()

    hbm, peak_kind = peaks()
    value = world * step_bytes * args.steps / total / 1e9
    achieved = (sum(alg) / 3) / (sum(per_mode) / 3) / 1e9
    traffic, _ = traffic_from_profile()
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg.note, "dims": list(cfg.dims), "nnz": cfg.nnz, "R": R, "modes": [0, 1, 2],
                   "factors": "fp32 N(0,1), seed 1", "threadlen": 8,
                   "l2": "no flush: each mode's F-COO stream (~0.92 GB) exceeds the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "pct_hbm": value / world / hbm,
        "gflops": world * flops * args.steps / total / 1e9,
        "per_mode": [{"mode": n, "ms": per_mode[n] * 1e3, "alg_bytes": alg[n], "GBps": alg[n] / per_mode[n] / 1e9,
                      "nseg": Xs[n].nseg, "nfib": Xs[n].nfib} for n in range(3)],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": "k_stream + k_carry_fixup per spmttkrp call (fp32 factors, R=32), "
                               "CUDA events around each call",
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json copy bandwidth)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s"},
        "gpu_launches": 2 * 3 * args.steps,
        "clocks": clocks,
        "build_s": {"generate": t_gen, "fcoo_build_3_modes": t_build},
    }
    # end to end through the C ABI with host buffers
    e2e_steps = max(5, min(50, args.steps))
    t_e2e, h2d, d2h = e2e_spmttkrp(fc, Xs, cfg.dims, R, e2e_steps, stream)
    t_e2e = max_over_ranks(pg, t_e2e)
    line["e2e"] = {"value": world * step_bytes / t_e2e / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                   "note": "per step: pinned H2D of the 3 factor matrices, 3 SpMTTKRP calls, D2H of the 3 results; "
                           "F-COO resident (built once, build_s)"}
    if rank == 0 and world == 1 and not args.no_cpu:
        T_host = host_tensor(T, cfg)
        Fh = [f.double().cpu().numpy() for f in F]
        nsample = min(cfg.nnz, args.cpu_sample)
        rates, threads = cpu_baseline_rows(T_host, Fh, nsample)
        n1 = min(cfg.nnz, args.cpu_sample_single)
        gbps1, dt1 = oracle_sample_rate(T_host, Fh, n1)
        line["cpu_baseline"] = {
            "value": rates["fp64"][0], "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"the oracle's SpMTTKRP loop (FP64), multi-threaded build (gcc -O3 -fopenmp, each output "
                      f"row summed by one thread, bitwise the serial oracle), modes 0-2 over the first {nsample} "
                      f"of the {cfg.nnz} nonzeros (a uniform random subset), {threads} threads, median of 5 runs "
                      f"({rates['fp64'][1]:.2f} s per run)",
            "fp32": {"value": rates["fp32"][0], "unit": "GB/s", "s_per_run": rates["fp32"][1],
                     "note": "same loop with FP32 values, factors and sums"},
            "cpu_count": os.cpu_count(), "cpu_model": host_cpu_model(),
            "single_thread_oracle": {"value": gbps1, "unit": "GB/s", "cores": 1,
                                     "sample": f"the FP64 oracle as the tests use it (gcc -O2, one thread), "
                                               f"first {n1} nonzeros, {dt1:.1f} s"}}
    g = gather_roof(profile_record(), cfg.nnz, per_mode[0], clocks.get("sm_mhz"),
                    torch.cuda.get_device_properties(dev).multi_processor_count)
    if g:
        line["roofline"]["gather"] = g
    line["roofline"]["gather_bound"] = gather_bound_record(
        fc, Xs, F, per_mode, cfg.nnz, clocks.get("sm_mhz"),
        torch.cuda.get_device_properties(dev).multi_processor_count, stream)
    # which roof binds: the L2-served factor-row gathers, not HBM (whose
    # fraction is the `frac` above) and not the L1 data path or L2 throughput
    gbr = line["roofline"]["gather_bound"]
    l2f = (g or {}).get("l2_frac")
    line["roofline"]["binding"] = (
        f"factor-row gathers served from L2, at the rows in flight the register file holds: the kernel takes "
        f"{1 / gbr['frac']:.2f}x the time of its row loads alone (gather_bound); HBM at {achieved / hbm:.1%}"
        + (f", L2 at {l2f:.0%} and the L1 data path at {g['frac']:.0%} of their peaks" if g and l2f else "")
        + " are not saturated")
    if not args.no_extras and rank == 0:
        for name, fn in (("mttkrp_bf16", lambda: bench_mttkrp_bf16(fc, Xs, cfg.dims, R)),
                         ("spttm", lambda: bench_spttm(fc, dev, args.quick)),
                         ("spttmc", lambda: bench_spttmc(fc, Xs, cfg.dims, dev, T)),
                         ("tucker", lambda: bench_tucker(fc, Xs, cfg.dims)),
                         ("cp_als", lambda: bench_cp_als(fc, Xs, cfg.dims, 20 if not args.quick else 5,
                                                         Xttm=ttm_handle(fc, T, cfg.dims, 2),
                                                         T_host=None if args.no_cpu else host_tensor(T, cfg))),
                         ("sparse_fit", lambda: bench_sparse_fit(fc, dev, args.quick, with_oracle=not args.no_cpu)),
                         # last: it compresses the workload's handles in place
                         ("mttkrp_idx16", lambda: bench_mttkrp_idx16(fc, Xs, cfg.dims, R))):
            try:
                line[name] = fn()
            except Exception as e:  # reported, not hidden
                line[name] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.synchronize()
    if not args.no_extras and rank == 0:
        try:  # last: the part of the line a short tail shows
            line["summary"] = summarize(line)
        except Exception as e:  # the line is printed whatever the summary does
            line["summary"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def summarize(line):
    """The headline of every extra result, compact, for the end of the line."""
    out = {}

    def get(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r(x, n=4):
        return round(x, n) if isinstance(x, float) else x

    if "spttm" in line:
        t = line["spttm"]
        out["spttm_4way_mode3"] = {"ms": r(get(t, "ms")), "GBps": r(get(t, "GBps"), 1),
                                   "pct_hbm": r(get(t, "GBps") / peaks()[0]) if get(t, "GBps") else None,
                                   "nfib": get(t, "nfib")}
    if "mttkrp_idx16" in line:
        t = line["mttkrp_idx16"]
        out["spmttkrp_idx16_R32"] = {"ms_per_mode": [r(x) for x in get(t, "per_mode_ms_idx16") or []],
                                     "ms_per_mode_idx32": [r(x) for x in get(t, "per_mode_ms_idx32") or []],
                                     "GBps": r(get(t, "GBps_idx16"), 1), "speedup": r(get(t, "speedup"), 3)}
    if "spttm" in line and "idx16" in line["spttm"]:
        t = line["spttm"]["idx16"]
        out["spttm_idx16"] = {"ms": r(get(t, "ms")), "GBps": r(get(t, "GBps"), 1), "speedup": r(get(t, "speedup"), 3)}
    if "mttkrp_bf16" in line:
        t = line["mttkrp_bf16"]
        out["spmttkrp_bf16_R32"] = {"ms_per_step": r(get(t, "ms_per_step")), "GBps": r(get(t, "GBps"), 1),
                                    "frac_of_gather_bound": r(get(t, "frac_of_gather_bound"))}
    if get(line, "roofline", "binding"):
        out["binding_roof"] = get(line, "roofline", "binding")
    gbr = get(line, "roofline", "gather_bound")
    if gbr:
        out["spmttkrp_fp32_R32_gather_bound"] = {"ms_per_mode": [r(x) for x in gbr["ms_per_mode"]],
                                                 "frac": r(gbr["frac"]),
                                                 "rows_per_sm_clk_kernel": [r(x) for x in gbr["rows_per_sm_clk_kernel"]],
                                                 "rows_per_sm_clk_bound": [r(x) for x in gbr["rows_per_sm_clk_bound"]]}
    if "cp_als" in line:
        c = line["cp_als"]
        out["cp_als_R64_20"] = {
            k: {"s_per_iter": r(get(c, k, "s_per_iter"), 6), "fit": r(get(c, k, "fit"), 7),
                "fit_diff_vs_oracle": r(get(c, k, "fit_diff_vs_oracle"), 8),
                "factor_rel_vs_oracle": [r(x) for x in (get(c, k, "factor_rel_vs_oracle") or [])]}
            for k in ("fp32", "bf16", "mixed") if k in c}
        out["cp_als_R64_20"]["oracle_fit"] = r(get(c, "oracle_fp64", "fit"), 7)
        out["cp_als_R64_20"]["mixed_speedup_vs_fp32"] = r(get(c, "mixed", "speedup_vs_fp32"), 3)
    if "sparse_fit" in line:
        f = line["sparse_fit"]
        out["sparse_fit"] = {"ms_per_step": r(get(f, "ms_per_step")), "loss_first": r(get(f, "loss_first"), 1),
                             "loss_last": r(get(f, "loss_last"), 1), "noise_floor": r(get(f, "noise_floor"), 1),
                             "loss_rel_diff_vs_oracle": r(get(f, "loss_rel_diff_vs_oracle"), 9)}
    if "spttmc" in line:
        out["spttmc_mode0_TFLOPs"] = {str(x.get("R")): r(get(x, "modes")[0].get("TFLOPs"), 2)
                                      for x in get(line, "spttmc", "ranks") or []}
    if "tucker" in line:
        out["tucker_R8_ms_per_iter"] = r(get(line, "tucker", "ms_per_iter"), 3)
    return out


def run_reference(args):
    """The FP64 oracle, as it stands, on the host cores: each step is the three
    SpMTTKRP modes over a bounded sample of the same workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload_config(args)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    T = synth.make_tensor(cfg, device=dev)
    T_host = {"dims": cfg.dims, "idx": [a.cpu().numpy().astype(np.uint32) for a in T.idx],
              "val": T.val.double().cpu().numpy()}
    Fh = [f.double().numpy() for f in synth.make_factors(cfg.dims, cfg.R, seed=1)]
    nsample = min(cfg.nnz, args.ref_sample)
    for _ in range(args.warmup):
        oracle_sample_rate(T_host, Fh, min(nsample, 100_000))
    rates, times = [], []
    for _ in range(args.steps):
        g, dt = oracle_sample_rate(T_host, Fh, nsample)
        rates.append(g)
        times.append(dt)
    value = statistics.mean(rates)
    sample = (f"FP64 C oracle SpMTTKRP, modes 0-2, first {nsample} of {cfg.nnz} nonzeros per step "
              f"(uniform random subset)")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": cfg.note, "dims": list(cfg.dims), "nnz": cfg.nnz, "R": cfg.R, "modes": [0, 1, 2]},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="small workload for a fast check")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--nnz", type=int, default=0, help="scale the workload to this many nonzeros (same dims)")
    ap.add_argument("--rank", type=int, default=0, help="override R")
    ap.add_argument("--cpu-sample", type=int, default=40_000_000)
    ap.add_argument("--cpu-sample-single", type=int, default=4_000_000)
    ap.add_argument("--ref-sample", type=int, default=2_000_000)
    ap.add_argument("--part", default="all",
                    choices=["all", "spttm", "spttmc", "tucker", "cp", "fit", "sweep", "bf16"],
                    help="only one extra line, for profiling: spttm (4-way workload, --nnz scales it), "
                         "bf16 (SpMTTKRP of the skewed 3-way workload with BF16 factors, --nnz and --rank "
                         "scale it), "
                         "spttmc (SpTTMc of every mode of the skewed 3-way workload, R = 8 and 16), "
                         "tucker (HOOI at R = 8 on the skewed 3-way workload), "
                         "cp (CP-ALS on the skewed 3-way workload), fit (sparse CP fit) or sweep "
                         "(SpTTM along every mode, SpMTTKRP at R = 8..64)")
    ap.add_argument("--sweeps", type=int, default=20, help="CP-ALS sweeps of the cp line")
    args = ap.parse_args()
    if args.part != "all":
        import paper_1705_09905_gb300 as fc

        dev = torch.device("cuda", 0)
        if args.part == "spttm":
            line = bench_spttm(fc, dev, args.quick, args.nnz)
        elif args.part == "fit":
            line = bench_sparse_fit(fc, dev, args.quick)
        elif args.part == "bf16":
            cfg = workload_config(args)
            _, Xs, _, _ = build_workload(cfg, dev)
            line = bench_mttkrp_bf16(fc, Xs, cfg.dims, cfg.R)
            line["workload"] = cfg.note
        elif args.part == "sweep":
            line = bench_sweep(fc, dev, args.quick)
        elif args.part == "tucker":
            cfg = workload_config(args)
            _, Xs, _, _ = build_workload(cfg, dev)
            line = bench_tucker(fc, Xs, cfg.dims, iters=args.sweeps if args.sweeps != 20 else 5)
        elif args.part == "spttmc":
            cfg = workload_config(args)
            T, Xs, _, _ = build_workload(cfg, dev)
            line = bench_spttmc(fc, Xs, cfg.dims, dev, T)
            line["tucker"] = bench_tucker(fc, Xs, cfg.dims)
        else:
            cfg = workload_config(args)
            T, Xs, _, _ = build_workload(cfg, dev)
            line = bench_cp_als(fc, Xs, cfg.dims, args.sweeps, Xttm=ttm_handle(fc, T, cfg.dims, 2),
                                T_host=host_tensor(T, cfg))
        print(json.dumps(line), flush=True)
        return
    if args.impl == "reference":
        args.steps = 5 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else args.warmup
        run_reference(args)
    else:
        args.steps = 300 if args.steps is None else args.steps
        args.warmup = 10 if args.warmup is None else args.warmup
        if args.warmup < 3:
            raise SystemExit("--warmup must be >= 3")
        run_ours(args)


if __name__ == "__main__":
    main()
