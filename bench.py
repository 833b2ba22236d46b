"""Throughput of the D3Q19 TRT sweep on GB300, in MFLUP/s (million fluid
lattice-node updates per second) and as a fraction of the HBM roofline.

Default workload: the 256^3 duct (bounce-back walls on four sides, periodic
along x), FP64 PDFs, in-place AA propagation, seeded |u| <= 0.01 initial field,
omega = 1, Lambda = 3/16. One "step" is one time step of the whole lattice.
The lattice (2.55 GB) is far larger than L2 (129 MB), so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line. --impl reference times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1711_11468_gb300 import inputs  # noqa: E402

WORKLOAD = inputs.DUCT_256
DIMS = WORKLOAD["dims"]
# FP64 pipe instructions per fluid lattice update of the FP64 AA sweep, from
# ncu per-opcode counters of the current kernels (DADD 63, DFMA 42, DMUL 14 per
# fluid cell; profiles/dense_aa_f64_duct128_ncu.md, whose figure a CPU test keeps
# equal to this one), the nominal FP64 pipe rate of GB300 (2 per clock per SM at
# 2.07 GHz; the roofline's peak is the live probe's measured rate), and the DRAM
# bytes one launch of that sweep moves on the 256^3 duct: dram__bytes_read + write
# of an even and an odd launch on the 160^3 duct (ncu), 300.6 B per fluid node,
# scaled to the 16,516,096 fluid nodes of the 256^3 duct.
FP64_INSTR_PER_FLUP = 119.0
FP64_INSTR_PER_SEC_NOMINAL = 152 * 2 * 2.07e9
F64_AA_TRAFFIC_PER_LAUNCH = round((1157.4e6 + 1243.8e6) / 2 / 3994240 * 16516096, -6)
GOLDEN_CHANNEL384 = os.path.join(ROOT, "tests", "golden", "channel384_oracle_profile.txt")

METRIC = "MFLUP/s and % of HBM roofline, FP64 vs FP32/FP16-shifted vs batched, at stated error"
UNIT = "MFLUP/s"

# Loop balance per fluid lattice update on a GPU (no write-allocate): 19 loads
# and 19 stores of S bytes, plus the int32 adjacency for the fluid list
# (18 entries every step for pull, every other step for AA).
def bytes_per_flup(elem_bytes: int, indirect: bool, propagation: str, write_allocate: bool = False) -> float:
    """Algorithmic bytes per fluid lattice update (the paper's loop balance, Table 1):
    19 PDFs read and 19 written, plus on a CPU a write-allocate read of the stored
    lines for one-step kernels with ordinary stores (a GPU has none), plus 18 4-byte
    links for a list: every step for pull, every other step for AA."""
    b = 2 * 19 * elem_bytes
    if write_allocate and propagation != "aa":
        b += 19 * elem_bytes
    if indirect:
        b += 72 if propagation == "pull" else 36
    return float(b)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("LBM_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mflups(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Replicas: every rank advances its own copy of the workload; the job's
    throughput is all ranks' fluid updates over the slowest rank's time."""
    return units_per_rank * world / max_seconds / 1e6


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- GPU arm
def make_duct(lbm, stream, precision, propagation, host_u=None, host_flags=None):
    desc = lbm.make_desc(DIMS, precision, lbm.LBM_DIRECT, propagation, periodic=(1, 0, 0))
    h = lbm.lbm_create_lattice(desc, stream)
    flags = inputs.duct_flags(*DIMS) if host_flags is None else host_flags
    lbm.lbm_set_geometry(h, 0, flags)
    lbm.lbm_set_params(h, 0, WORKLOAD["omega"], WORKLOAD["Lambda"], WORKLOAD["force"])
    if host_u is None:
        host_u = inputs.velocity_perturbation(*DIMS, seed=WORKLOAD["seed"], amplitude=WORKLOAD["amplitude"],
                                              flags=flags)
    lbm.lbm_init_equilibrium(h, 0, None, host_u)
    return h, flags


def time_steps(lbm, h, steps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lbm.lbm_step(h, steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def make_porous(lbm, stream, precision, propagation, pack):
    c = inputs.POROUS_256
    desc = lbm.make_desc(c["dims"], precision, lbm.LBM_INDIRECT, propagation)
    h = lbm.lbm_create_lattice(desc, stream)
    lbm.lbm_set_geometry_spheres(h, 0, pack.spheres)
    lbm.lbm_set_params(h, 0, c["omega"], c["Lambda"], c["force"])
    lbm.lbm_init_equilibrium(h, 0)
    return h


def porous_variant(lbm, stream, precision, propagation, steps, pack, peak):
    """The porous medium on a fluid list, autotuned (block size and link
    encoding), then timed with the link table and with the run-indexed code
    (reduced indirect addressing) at the chosen block size."""
    h = make_porous(lbm, stream, precision, propagation, pack)
    timed = {}
    try:
        nf = lbm.lbm_fluid_count(h, 0)
        table_bytes, ria_bytes = lbm.lbm_adjacency_bytes(h, 0)
        lbm.lbm_autotune(h, 4)
        chosen = lbm.lbm_get_run_indexing(h)
        for ria in (chosen, not chosen):
            lbm.lbm_set_run_indexing(h, ria)
            lbm.lbm_step(h, 4)
            timed[ria] = time_steps(lbm, h, steps, stream)
        lbm.lbm_set_run_indexing(h, chosen)
        tuning = lbm.lbm_get_tuning(h)
    finally:
        lbm.lbm_destroy(h)
    elem = {lbm.LBM_F64: 8, lbm.LBM_F32_SHIFTED: 4, lbm.LBM_F16_SHIFTED: 2, lbm.LBM_F64_DOUBLE_FLOAT: 8,
            lbm.LBM_F16_SHIFTED_STOCHASTIC: 2}[precision]
    prop = "pull" if propagation == lbm.LBM_PULL_TWO_GRID else "aa"
    # index bytes per fluid update: pull reads the links every step, AA on odd steps only
    index_share = 1.0 if prop == "pull" else 0.5
    pdf_bpf = bytes_per_flup(elem, False, prop)
    bpf = {True: pdf_bpf + index_share * ria_bytes / nf, False: pdf_bpf + index_share * table_bytes / nf}
    out = {}
    for ria, sec in timed.items():
        mflups = nf * steps / sec / 1e6
        gbs = mflups * 1e6 * bpf[ria] / 1e9
        out["run_indexed" if ria else "link_table"] = {
            "mflups": round(mflups, 1), "bytes_per_flup": round(bpf[ria], 1), "achieved_gbs": round(gbs, 1),
            "roofline_frac": round(gbs / peak, 4)}
    best = out["run_indexed" if chosen else "link_table"]
    return {"mflups": best["mflups"], "bytes_per_flup": best["bytes_per_flup"], "achieved_gbs": best["achieved_gbs"],
            "roofline_frac": best["roofline_frac"], "autotuned": {"threads": tuning[0], "run_indexing": chosen},
            "by_encoding": out, "steps": steps, "fluid_cells": nf,
            "porosity": round(nf / float(np.prod(inputs.POROUS_256["dims"])), 4),
            "workload": "porous 256^3, spheres r 4-12, fluid list + int32 adjacency, half-way bounce-back"}


def batch_variant(lbm, stream, steps, peak):
    """512 independent lattices (channels on full arrays, porous media on fluid
    lists), FP32-shifted, one launch per step replayed from CUDA graphs."""
    specs = inputs.batch_specs(**{k: v for k, v in inputs.BATCH_512.items() if k in ("count", "seed")})
    descs = []
    for sp in specs:
        addr = lbm.LBM_DIRECT if sp.kind == "channel" else lbm.LBM_INDIRECT
        per = (1, 0, 1) if sp.kind == "channel" else (1, 1, 1)
        descs.append(lbm.make_desc(sp.dims, lbm.LBM_F32_SHIFTED, addr, lbm.LBM_AA_INPLACE, per))

    def populate(h, k, sp, lattice):
        if sp.kind == "channel":
            lbm.lbm_set_geometry(h, lattice, sp.flags)
        else:
            lbm.lbm_set_geometry_spheres(h, lattice, sp.spheres)
        lbm.lbm_set_params(h, lattice, sp.omega, sp.Lambda, sp.force)
        lbm.lbm_init_equilibrium(h, lattice)

    h = lbm.lbm_create_batch(descs, stream)
    try:
        for k, sp in enumerate(specs):
            populate(h, k, sp, k)
        nf = sum(lbm.lbm_fluid_count(h, k) for k in range(len(specs)))
        nf_list = sum(lbm.lbm_fluid_count(h, k) for k, sp in enumerate(specs) if sp.kind != "channel")
        ncells = sum(int(np.prod(sp.dims)) for sp in specs)
        lbm.lbm_autotune(h, 6)
        tuning = lbm.lbm_get_tuning(h)
        lbm.lbm_step(h, 4)
        sec = time_steps(lbm, h, steps, stream)
        mem = lbm.lbm_memory_bytes(h)
    finally:
        lbm.lbm_destroy(h)
    mflups = nf * steps / sec / 1e6
    # one launch per lattice per step, for comparison
    singles = [lbm.lbm_create_lattice(d, stream) for d in descs]
    try:
        for k, sp in enumerate(specs):
            populate(singles[k], k, sp, 0)
        import torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for hh in singles:
            lbm.lbm_step(hh, 2)
        torch.cuda.synchronize()
        sk = max(2, steps // 5)
        e0.record(stream)
        for _ in range(sk):
            for hh in singles:
                lbm.lbm_step(hh, 1)
        e1.record(stream)
        e1.synchronize()
        single_mflups = nf * sk / (e0.elapsed_time(e1) / 1e3) / 1e6
    finally:
        for hh in singles:
            lbm.lbm_destroy(hh)
    n_list = sum(1 for sp in specs if sp.kind != "channel")
    # bytes per fluid update: dense channels 152, lists 152 + 36 (AA: 72 B of links every other
    # step), weighted by the fluid nodes of each kind
    bpf = bytes_per_flup(4, False, "aa") + (bytes_per_flup(4, True, "aa") - bytes_per_flup(4, False, "aa")) * nf_list / nf
    return {"mflups": round(mflups, 1), "lattices": len(specs), "fluid_cells": nf, "list_fluid_cells": nf_list,
            "cells": ncells, "bytes_per_flup": round(bpf, 1),
            "achieved_gbs": round(mflups * 1e6 * bpf / 1e9, 1), "roofline_frac": round(mflups * 1e6 * bpf / 1e9 / peak, 4),
            "porous_lattices": n_list, "tuning": {"threads": tuning[0], "cells_per_thread": tuning[1],
                                                  "ctas_per_sm": tuning[2]},
            "one_launch_per_lattice_mflups": round(single_mflups, 1), "steps": steps,
            "device_bytes": mem, "bytes_per_flup_range": [152.0, 188.0],
            "roofline_frac_at_152": round(mflups * 1e6 * 152.0 / 1e9 / peak, 4)}


def geometry_sweep(lbm, stream, steps):
    """The paper's heterogeneity study (Sec. 4.5) on 256^3, FP32-shifted AA:
    `blocks` of edge b with gaps of b (b = 2 ... 16) and the homogeneous `pipe`,
    each on the full array and on the fluid list (half-way bounce-back)."""
    out = {}
    geoms = [(f"blocks_{b}", inputs.blocks_flags(*DIMS, block=b, gap=b), (1, 1, 1)) for b in (2, 4, 8, 16)]
    geoms.append(("pipe", inputs.pipe_flags(*DIMS, solid=inputs.SOLID_HALFWAY), (1, 0, 0)))
    for name, flags, per in geoms:
        nf = int(np.count_nonzero(flags == 0))
        row = {"porosity": round(nf / flags.size, 4)}
        for addr, tag in ((lbm.LBM_DIRECT, "full_array"), (lbm.LBM_INDIRECT, "list")):
            h = lbm.lbm_create_lattice(lbm.make_desc(DIMS, lbm.LBM_F32_SHIFTED, addr, lbm.LBM_AA_INPLACE, per), stream)
            try:
                lbm.lbm_set_geometry(h, 0, flags)
                lbm.lbm_set_params(h, 0, 1.0, 3.0 / 16.0, (1e-6, 0.0, 0.0))
                lbm.lbm_init_equilibrium(h, 0)
                lbm.lbm_step(h, 4)
                sec = time_steps(lbm, h, steps, stream)
            finally:
                lbm.lbm_destroy(h)
            row[tag + "_mflups"] = round(nf * steps / sec / 1e6, 1)
        out[name] = row
    return out


def startup_series(y, t, F, nu, a, b, nterms=4001):
    """Plane Poiseuille start-up from rest: steady parabola minus its decaying modes."""
    L = b - a
    s = F / (2 * nu) * (y - a) * (b - y)
    for n in range(1, nterms, 2):
        s = s - 4 * F * L * L / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * (y - a) / L) \
            * np.exp(-nu * n * n * np.pi ** 2 * t / L ** 2)
    return s


def accuracy_poiseuille64(lbm, stream):
    """The verification set-up (Sec. 2.1) on 64^3 after 100 steps, per storage
    format: max-relative error of the mean velocity profile against the analytic
    start-up series at t + 1/2 and against the FP64-arithmetic GPU sweep."""
    c = inputs.POISEUILLE_64
    dims, ny = c["dims"], c["dims"][1]
    profiles = {}
    for name, prec in (("f64", lbm.LBM_F64), ("f64_double_float", lbm.LBM_F64_DOUBLE_FLOAT),
                       ("f32_shifted", lbm.LBM_F32_SHIFTED), ("f16_shifted", lbm.LBM_F16_SHIFTED),
                       ("f32_shifted_double_float", lbm.LBM_F32_SHIFTED_DOUBLE_FLOAT),
                       ("f16_shifted_stochastic", lbm.LBM_F16_SHIFTED_STOCHASTIC)):
        h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, lbm.LBM_DIRECT, lbm.LBM_AA_INPLACE, (1, 0, 1)), stream)
        try:
            lbm.lbm_set_geometry(h, 0, inputs.channel_flags(*dims))
            lbm.lbm_set_params(h, 0, c["omega"], c["Lambda"], c["force"])
            lbm.lbm_init_equilibrium(h, 0)
            lbm.lbm_step(h, c["steps"])
            profiles[name] = lbm.lbm_read_profile(h, 0, 1, 0)
        finally:
            lbm.lbm_destroy(h)
    nu = (1.0 / c["omega"] - 0.5) / 3.0
    ana = startup_series(np.arange(ny, dtype=float), c["steps"] + 0.5, c["force"][0], nu, 0.5, ny - 1.5)
    m = slice(1, ny - 1)
    ref = profiles["f64"]
    return {k: {"vs_analytic": float(np.abs(v[m] - ana[m]).max() / np.abs(ana[m]).max()),
                "vs_f64": float(np.abs(v[m] - ref[m]).max() / np.abs(ref[m]).max())}
            for k, v in profiles.items()}


def microbench(lbm, stream, elem: int = 8, n: int = 1 << 24, reps: int = 5):
    """copy-19 and update-19 (Sec. 4.1) on 19 arrays of n elements, and the
    host link's copy bandwidth each way: GB/s."""
    import torch
    stride = n
    a = torch.empty(19 * stride * elem, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    a.zero_()
    b.zero_()
    out = {}
    for name in ("copy19", "update19"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(reps + 1):
            e0.record(stream)
            if name == "copy19":
                lbm.lbm_bench_copy19(a.data_ptr(), b.data_ptr(), n, stride, elem, stream)
            else:
                lbm.lbm_bench_update19(a.data_ptr(), n, stride, elem, stream)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name + "_gbs"] = round(2 * 19 * n * elem / best / 1e9, 1)
    del a, b
    out.update(host_link(stream))
    return out


def host_link(stream, nbytes: int = 400 << 20, reps: int = 3):
    """Page-locked host memory <-> HBM by copy-engine transfers: GB/s each way,
    best of `reps` (the floor under the end-to-end number's uploads and
    read-backs)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h.zero_()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}
    with torch.cuda.stream(stream):
        for name, dst, src in (("h2d_pinned_gbs", d, h), ("d2h_pinned_gbs", h, d)):
            best = 1e30
            for _ in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = round(nbytes / best / 1e9, 1)
    del h, d
    return out


def targets_status(f64_mflups, f64_hbm_frac, variants, accuracy384):
    """The workload's targets beside what this run measured: FP64 PDFs on the
    dense duct at >= 80 % of the HBM roofline (by the plain FP64 sweep, bound
    by the FP64 pipe, and by FP64 storage with the double-float collision), and
    FP32-/FP16-shifted storage and the batch beating the plain FP64 sweep, with
    the 384^3 accuracy of the FP32 formats against their 1e-5 target."""
    if not variants:
        return {}
    out = {"f64_dense_hbm_frac_target": 0.8, "f64_arithmetic_hbm_frac": f64_hbm_frac}
    df = variants.get("f64_double_float_aa", {})
    if df:
        out["f64_storage_double_float_hbm_frac"] = df.get("roofline_frac")
    for name in ("f32_shifted_aa", "f16_shifted_aa", "f32_shifted_double_float_aa", "f16_shifted_stochastic_aa",
                 "f32_batched_512"):
        v = variants.get(name, {})
        if v.get("mflups"):
            out[name + "_speedup_over_f64"] = round(v["mflups"] / f64_mflups, 2)
    for name in ("f32_shifted", "f32_shifted_double_float"):
        e = accuracy384.get(name, {}).get("max_rel_vs_oracle")
        if e is not None:
            out[name + "_meets_1e-5"] = bool(e <= 1e-5)
    return out


def fp64_pipe_rate(lbm, stream, iterations: int = 8192, reps: int = 5) -> float:
    """FP64 pipe throughput in G FP64 instructions per second: one full wave of
    resident CTAs, each thread running 16 independent chains of fused
    multiply-adds (about 60 ms per launch); one untimed launch first, then the
    best of `reps`. Chain counts of 4 to 32, blocks of 128 to 1024 threads and
    add or multiply chains all read the same rate on GB300."""
    import torch
    blocks = lbm.lbm_bench_fma64_wave()
    buf = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    best = 1e30
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lbm.lbm_bench_fma64(buf.data_ptr(), blocks, iterations, stream)
        e1.record(stream)
        e1.synchronize()
        if r > 0:
            best = min(best, e0.elapsed_time(e1) / 1e3)
    del buf
    return 16.0 * iterations * blocks * 256 / best / 1e9


def read_golden_profile(path=GOLDEN_CHANNEL384):
    vals = {}
    with open(path) as fh:
        for ln in fh:
            if ln.startswith("#") or not ln.strip():
                continue
            y, v = ln.split()
            vals[int(y)] = float.fromhex(v)
    return np.array([vals[y] for y in range(len(vals))])


def accuracy_channel384(lbm, stream):
    """Every storage format on the 384^3 body-force channel (F = 1e-7, 5000 AA
    steps from rest, the Sec. 2.1 verification set-up at the reduced-precision
    workload's size): the mean velocity profile u_x(y) against the FP64
    oracle's profile (stored by tests/golden/make_channel384_profile.py; the
    oracle is not run here) and against the start-up series at t + 1/2."""
    c = inputs.CHANNEL_384
    dims, steps = c["dims"], c["steps"]
    ny = dims[1]
    ref = read_golden_profile()
    nu = (1.0 / c["omega"] - 0.5) / 3.0
    ana = startup_series(np.arange(ny, dtype=float), steps + 0.5, c["force"][0], nu, 0.5, ny - 1.5)
    m = slice(1, ny - 1)
    out = {"workload": "channel 384^3, F = 1e-7 along x, omega 1, Lambda 3/16, 5000 AA steps from rest",
           "oracle_max_rel_vs_analytic": float(np.abs(ref[m] - ana[m]).max() / np.abs(ana[m]).max()),
           "target_f32": 1e-5}
    names = [("f64", lbm.LBM_F64), ("f64_double_float", lbm.LBM_F64_DOUBLE_FLOAT),
             ("f32_shifted", lbm.LBM_F32_SHIFTED), ("f32_shifted_double_float", lbm.LBM_F32_SHIFTED_DOUBLE_FLOAT),
             ("f16_shifted", lbm.LBM_F16_SHIFTED), ("f16_shifted_stochastic", lbm.LBM_F16_SHIFTED_STOCHASTIC)]
    ncells = float(np.prod(dims))
    for name, prec in names:
        h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, lbm.LBM_DIRECT, lbm.LBM_AA_INPLACE, (1, 0, 1)), stream)
        try:
            lbm.lbm_set_geometry(h, 0, inputs.channel_flags(*dims))
            lbm.lbm_set_params(h, 0, c["omega"], c["Lambda"], c["force"])
            lbm.lbm_init_equilibrium(h, 0)
            lbm.lbm_step(h, steps)
            prof = lbm.lbm_read_profile(h, 0, 1, 0)
            mass = lbm.lbm_read_moments(h, 0)[0]
        finally:
            lbm.lbm_destroy(h)
        out[name] = {
            "max_rel_vs_oracle": float(np.abs(prof[m] - ref[m]).max() / np.abs(ref[m]).max()),
            "l2_rel_vs_oracle": float(np.linalg.norm(prof[m] - ref[m]) / np.linalg.norm(ref[m])),
            "max_rel_vs_analytic": float(np.abs(prof[m] - ana[m]).max() / np.abs(ana[m]).max()),
            "l2_rel_vs_analytic": float(np.linalg.norm(prof[m] - ana[m]) / np.linalg.norm(ana[m])),
            "mass_rel_drift": float(abs(mass - ncells) / ncells),
        }
    return out


def variant(lbm, stream, precision, propagation, steps, nf, peak, steps_per_pass=0):
    """The duct at another storage format or propagation, autotuned; with
    steps_per_pass set, temporal blocking is fixed to it after tuning (its
    launch shape is fixed by the library)."""
    h, _ = make_duct(lbm, stream, precision, propagation)
    try:
        lbm.lbm_autotune(h, 4)
        if steps_per_pass:
            lbm.lbm_set_temporal_blocking(h, steps_per_pass)
        lbm.lbm_step(h, 4)
        sec = time_steps(lbm, h, steps, stream)
        spp = lbm.lbm_get_temporal_blocking(h)
    finally:
        lbm.lbm_destroy(h)
    mflups = nf * steps / sec / 1e6
    elem = {lbm.LBM_F64: 8, lbm.LBM_F32_SHIFTED: 4, lbm.LBM_F16_SHIFTED: 2, lbm.LBM_F64_DOUBLE_FLOAT: 8,
            lbm.LBM_F32_SHIFTED_DOUBLE_FLOAT: 4, lbm.LBM_F16_SHIFTED_STOCHASTIC: 2}[precision]
    bpf = bytes_per_flup(elem, False, "pull" if propagation == lbm.LBM_PULL_TWO_GRID else "aa") / spp
    gbs = mflups * 1e6 * bpf / 1e9
    return {"mflups": round(mflups, 1), "bytes_per_flup": bpf, "achieved_gbs": round(gbs, 1),
            "roofline_frac": round(gbs / peak, 4), "steps": steps, "steps_per_pass": spp}


def run_sweep_only(args):
    """Profiling mode: build the workload, then warm-up and timed steps only."""
    import torch

    from paper_1711_11468_gb300 import lbm
    torch.cuda.set_device(0)
    lbm.load()
    stream = torch.cuda.current_stream()
    prec = lbm.PRECISION[args.precision]
    prop = lbm.LBM_AA_INPLACE if args.prop == "aa" else lbm.LBM_PULL_TWO_GRID
    if args.workload == "duct":
        h, flags = make_duct(lbm, stream, prec, prop)
        nf = int(np.count_nonzero(flags == 0))
    elif args.workload == "channel":
        c = inputs.CHANNEL_384 if DIMS[0] >= 384 else inputs.POISEUILLE_64
        flags = inputs.channel_flags(*DIMS)
        h = lbm.lbm_create_lattice(lbm.make_desc(DIMS, prec, lbm.LBM_DIRECT, prop, (1, 0, 1)), stream)
        lbm.lbm_set_geometry(h, 0, flags)
        lbm.lbm_set_params(h, 0, c["omega"], c["Lambda"], c["force"])
        lbm.lbm_init_equilibrium(h, 0)
        nf = int(np.count_nonzero(flags == 0))
    elif args.workload == "porous":
        c = inputs.POROUS_256
        pack = inputs.sphere_pack(DIMS, c["seed"], c["r_min"], c["r_max"], c["porosity"])
        desc = lbm.make_desc(DIMS, prec, lbm.LBM_INDIRECT, prop)
        h = lbm.lbm_create_lattice(desc, stream)
        lbm.lbm_set_geometry_spheres(h, 0, pack.spheres)
        lbm.lbm_set_params(h, 0, c["omega"], c["Lambda"], c["force"])
        lbm.lbm_init_equilibrium(h, 0)
        nf = lbm.lbm_fluid_count(h, 0)
    else:
        specs = inputs.batch_specs(count=args.batch_count, seed=inputs.BATCH_512["seed"])
        descs = [lbm.make_desc(sp.dims, prec, lbm.LBM_DIRECT if sp.kind == "channel" else lbm.LBM_INDIRECT, prop,
                               (1, 0, 1) if sp.kind == "channel" else (1, 1, 1)) for sp in specs]
        h = lbm.lbm_create_batch(descs, stream)
        for k, sp in enumerate(specs):
            if sp.kind == "channel":
                lbm.lbm_set_geometry(h, k, sp.flags)
            else:
                lbm.lbm_set_geometry_spheres(h, k, sp.spheres)
            lbm.lbm_set_params(h, k, sp.omega, sp.Lambda, sp.force)
            lbm.lbm_init_equilibrium(h, k)
        nf = sum(lbm.lbm_fluid_count(h, k) for k in range(len(specs)))
    if args.tuning:
        lbm.lbm_set_tuning(h, *[int(v) for v in args.tuning.split(",")])
    if args.run_indexing:
        lbm.lbm_set_run_indexing(h, args.run_indexing == "on")
    if args.steps_per_pass:
        lbm.lbm_set_temporal_blocking(h, args.steps_per_pass)
    lbm.lbm_step(h, args.warmup)
    sec = time_steps(lbm, h, args.steps, stream)
    lbm.lbm_destroy(h)
    print(json.dumps({"mode": "sweep-only", "config": args.config, "workload": args.workload, "dims": list(DIMS),
                      "precision": args.precision, "prop": args.prop, "steps": args.steps,
                      "mflups": round(nf * args.steps / sec / 1e6, 1)}), flush=True)


def run_gpu(args):
    import torch

    from paper_1711_11468_gb300 import lbm
    if args.sweep_only:
        return run_sweep_only(args)
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    lbm.load()
    lbm.use_torch_allocator()
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()

    h, flags = make_duct(lbm, stream, lbm.LBM_F64, lbm.LBM_AA_INPLACE)
    nf = int(np.count_nonzero(flags == 0))
    lbm.lbm_autotune(h, 4)
    threads = lbm.lbm_get_tuning(h)[0]
    lbm.lbm_step(h, args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    sec = time_steps(lbm, h, args.steps, stream)
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec_max = max_over_ranks(sec, world, f"cuda:{local}")
    moments = lbm.lbm_read_moments(h, 0)
    lbm.lbm_destroy(h)

    value = whole_job_mflups(nf * args.steps, world, sec_max)
    bpf = bytes_per_flup(8, False, "aa")
    achieved = value / world * 1e6 * bpf / 1e9

    # the FP64 pipe's measured rate, the denominator of the sweep's ALU roofline
    fp64_rate_g = fp64_pipe_rate(lbm, stream)

    # end to end through the C ABI from pinned host buffers: the geometry and the
    # initial velocity field up, K steps, density and velocity back. The host
    # buffers are allocated and filled before the timed region; the launch shape
    # comes from the autotuner's cache (the signature was tuned above).
    N = flags.size
    pinned = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    flags_in = pinned((N,), torch.uint8)
    flags_in[:] = flags
    u_in = pinned((3, N), torch.float64)
    u_in[:] = inputs.velocity_perturbation(*DIMS, seed=WORKLOAD["seed"], amplitude=WORKLOAD["amplitude"],
                                           flags=flags)
    rho_out, u_out = pinned((N,), torch.float64), pinned((3, N), torch.float64)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2, _ = make_duct(lbm, stream, lbm.LBM_F64, lbm.LBM_AA_INPLACE, host_u=u_in, host_flags=flags_in)
    lbm.lbm_autotune(h2, 4)
    lbm.lbm_step(h2, args.steps)
    lbm.lbm_read_macroscopic(h2, 0, rho_out, u_out)
    e2e_sec = time.perf_counter() - t0
    lbm.lbm_destroy(h2)
    e2e_sec = max_over_ranks(e2e_sec, world, f"cuda:{local}")
    e2e_value = whole_job_mflups(nf * args.steps, world, e2e_sec)
    del flags_in, u_in, rho_out, u_out

    variants = {}
    micro = {}
    accuracy = {}
    accuracy384 = {}
    if rank == 0 and not args.no_variants:
        vs = min(args.steps, 200)
        variants["f64_pull_two_grid"] = variant(lbm, stream, lbm.LBM_F64, lbm.LBM_PULL_TWO_GRID, vs, nf, peak)
        variants["f64_double_float_aa"] = variant(lbm, stream, lbm.LBM_F64_DOUBLE_FLOAT, lbm.LBM_AA_INPLACE, vs, nf,
                                                  peak)
        variants["f64_double_float_pull"] = variant(lbm, stream, lbm.LBM_F64_DOUBLE_FLOAT, lbm.LBM_PULL_TWO_GRID, vs,
                                                    nf, peak)
        variants["f32_shifted_aa"] = variant(lbm, stream, lbm.LBM_F32_SHIFTED, lbm.LBM_AA_INPLACE, vs, nf, peak)
        variants["f16_shifted_aa"] = variant(lbm, stream, lbm.LBM_F16_SHIFTED, lbm.LBM_AA_INPLACE, vs, nf, peak)
        variants["f16_shifted_stochastic_aa"] = variant(lbm, stream, lbm.LBM_F16_SHIFTED_STOCHASTIC,
                                                        lbm.LBM_AA_INPLACE, vs, nf, peak)
        variants["f32_shifted_pull_two_steps_per_pass"] = variant(lbm, stream, lbm.LBM_F32_SHIFTED,
                                                                  lbm.LBM_PULL_TWO_GRID, vs, nf, peak, 2)
        variants["f16_shifted_pull_two_steps_per_pass"] = variant(lbm, stream, lbm.LBM_F16_SHIFTED,
                                                                  lbm.LBM_PULL_TWO_GRID, vs, nf, peak, 2)
        variants["f32_shifted_double_float_aa"] = variant(lbm, stream, lbm.LBM_F32_SHIFTED_DOUBLE_FLOAT,
                                                          lbm.LBM_AA_INPLACE, vs, nf, peak)
        c2 = inputs.POROUS_256
        pack = inputs.sphere_pack(c2["dims"], c2["seed"], c2["r_min"], c2["r_max"], c2["porosity"])
        variants["f64_list_aa_porous256"] = porous_variant(lbm, stream, lbm.LBM_F64, lbm.LBM_AA_INPLACE, vs, pack,
                                                           peak)
        variants["f64_list_pull_porous256"] = porous_variant(lbm, stream, lbm.LBM_F64, lbm.LBM_PULL_TWO_GRID, vs,
                                                             pack, peak)
        variants["f64_double_float_list_aa_porous256"] = porous_variant(lbm, stream, lbm.LBM_F64_DOUBLE_FLOAT,
                                                                        lbm.LBM_AA_INPLACE, vs, pack, peak)
        variants["f32_list_aa_porous256"] = porous_variant(lbm, stream, lbm.LBM_F32_SHIFTED, lbm.LBM_AA_INPLACE, vs,
                                                           pack, peak)
        variants["f32_list_pull_porous256"] = porous_variant(lbm, stream, lbm.LBM_F32_SHIFTED, lbm.LBM_PULL_TWO_GRID,
                                                             vs, pack, peak)
        variants["f16_list_aa_porous256"] = porous_variant(lbm, stream, lbm.LBM_F16_SHIFTED, lbm.LBM_AA_INPLACE, vs,
                                                           pack, peak)
        variants["f32_batched_512"] = batch_variant(lbm, stream, min(args.steps, 500), peak)
        variants["f32_aa_geometries256"] = geometry_sweep(lbm, stream, min(args.steps, 50))
        micro = microbench(lbm, stream)
        accuracy = accuracy_poiseuille64(lbm, stream)
        accuracy384 = accuracy_channel384(lbm, stream)

    # The FP64 sweep is bound by the FP64 pipe: its ALU roofline counts FP64 pipe
    # instructions per fluid update (ncu) against the pipe's measured rate.
    alu_achieved = value / world * 1e6 * FP64_INSTR_PER_FLUP / 1e9
    alu = {"bound": "alu", "achieved": round(alu_achieved, 1), "peak": round(fp64_rate_g, 1),
           "unit": "G FP64 instr/s", "frac": round(alu_achieved / fp64_rate_g, 4),
           "traffic": F64_AA_TRAFFIC_PER_LAUNCH,
           "traffic_per_fluid_cell": (round(F64_AA_TRAFFIC_PER_LAUNCH / nf, 1) if F64_AA_TRAFFIC_PER_LAUNCH else None),
           "instr_per_flup": FP64_INSTR_PER_FLUP,
           "peak_source": "measured: live FP64 FMA probe (one wave of resident CTAs, 16 chains per thread)",
           "peak_nominal": round(FP64_INSTR_PER_SEC_NOMINAL / 1e9, 1),
           "frac_of_nominal": round(alu_achieved * 1e9 / FP64_INSTR_PER_SEC_NOMINAL, 4)}
    hbm = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4), "bytes_per_flup": bpf, "target_frac": 0.8,
           "peak_source": peak_kind + " copy bandwidth"}
    roofline = alu if alu["frac"] > hbm["frac"] else dict(hbm, traffic=None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sec_max * 1e3 / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded |u|<=0.01 equilibrium field)",
            "config": {"workload": "D3Q19 TRT duct 256^3, FP64 PDFs, direct addressing, SoA, in-place AA, "
                                   "full-way bounce-back walls on y and z, periodic x",
                       "dims": list(DIMS), "fluid_cells": nf, "omega": WORKLOAD["omega"],
                       "Lambda": WORKLOAD["Lambda"], "l2": "inputs larger than L2 (2.55 GB lattice)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "roofline_hbm": hbm,
            # per-cell view: all N cells counted as updated (solid walls included); the AA
            # kernels skip solid cells, so their PDF bytes per cell update are bpf * N_f / N
            "per_cell": {"cells": N, "mlups": round(value * N / nf, 1),
                         "bytes_per_cell_update": round(bpf * nf / N, 1)},
            "microbench": dict(micro, fp64_fma_per_s_g=round(fp64_rate_g, 1)),
            "tuning": {"threads": threads},
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": (N + 3 * N * 8) / args.steps,
                    "d2h_bytes_per_step": 4 * N * 8 / args.steps},
            "gpu_launches": args.steps,
            "clocks": clk,
            "mass_after": moments[0],
            "variants": variants,
            "accuracy_poiseuille64_max_rel": accuracy,
            "accuracy_channel384": accuracy384,
            "targets": targets_status(value / world, hbm["frac"], variants, accuracy384),
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ CPU oracle arm
def cpu_sample(seconds: float, nthreads: int = 0):
    """Oracle push steps on the duct workload until `seconds` of CPU work
    (nthreads <= 0: every core OpenMP offers)."""
    import oracle
    oracle.build()
    flags = inputs.duct_flags(*DIMS)
    nf = int(np.count_nonzero(flags == 0))
    u = inputs.velocity_perturbation(*DIMS, seed=WORKLOAD["seed"], amplitude=WORKLOAD["amplitude"], flags=flags)
    f = oracle.init_equilibrium(DIMS, flags, None, u)
    g = np.zeros_like(f)
    wm = oracle.omega_minus(WORKLOAD["omega"], WORKLOAD["Lambda"])
    steps, t = 0, 0.0
    while t < seconds or steps == 0:
        t0 = time.perf_counter()
        oracle.step(DIMS, flags, WORKLOAD["omega"], wm, WORKLOAD["force"], f, g, nthreads)
        t += time.perf_counter() - t0
        f, g = g, f
        steps += 1
    return nf * steps / t / 1e6, steps, t, nthreads if nthreads > 0 else oracle.max_threads()


def cpu_baseline(seconds: float):
    v, steps, t, cores = cpu_sample(seconds)
    v1, steps1, t1, _ = cpu_sample(0.0, 1)   # one step on one core
    return {"value": round(v, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle steps of the 256^3 duct ({t:.1f} s, FP64 push, OpenMP)",
            "value_1thread": round(v1, 3), "sample_1thread": f"{steps1} oracle step on 1 core ({t1:.1f} s)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    v, steps, t, cores = cpu_sample(args.cpu_seconds)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "D3Q19 TRT duct 256^3, FP64 CPU oracle (two-grid push)", "dims": list(DIMS)},
            "cpu_baseline": {"value": round(v, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} oracle steps of the 256^3 duct ({t:.1f} s)"},
            "e2e": {"value": round(v, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-only", action="store_true", help="profiling: warm-up and timed steps only")
    ap.add_argument("--dims", type=int, default=0, help="profiling: cubic duct of this size instead of 256")
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "f16", "f64df", "f32df", "f16sr"],
                    help="profiling (with --sweep-only)")
    ap.add_argument("--prop", default="aa", choices=["aa", "pull"], help="profiling (with --sweep-only)")
    ap.add_argument("--workload", default="duct", choices=["duct", "channel", "porous", "batch"],
                    help="profiling (with --sweep-only)")
    ap.add_argument("--config", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4],
                    help="profiling (with --sweep-only): the five workloads - 0 Poiseuille channel 64^3 FP64, "
                         "1 duct 256^3 FP64, 2 porous 256^3 FP64 fluid list, 3 channel 384^3 (--precision), "
                         "4 batch of 512 FP32 lattices")
    ap.add_argument("--batch-count", type=int, default=512, help="profiling: lattices in the batch workload")
    ap.add_argument("--tuning", default="", help="profiling: threads,cells_per_thread,ctas_per_sm")
    ap.add_argument("--steps-per-pass", type=int, default=0, choices=[0, 1, 2],
                    help="profiling: temporal blocking of full-array pull sweeps (2 = two steps per launch)")
    ap.add_argument("--run-indexing", default="", choices=["", "on", "off"],
                    help="profiling: fluid lists read the run-indexed links (on) or the link table (off)")
    args = ap.parse_args()
    if args.config >= 0:
        args.sweep_only = True
        workload, dims, precision = {0: ("channel", 64, "f64"), 1: ("duct", 256, "f64"), 2: ("porous", 256, "f64"),
                                     3: ("channel", 384, args.precision), 4: ("batch", 0, "f32")}[args.config]
        args.workload = workload
        args.dims = dims
        args.precision = precision
    if args.dims:
        global DIMS
        DIMS = (args.dims, args.dims, args.dims)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
