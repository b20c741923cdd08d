#!/usr/bin/env python3
"""Benchmark of the FSPB D_ij path: voxel-beamlet pairs/s and 9-field latency.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload prostate_256|slabs_128|water_32|batched|serving|table_study|superposition|table1]

One step = the whole path (beamlet set-up, Siddon depth tables, VOI
enumeration, FSPB evaluation, threshold + CSR compaction) for the 9-field
synthetic prostate plan (256x256x100 voxels at 2x2x2.5 mm, 9 fields of 16x16
beamlets of 5 mm), inputs resident in HBM.  K steps are timed with CUDA events
on the launching stream; a 256 MB buffer is written between steps so every
step starts with a cold L2.  Under torchrun each rank computes its own plan
on its own GPU (independent replicas, no data-path collective); the timing is
the max over ranks.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the only reference this method has) on a bounded row sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 operations of one voxel-beamlet pair as the evaluation kernel forms it
# (FMA = 2, a packed FP32x2 instruction = two lanes' worth; the exact
# integer <-> float conversions done with FP32 adds are not counted):
# geometry 14 (t, x' and z' in float-float, a_t and b_t), depth 4, beam-model
# table 10, per profile term 23 (scaled arguments y1 and y2: 12, the erf
# pair's combination: 8, the sum of Eq. 3: 3) and 4 erfc evaluations of 18
# (denominator 2, degree-7 Horner 14, the square and the product: 2), and
# the inverse square and products 3: 14 + 4 + 10 + 3 x (23 + 72) + 3.
F_PAIR = 316
FP32_LANES_PER_SM = 128
# MUFU operations (rcp.approx, ex2.approx) of one pair in the evaluation
# kernel's formulation, by lateral profile.  Per profile term one reciprocal
# 1/s and four tails (X and Z at y1 and y2); a Gaussian tail (erfc) is one
# reciprocal t = 1/(1 + p y) and one ex2, a Laplace tail one ex2, a logistic
# tail one ex2 and one reciprocal; one reciprocal 1/t per pair.
MUFU_PAIR = {0: {"rcp": 16, "ex2": 12}, 1: {"rcp": 4, "ex2": 12}, 2: {"rcp": 16, "ex2": 12}}
# HBM3e bandwidth of the part as specified (GB/s), next to the measured copy
HBM_NOMINAL_GBS = 7900.0
# DRAM bytes (read + write) of the evaluation kernel per candidate pair, from
# one Nsight Compute capture of the kernel as built on the 2-field prostate
# (27.85 M pairs, 2.8 MB read + 165.7 MB written); the full workload's
# traffic is this times its pairs
KEVAL_DRAM_BYTES_PER_PAIR = 6.051


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="prostate_256")
    p.add_argument("--cpu-sample-stride", type=int, default=4)
    p.add_argument("--instances", type=int, default=32, help="batched: re-plan instances")
    p.add_argument("--requests", type=int, default=64, help="serving: requests")
    p.add_argument("--rate", type=float, default=4.0, help="serving: mean Poisson arrival rate (1/s)")
    p.add_argument("--no-sub", action="store_true",
                   help="default line without its batched and serving sub-measurements")
    p.add_argument("--stages", action="store_true",
                   help="per-stage device times of W + K whole computations of the workload, one JSON line "
                        "(no tuning, oracle or end-to-end legs: a short program for kernel profilers)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (the job ends when its slowest rank
    does); the identity with one process."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, seconds: float) -> float:
    """Units per second of the whole job: every rank processes its own
    replica's units each step, and the job takes the slowest rank's time."""
    return world * units_per_rank_step * steps / seconds


def oracle_sample(w, stride, nthreads=0):
    """Oracle pairs/s on every `stride`-th row of the workload (all host
    cores, or `nthreads` of them)."""
    import numpy as np
    from oracle import oracle as O
    rows = np.arange(0, w.nrows, stride, dtype=np.int64)
    t = time.perf_counter()
    r = O.compute_workload(w, rows=rows, nthreads=nthreads)
    dt = time.perf_counter() - t
    cores = nthreads if nthreads > 0 else O.max_threads()
    return {"value": r.pairs / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows.size} of {w.nrows} rows (every {stride}th), {r.pairs} pairs, {dt:.2f} s",
            "seconds": dt, "pairs": int(r.pairs)}


class Clocks:
    """SM clock, power and clock-event reasons sampled every 10 ms from NVML
    (read-only queries through libnvidia-ml) while the timed region runs;
    nvidia-smi every 200 ms where the library cannot be loaded."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of NVML
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
            "hw_power_brake_slowdown": 0x80}

    def __init__(self, uuid):
        import threading
        self.sm, self.mx, self.reasons, self.p = [], [], set(), None
        self.source = "nvml"
        self.nvml = self._nvml(uuid)
        if self.nvml is None:
            self.source = "nvidia-smi"
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            try:
                self.p = subprocess.Popen(["nvidia-smi", f"--id={uuid}", f"--query-gpu={self.Q}",
                                           "--format=csv,noheader", "-lms", "200"], stdout=self.f,
                                          stderr=subprocess.DEVNULL)
            except OSError:
                self.p = None
            return
        self.stop_flag = threading.Event()
        self.t = threading.Thread(target=self._poll, daemon=True)
        self.t.start()

    def _nvml(self, uuid):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if not str(uuid).startswith("GPU-") or lib.nvmlDeviceGetHandleByUUID(str(uuid).encode(),
                                                                                 ctypes.byref(h)) != 0:
                return None
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0:
                return None
            self.max_mhz = float(mx.value)
            return lib, h
        except (OSError, AttributeError):
            return None

    def _poll(self):
        import ctypes
        lib, h = self.nvml
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_flag.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                self.sm.append(float(clk.value))
                self.mx.append(self.max_mhz)
            if lib.nvmlDeviceGetCurrentClocksEventReasons(h, ctypes.byref(rs)) == 0:
                for n, bit in self.BITS.items():
                    if rs.value & bit:
                        self.reasons.add(n)
            self.stop_flag.wait(0.01)

    def stop(self):
        if self.nvml is not None:
            self.stop_flag.set()
            self.t.join()
        elif self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.flush()
            rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
            os.unlink(self.f.name)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for r in rows:
                try:
                    self.sm.append(float(r[1].split()[0]))
                    self.mx.append(float(r[2].split()[0]))
                except (ValueError, IndexError):
                    continue
                for n, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        self.reasons.add(n)
        if not self.sm:
            return None
        return {"sm_mhz": statistics.median(self.sm), "sm_max_mhz": max(self.mx), "reasons": sorted(self.reasons),
                "samples": len(self.sm), "source": self.source}


def gpu_id(props, index):
    """nvidia-smi --id for this CUDA device: its UUID when torch exposes it."""
    u = getattr(props, "uuid", None)
    if u:
        u = str(u)
        return u if u.startswith("GPU-") else "GPU-" + u
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        return vis.split(",")[index]
    return str(index)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_0908_4417_gb300 import phantoms as P
    from oracle import oracle as O
    O.build()
    w = P.get(args.workload)
    vals = []
    for _ in range(max(1, args.warmup // 3)):
        oracle_sample(w, args.cpu_sample_stride * 4)
    tot_pairs, tot_s = 0, 0.0
    for _ in range(args.steps):
        s = oracle_sample(w, args.cpu_sample_stride * 4)
        tot_pairs += s["pairs"]
        tot_s += s["seconds"]
        vals.append(s)
    v = tot_pairs / tot_s
    out = {"impl": "reference", "metric": "voxel-beamlet pairs/s", "value": v, "unit": "pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "rows": w.nrows, "fields": len(w.beams), "grid": list(w.grid.shape[::-1])},
           "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"] + f" per step, {args.steps} steps"},
           "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_0908_4417_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    dsc.lib()
    w = P.get(args.workload)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream

    # cpu baseline first (host cores, before the timed GPU work), rank 0 at N=1 only
    cpu = None
    if rank == 0 and world == 1:
        from oracle import oracle as O
        O.build()
        cpu = oracle_sample(w, args.cpu_sample_stride)
        cpu1 = oracle_sample(w, args.cpu_sample_stride * 4, nthreads=1)
        cpu["single_core"] = {k: cpu1[k] for k in ("value", "unit", "cores", "sample")}

    g = dsc.dsc_create_geometry(w.grid, w.density, False, w.model, sp)
    for b in w.beams:
        dsc.dsc_add_beam(g, b)
    timing = dsc.compute_opts(w.tau, w.value_dtype, w.h_frac, dsc.DSC_FLAG_TIMING)
    plain = dsc.compute_opts(w.tau, w.value_dtype, w.h_frac, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    props = torch.cuda.get_device_properties(dev)

    def steps(opts, n, keep):
        """n computations, each after an L2 flush; per-step device ms (and results if kept)"""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        results = []
        for k in range(n):
            flush.fill_(k & 0xff)
            evs[k][0].record(stream)
            results.append(dsc.dsc_compute_dij(g, opts, sp))
            evs[k][1].record(stream)
        stream.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        if not keep:
            for r in results:
                dsc.dsc_release_result(r)
            results = []
        return ms, results

    with torch.cuda.stream(stream):
        # tile shape from the autotuner on this workload, before any timing
        (tc, bps), tune_ms = dsc.dsc_autotune([g], plain, sp, reps=3)
        for k in range(args.warmup):
            r = dsc.dsc_compute_dij(g, timing if k == 0 else plain, sp)
            dsc.dsc_result_wait(r)
            v = dsc.dsc_get_csr(r, False)
            pairs, nnz, nrows, nbeams = int(v.pairs), int(v.nnz), int(v.nrows), int(v.nbeams)
            if k == 0:
                table_entries = int(dsc.dsc_get_beamlets(r, nrows)[:, 15].sum())
                refine_nt, refine_nm, refine_fp32 = dsc.dsc_get_refine_counts(r)
                tiles, tiles_read = dsc.dsc_get_tile_counts(r)
            dsc.dsc_release_result(r)
        # ---- timed region: K steps, device time ----
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = Clocks(gpu_id(props, local if world > 1 else 0))
        n0 = dsc.dsc_launch_count()
        step_ms, _ = steps(plain, args.steps, False)
        launches = dsc.dsc_launch_count() - n0
        clocks = clk.stop()
        total_s = max_over_ranks(sum(step_ms) / 1e3, dev)
        # ---- stage breakdown: the same steps with per-stage events (outside the timed region) ----
        _, results = steps(timing, max(3, min(args.steps, 10)), True)
        stages = [dsc.dsc_get_stage_times(r) for r in results]
        for r in results:
            dsc.dsc_release_result(r)

        # ---- end to end through the C ABI with pinned host buffers ----
        host_rho = torch.from_numpy(np.ascontiguousarray(w.density)).pin_memory()
        vsize = 2 if w.value_dtype == dsc.DSC_VALUE_BF16 else 4
        def host_set():
            return (torch.empty(nrows + 1, dtype=torch.int64).pin_memory(),
                    torch.empty(max(nnz, 1), dtype=torch.int32).pin_memory(),
                    torch.empty(max(nnz, 1) * 4, dtype=torch.uint8).pin_memory(),
                    torch.empty(max(nbeams, 1), dtype=torch.float32).pin_memory())

        # two pinned sets: a step's CSR lands in one while the other's copy is queued
        hsets = (host_set(), host_set())
        h_rp, h_col, h_val, h_sc = hsets[0]
        # n steps, each moving its density up, computing and moving its CSR
        # down, all inside the timed region, which starts and ends with
        # nothing in flight.  Steps are pipelined: step k+1's upload and
        # computation are queued before step k's read-back, and step k's
        # read-back (dsc_copy_csr_to_host_async) is queued behind step k-1's
        # on a second stream, so the host link does not wait for the host.
        e2e_steps = max(10, args.steps)
        cstream = torch.cuda.Stream(dev)
        csp = cstream.cuda_stream

        def read_back_async(res, k):
            hb = hsets[k & 1]
            dsc.dsc_copy_csr_to_host_async(res, hb[0].data_ptr(), hb[1].data_ptr(), hb[2].data_ptr(),
                                           hb[3].data_ptr(), csp)
            e = torch.cuda.Event()
            e.record(cstream)
            return e

        def end_to_end(opts_e, n):
            res, down = [None] * n, [None] * n
            stream.synchronize()
            cstream.synchronize()
            t0 = time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(n):
                dsc.dsc_upload_density(g, host_rho.data_ptr(), False, sp)
                res[k] = dsc.dsc_compute_dij(g, opts_e, sp)
                if k >= 1:
                    down[k - 1] = read_back_async(res[k - 1], k - 1)
                if k >= 2:                         # its host set is reused by step k's read-back
                    down[k - 2].synchronize()
                    dsc.dsc_release_result(res[k - 2])
            down[n - 1] = read_back_async(res[n - 1], n - 1)
            for j in (n - 2, n - 1):
                down[j].synchronize()
                dsc.dsc_release_result(res[j])
            stream.wait_event(down[n - 1])
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record(stream)
            stream.synchronize()
            return max_over_ranks(e0.elapsed_time(e1) / 1e3, dev), max_over_ranks(time.perf_counter() - t0, dev)

        # untimed: both pinned sets and the host link warmed first (the first
        # copies into fresh pinned memory run slower)
        # The host link is shared with the machine's other GPUs and their
        # hosts' traffic, and single runs scatter by over 20%: three runs of
        # e2e_steps each, the median reported (all three listed)
        def e2e_median(opts_e):
            end_to_end(opts_e, 4)
            runs = sorted(end_to_end(opts_e, e2e_steps) for _ in range(3))
            return runs[1], [round(1e3 * r[0] / e2e_steps, 4) for r in runs]

        (e2e_s, wall_s), e2e_runs = e2e_median(plain)
        # the same with BF16 storage (per-beam scale): 6 instead of 8 bytes per kept entry read back
        opts16 = dsc.compute_opts(w.tau, dsc.DSC_VALUE_BF16, w.h_frac, 0)
        (e2e16_s, wall16_s), e2e16_runs = e2e_median(opts16)

        def copies_alone(opts_e, reps=3):
            """A step's own read-back and upload, each alone on an idle GPU (the
            same pinned buffers and calls as the pipelined loop; shortest of
            reps): the bound of the pipelined end-to-end step."""
            r = dsc.dsc_compute_dij(g, opts_e, sp)
            dsc.dsc_result_wait(r)
            down, up = [], []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(cstream)
                dsc.dsc_copy_csr_to_host(r, h_rp.data_ptr(), h_col.data_ptr(), h_val.data_ptr(), h_sc.data_ptr(),
                                         csp)
                b.record(cstream)
                cstream.synchronize()
                down.append(a.elapsed_time(b))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                dsc.dsc_upload_density(g, host_rho.data_ptr(), False, sp)
                b.record(stream)
                stream.synchronize()
                up.append(a.elapsed_time(b))
            dsc.dsc_release_result(r)
            return min(down), min(up)

        copy_ms = copies_alone(plain)
        copy16_ms = copies_alone(opts16)

        # ---- the ALU denominators measured on this GPU (outside the timed region) ----
        pclk = Clocks(gpu_id(props, local if world > 1 else 0))
        alu = dsc.dsc_measure_alu_peaks(200.0, sp)
        alu["clocks"] = pclk.stop()
        # the host link's rate each way, the bound of the end-to-end path
        # (pinned copies of one step's CSR size, outside the timed region)
        link = dsc.dsc_measure_host_link(max(1 << 20, int((nrows + 1) * 8 + nnz * (4 + vsize) + nbeams * 4)), 3, sp)

    dsc.dsc_destroy_geometry(g)
    if rank != 0:
        return
    sub = {}
    if world == 1 and not args.no_sub:
        # the batched (32 uneven re-plan instances) and served (Poisson 4/s)
        # forms against plain per-plan launches, compact: a few steps each
        sub["batched"] = measure_batched(dsc, P.batched(32), stream, steps=3, warmup=1, reps=1)
        sub["serving"] = measure_serving(dsc, P, 32, 4.0, stream, bf16_share=0.25)
    ms = 1e3 * total_s / args.steps
    value = whole_job_rate(pairs, args.steps, world, total_s)
    eval_ms = statistics.mean(s["eval"] for s in stages)
    achieved = F_PAIR * pairs / (eval_ms / 1e3) / 1e12
    peak_mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_mhz = float(mp.get("sm_max_mhz", peak_mhz))
    except (OSError, ValueError):
        pass
    peak = 2 * FP32_LANES_PER_SM * props.multi_processor_count * peak_mhz * 1e6 / 1e12
    stage_ms = {k: round(statistics.mean(s[k] for s in stages), 4) for k in stages[0]}
    h2d = int(host_rho.numel() * 4)
    d2h = int((nrows + 1) * 8 + nnz * 4 + nnz * vsize + nbeams * 4)
    d2h16 = int((nrows + 1) * 8 + nnz * 4 + nnz * 2 + nbeams * 4)

    def link_bound(d2h_bytes, e2e_ms, copies):
        # a step's result down and (pipelined, the other direction) the next
        # step's density up: the slower of the two, each timed alone with the
        # step's own buffers and calls
        down_ms, up_ms = copies
        ms = max(down_ms, up_ms)
        return {"bound_ms_per_step": ms, "frac_of_bound": ms / e2e_ms,
                "d2h_gbs_of_read_back": d2h_bytes / (down_ms * 1e6), "h2d_gbs_of_upload": h2d / (up_ms * 1e6),
                "link_gbs_one_copy": {"d2h": link["d2h_gbs"], "h2d": link["h2d_gbs"]},
                "basis": "the step's CSR read-back (dsc_copy_csr_to_host) and density upload, each alone on an "
                         "idle GPU with the same pinned buffers, shortest of 3; bound = the slower of the two. "
                         "link_gbs_one_copy: one pinned copy of the CSR's size each way (dsc_measure_host_link)"}
    sms = props.multi_processor_count
    hbm_meas = None
    try:
        hbm_meas = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    # MUFU bound of the evaluation kernel: the time its reciprocals and
    # exponentials take at the measured rates, as a share of its time
    m_pair = MUFU_PAIR[int(w.model.profile)]
    mufu_ms = 1e3 * pairs * (m_pair["rcp"] / (alu["rcp_tops"] * 1e12) + m_pair["ex2"] / (alu["ex2_tops"] * 1e12))
    fp32_ms = 1e3 * F_PAIR * pairs / (alu["fp32_tflops"] * 1e12)
    hbm_ms = 1e3 * KEVAL_DRAM_BYTES_PER_PAIR * pairs / (hbm_meas * 1e9) if hbm_meas else 0.0
    binding = max((fp32_ms, "fp32"), (mufu_ms, "mufu"), (hbm_ms, "hbm"))
    # HBM bound of the step: the bytes the path must move (CSR out, density
    # in once, depth tables written and read back) over the step's time
    step_bytes = nnz * (4 + vsize) + 8 * (nrows + 1) + 4 * nbeams + h2d + 2 * 4 * table_entries
    step_gbs = step_bytes / (ms / 1e3) / 1e9
    eval_gbs = KEVAL_DRAM_BYTES_PER_PAIR * pairs / (eval_ms / 1e3) / 1e9
    # the step's roofline: the largest of its arithmetic (FP32, MUFU) and
    # algorithmic-byte times at the measured rates, against the step's time
    step_hbm_ms = 1e3 * step_bytes / (hbm_meas * 1e9) if hbm_meas else 0.0
    t_roof = max((fp32_ms, "fp32"), (mufu_ms, "mufu"), (step_hbm_ms, "hbm"))
    out = {
        "metric": "voxel-beamlet pairs/s",
        "value": value,
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "grid": [w.grid.nx, w.grid.ny, w.grid.nz],
                   "spacing_mm": [w.grid.dx, w.grid.dy, w.grid.dz], "fields": len(w.beams), "rows": nrows,
                   "pairs_per_step": pairs, "nnz_per_step": nnz, "value_dtype": "f32" if vsize == 4 else "bf16",
                   "rel_threshold": w.tau, "l2": "flushed between steps (256 MB write)",
                   "latency_ms_9field": ms,
                   "tuning": {"target_cand": tc, "eval_blocks_per_sm": bps, "autotune_median_ms": tune_ms},
                   "step_ms": {"min": round(min(step_ms), 4), "median": round(statistics.median(step_ms), 4),
                               "max": round(max(step_ms), 4)},
                   "stage_ms": stage_ms,
                   "stage_basis": "per-stage CUDA events in separate steps after the timed region",
                   "fp64_refined_pairs": {"near_threshold": refine_nt, "near_row_max": refine_nm,
                                          "fp32_decided_past_capacity": refine_fp32},
                   "compaction_tiles": {"tiles": tiles, "candidates_per_tile": 128,
                                        "values_read_by_count_pass": tiles_read}},
        "e2e": {"value": whole_job_rate(pairs, e2e_steps, world, e2e_s), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s / e2e_steps,
                "host_wall_ms_per_step": 1e3 * wall_s / e2e_steps,
                "host_link": link_bound(d2h, 1e3 * e2e_s / e2e_steps, copy_ms), "steps": e2e_steps,
                "runs_ms_per_step": e2e_runs,
                "basis": "every step's density upload (pinned), computation and CSR read-back (pinned) inside the "
                         "region, which starts and ends with nothing in flight (CUDA events on the compute stream); "
                         "steps pipelined, each read-back queued with dsc_copy_csr_to_host_async on a second stream "
                         "behind the previous one (two pinned host sets); the median of three such runs"},
        "e2e_bf16": {"value": whole_job_rate(pairs, e2e_steps, world, e2e16_s), "unit": "pairs/s",
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h16,
                     "ms_per_step": 1e3 * e2e16_s / e2e_steps, "host_wall_ms_per_step": 1e3 * wall16_s / e2e_steps,
                     "value_dtype": "bf16 with per-beam scale", "runs_ms_per_step": e2e16_runs,
                     "host_link": link_bound(d2h16, 1e3 * e2e16_s / e2e_steps, copy16_ms)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": KEVAL_DRAM_BYTES_PER_PAIR * pairs,
                     "traffic_basis": "ncu dram bytes per pair of k_eval on prostate_256_2f, times pairs",
                     "kernel": "k_eval",
                     "flop_per_pair": F_PAIR, "eval_ms": eval_ms,
                     "peak_basis": f"FP32 FMA 2x{FP32_LANES_PER_SM} lanes x {sms} SMs "
                                   f"x {peak_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
                     "measured_peak": alu["fp32_tflops"], "frac_of_measured": achieved / alu["fp32_tflops"],
                     "fp32_bound_ms_measured": fp32_ms,
                     "binding": {"resource": binding[1], "bound_ms": binding[0], "frac": binding[0] / eval_ms,
                                 "basis": "the largest of the FP32, MUFU and DRAM times of k_eval's work at the "
                                          "measured rates, over its measured time"},
                     "mufu": {"ops_per_pair": m_pair, "bound_ms": mufu_ms, "frac": mufu_ms / eval_ms,
                              "rates_tops": {"rcp": alu["rcp_tops"], "ex2": alu["ex2_tops"]},
                              "results_per_clk_sm": {
                                  "rcp": alu["rcp_tops"] * 1e12 / (sms * alu["clocks"]["sm_mhz"] * 1e6)
                                  if alu.get("clocks") else None,
                                  "ex2": alu["ex2_tops"] * 1e12 / (sms * alu["clocks"]["sm_mhz"] * 1e6)
                                  if alu.get("clocks") else None},
                              "basis": "pairs x (rcp / rcp rate + ex2 / ex2 rate), rates from the library's "
                                       "measured MUFU loops; frac = that time / k_eval time"},
                     "hbm": {"step_bytes": step_bytes, "step_achieved": step_gbs, "unit": "GB/s",
                             "peak_measured": hbm_meas, "peak_nominal": HBM_NOMINAL_GBS,
                             "step_frac_of_measured": step_gbs / hbm_meas if hbm_meas else None,
                             "step_frac_of_nominal": step_gbs / HBM_NOMINAL_GBS,
                             "k_eval_achieved": eval_gbs,
                             "k_eval_frac_of_measured": eval_gbs / hbm_meas if hbm_meas else None,
                             "k_eval_frac_of_nominal": eval_gbs / HBM_NOMINAL_GBS,
                             "step_bytes_basis": "CSR (col + value + row pointers + beam scales) + density once "
                                                 "+ depth tables written and read"},
                     "measured_alu": alu,
                     "step": {"t_roof_ms": t_roof[0], "resource": t_roof[1], "frac": t_roof[0] / ms,
                              "fp32_ms": fp32_ms, "mufu_ms": mufu_ms, "hbm_ms": step_hbm_ms,
                              "basis": "T_roof = max(pairs x F_pair / measured FP32 rate, the pairs' MUFU operations "
                                       "at the measured rates, the step's algorithmic bytes / measured HBM copy "
                                       "bandwidth); frac = T_roof / the step's time"}},
        "clocks": clocks,
    }
    if cpu is not None:
        out["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "single_core")}
    out.update(sub)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _timed(fn, stream, steps):
    """Device time (s) of `steps` calls of fn on `stream`, events on that stream."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / 1e3


def measure_batched(dsc, ws, stream, steps, warmup, reps=3):
    """Many uneven re-plan instances in one batched launch sequence (one
    persistent evaluation over a shared work queue, replayed as a CUDA graph)
    against the same instances as sequential per-plan launches, same tile
    shape (the autotuner's, on these instances).  Device time per batch with
    CUDA events on the launching stream."""
    sp = stream.cuda_stream
    gs = []
    for w in ws:
        g = dsc.dsc_create_geometry(w.grid, w.density, False, w.model, sp)
        for b in w.beams:
            dsc.dsc_add_beam(g, b)
        gs.append(g)
    opts = dsc.compute_opts(1e-3, dsc.DSC_VALUE_F32, 0.5, 0)
    held = []

    def batch():
        held.extend(dsc.dsc_compute_dij_batch(gs, opts, sp))

    def sequential():
        for g in gs:
            held.append(dsc.dsc_compute_dij(g, opts, sp))

    def drain():
        stream.synchronize()
        for r in held:
            dsc.dsc_release_result(r)
        held.clear()

    import torch
    with torch.cuda.stream(stream):
        (tc, bps), tune_ms = dsc.dsc_autotune(gs, opts, sp, reps=reps)
        for _ in range(warmup):
            batch(); drain(); sequential(); drain()
        batch()
        stream.synchronize()
        pairs = sum(int(dsc.dsc_get_csr(r, False).pairs) for r in held)
        nnz = sum(int(dsc.dsc_get_csr(r, False).nnz) for r in held)
        drain()
        n0 = dsc.dsc_launch_count()
        t_batch = 0.0
        for _ in range(steps):
            t_batch += _timed(batch, stream, 1)
            drain()
        launches = dsc.dsc_launch_count() - n0
        t_seq = 0.0
        for _ in range(steps):
            t_seq += _timed(sequential, stream, 1)
            drain()
    for g in gs:
        dsc.dsc_destroy_geometry(g)
    return {"instances": len(ws), "rows": sum(w.nrows for w in ws), "pairs_per_batch": pairs, "nnz_per_batch": nnz,
            "steps": steps, "batched_pairs_per_s": pairs * steps / t_batch, "batched_ms": 1e3 * t_batch / steps,
            "sequential_pairs_per_s": pairs * steps / t_seq, "sequential_ms": 1e3 * t_seq / steps,
            "batched_over_sequential": t_seq / t_batch,
            "tuning": {"target_cand": tc, "eval_blocks_per_sm": bps, "autotune_median_ms": tune_ms},
            "gpu_launches_per_batch": launches // max(steps, 1),
            "basis": "device time (CUDA events) per batch of all instances; sequential = one dsc_compute_dij per "
                     "instance on the same stream, same tile shape",
            "parity": "tests/test_gpu_parity.py::test_batched_instances_against_oracle (4 instances in full, "
                      "28 on 64 sampled rows) and ::test_batched_bf16_instances"}


def run_batched(args):
    """The batched re-plan workload alone, as its own JSON line."""
    import torch
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    m = measure_batched(dsc, P.batched(args.instances), stream, args.steps, args.warmup)
    out = {"metric": "voxel-beamlet pairs/s (batched re-plan instances)", "value": m["batched_pairs_per_s"],
           "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": m["batched_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batched_{args.instances}", "l2": "working set far above L2 (no flush needed)",
                      **m},
           "gpu_launches": int(m["gpu_launches_per_batch"] * args.steps)}
    print(json.dumps(out), flush=True)


def measure_serving(dsc, P, n_requests, rate, stream, bf16_share=0.0):
    """Continuous-batching server on a seeded Poisson stream of re-plan
    requests (8 resident geometries, fresh 5-9-field beam sets from the
    batched distribution, HBM-footprint admission, 2 device slots), then the
    same requests submitted at once (server throughput) and as sequential
    per-plan launches.  Latency is submit to device completion; the device
    intervals of the slots' launches (CUDA events) show the overlap."""
    import numpy as np
    sp = stream.cuda_stream
    base = [P.batched_instance(7000 + k) for k in range(8)]
    gs = [dsc.dsc_create_geometry(w.grid, w.density, False, w.model, sp) for w in base]
    stream.synchronize()
    draw = P._Draw(8080)
    reqs = []
    for i in range(n_requests):
        k = draw.randint(0, len(base) - 1)
        b0 = base[k].beams[0]
        nf = draw.randint(5, 9)
        beams = [P.Beam(360.0 * draw.u(), b0.sad, b0.iso, b0.a, b0.b, b0.n_u, b0.n_v) for _ in range(nf)]
        reqs.append((k, beams))
    gaps = -np.log(P.uniform01(8081, np.arange(n_requests, dtype=np.uint64))) / rate
    arrive = np.cumsum(gaps) - gaps[0]
    opts = dsc.compute_opts(1e-3, dsc.DSC_VALUE_F32, 0.5, 0)
    opts_bf16 = dsc.compute_opts(1e-3, dsc.DSC_VALUE_BF16, 0.5, 0)
    n_bf16 = int(round(bf16_share * n_requests))

    def serve(times):
        srv = dsc.dsc_server_create(96 << 30, max_inflight=2, max_batch=8)
        t0 = time.perf_counter()
        ids = []
        for i, ((k, beams), ta) in enumerate(zip(reqs, times)):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(dsc.dsc_server_submit(srv, gs[k], beams, opts_bf16 if i < n_bf16 else opts))
        spans = []
        for rid in ids:
            r = dsc.dsc_server_poll(srv, rid, -1)
            spans.append(dsc.dsc_get_server_timing(r))
            dsc.dsc_release_result(r)
        span = time.perf_counter() - t0
        st = dsc.dsc_server_stats(srv)
        dsc.dsc_server_destroy(srv)
        # launches (distinct device intervals) whose interval intersects one on the other slot
        launches = sorted(set(spans))
        overl = sum(1 for a in launches if any(b[0] != a[0] and a[1] < b[2] and b[1] < a[2] for b in launches))
        st["launches"] = len(launches)
        st["launches_overlapping_other_slot"] = overl
        return st, span

    def sequential():
        t0 = time.perf_counter()
        lat, pairs = [], 0
        for i, (k, beams) in enumerate(reqs):
            ts = time.perf_counter()
            g = gs[k]
            dsc.dsc_clear_beams(g)
            for b in beams:
                dsc.dsc_add_beam(g, b)
            r = dsc.dsc_compute_dij(g, opts_bf16 if i < n_bf16 else opts, sp)
            dsc.dsc_result_wait(r)
            pairs += int(dsc.dsc_get_csr(r, False).pairs)
            dsc.dsc_release_result(r)
            lat.append(1e3 * (time.perf_counter() - ts))
        return pairs, time.perf_counter() - t0, lat

    serve(np.zeros(min(8, n_requests)))               # warm-up (module load, pools)
    st_p, span_p = serve(arrive)                        # Poisson arrivals
    st_s, span_s = serve(np.zeros(n_requests))          # all at once: server throughput
    pairs_q, span_q, lat_q = sequential()
    for g in gs:
        dsc.dsc_destroy_geometry(g)
    lat_q = sorted(lat_q)
    return {"requests": n_requests, "resident_geometries": len(gs), "poisson_rate_per_s": rate,
            "bf16_requests": n_bf16, "slots": 2, "max_batch": 8,
            "poisson_p50_ms": st_p["p50_ms"], "poisson_p99_ms": st_p["p99_ms"],
            "poisson_pairs_per_s": st_p["pairs_done"] / span_p,
            "saturated_p50_ms": st_s["p50_ms"], "saturated_p99_ms": st_s["p99_ms"],
            "saturated_pairs_per_s": st_s["pairs_done"] / span_s,
            "sequential_pairs_per_s": pairs_q / span_q,
            "sequential_p50_ms": lat_q[len(lat_q) // 2],
            "sequential_p99_ms": lat_q[min(len(lat_q) - 1, int(0.99 * len(lat_q)))],
            "served_over_sequential": (st_s["pairs_done"] / span_s) / (pairs_q / span_q),
            "saturated_launches": st_s["launches"],
            "saturated_launches_overlapping_other_slot": st_s["launches_overlapping_other_slot"],
            "basis": "latency = submit to device completion (host clock); pairs/s = pairs of all requests over "
                     "the wall time from first submit to last result; overlap from CUDA events on the slots' "
                     "streams",
            "parity": "tests/test_gpu_parity.py::test_server_results_same_alone_and_in_mix (results identical "
                      "alone and in the mix, slots overlapping on the device) and "
                      "::test_server_bf16_request_against_oracle"}


def run_serving(args):
    """The serving workload alone, as its own JSON line."""
    import torch
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    m = measure_serving(dsc, P, args.requests, args.rate, stream)
    out = {"metric": "voxel-beamlet pairs/s (served re-plan requests)", "value": m["saturated_pairs_per_s"],
           "unit": "pairs/s", "n_gpus": 1, "steps": args.requests, "warmup": min(8, args.requests),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": {"workload": f"serving_{args.requests}", **m}}
    print(json.dumps(out), flush=True)


def run_table_study(args):
    """The paper's element-length study (Section 3.2): the depth table at
    full, 1/2, 1/3 and 1/4 voxel spacing, built both as the exact integral
    (Siddon) and as the paper's trilinear samples, on the 9-field prostate.
    Per configuration: the table stage and the whole computation's device
    time (median of `steps`), and the change of the kept D_ij against the
    finest trilinear table (max relative change over entries kept by both,
    entries kept by only one)."""
    import numpy as np
    import torch
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream
    w = P.get("prostate_256")
    g = dsc.geometry_from_workload(w, sp)
    fracs = [(1.0, "1"), (0.5, "1/2"), (1.0 / 3.0, "1/3"), (0.25, "1/4")]
    # h = fraction x min voxel side (2 mm); the voxel's own size along a ray is 2-2.5 mm
    confs = [(mode, f, lab) for mode in (0, 1) for f, lab in fracs]

    def keys(c):
        rows = np.repeat(np.arange(c.nrows, dtype=np.int64), np.diff(c.row_ptr))
        return rows * c.ncols + c.col.astype(np.int64)

    def run(mode, f, timing):
        flags = (dsc.DSC_FLAG_TRILINEAR_TABLE if mode else 0) | (dsc.DSC_FLAG_TIMING if timing else 0)
        return dsc.dsc_compute_dij(g, dsc.compute_opts(w.tau, w.value_dtype, f, flags), sp)

    with torch.cuda.stream(stream):
        r = run(1, 0.25, False)
        ref = dsc.HostCSR(r)
        dsc.dsc_release_result(r)
        ref_k = keys(ref)
        out = []
        for mode, f, lab in confs:
            for _ in range(max(1, args.warmup)):
                dsc.dsc_release_result(run(mode, f, True))
            tab_ms, tot_ms = [], []
            for _ in range(args.steps):
                r = run(mode, f, True)
                t = dsc.dsc_get_stage_times(r)
                tab_ms.append(t["siddon"])
                tot_ms.append(t["total"])
                dsc.dsc_release_result(r)
            r = run(mode, f, False)
            c = dsc.HostCSR(r)
            dsc.dsc_release_result(r)
            k = keys(c)
            _, ia, ib = np.intersect1d(k, ref_k, assume_unique=True, return_indices=True)
            rel = np.abs(c.val[ia].astype(np.float64) / ref.val[ib].astype(np.float64) - 1.0)
            out.append({"table": "trilinear" if mode else "exact", "element": lab + " voxel",
                        "h_mm": f * min(w.grid.dx, w.grid.dy, w.grid.dz),
                        "table_ms": round(statistics.median(tab_ms), 4), "total_ms": round(statistics.median(tot_ms), 4),
                        "nnz": int(c.nnz), "max_rel_change_vs_finest": float(rel.max()) if rel.size else 0.0,
                        "mean_rel_change_vs_finest": float(rel.mean()) if rel.size else 0.0,
                        "only_here": int(k.size - ia.size), "only_in_finest": int(ref_k.size - ib.size)})
    dsc.dsc_destroy_geometry(g)
    tri = [o for o in out if o["table"] == "trilinear"]
    line = {"metric": "depth-table element-length study (9-field prostate)", "value": tri[1]["total_ms"],
            "unit": "ms (trilinear table at 1/2 voxel, whole computation)", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "prostate_256", "reference": "trilinear, 1/4 voxel",
                                           "configs": out}}
    print(json.dumps(line), flush=True)


def run_superposition(args):
    """Eq. 1 on the resident D_ij of the 9-field prostate: dose = sum_j w_j D_j
    (dsc_dose) and the transpose product D g (dsc_beamlet_dot), each timed
    over K calls with CUDA events after W warm-up calls, against HBM
    bandwidth (algorithmic bytes: the CSR read once, 8 B per kept entry, plus
    the per-voxel and per-row vectors)."""
    import numpy as np
    import torch
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream
    w = P.get("prostate_256")
    g = dsc.geometry_from_workload(w, sp)
    res = dsc.dsc_compute_dij(g, dsc.compute_opts(w.tau, w.value_dtype, w.h_frac, 0), sp)
    v = dsc.dsc_get_csr(res, False)
    nrows, ncols, nnz = int(v.nrows), int(v.ncols), int(v.nnz)
    rng = np.random.default_rng(1)
    wt = torch.from_numpy(rng.random(nrows).astype(np.float32)).to(dev)
    gt = torch.from_numpy(rng.random(ncols).astype(np.float32)).to(dev)
    dose = torch.empty(ncols, dtype=torch.float32, device=dev)
    out = torch.empty(nrows, dtype=torch.float32, device=dev)
    peak = None
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in evs:
            a.record(stream)
            fn()
            b.record(stream)
        stream.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    with torch.cuda.stream(stream):
        n0 = dsc.dsc_launch_count()
        t_dose = timed(lambda: dsc.dsc_dose(res, wt.data_ptr(), dose.data_ptr(), sp))
        t_dot = timed(lambda: dsc.dsc_beamlet_dot(res, gt.data_ptr(), out.data_ptr(), sp))
        launches = dsc.dsc_launch_count() - n0
    b_dose = nnz * 8 + (nrows + 1) * 8 + nrows * 4 + ncols * (8 + 8 + 4)
    b_dot = nnz * 8 + (nrows + 1) * 8 + ncols * 4 + nrows * 4
    dsc.dsc_release_result(res)
    dsc.dsc_destroy_geometry(g)
    gbs_dose, gbs_dot = b_dose / t_dose / 1e6, b_dot / t_dot / 1e6
    line = {"metric": "dose superposition (Eq. 1) on the resident CSR", "value": t_dose, "unit": "ms per dose",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "prostate_256", "nrows": nrows, "ncols": ncols, "nnz": nnz,
                       "dose_ms": t_dose, "beamlet_dot_ms": t_dot},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak,
                         "dose": {"achieved": gbs_dose, "frac": gbs_dose / peak if peak else None, "bytes": b_dose},
                         "beamlet_dot": {"achieved": gbs_dot, "frac": gbs_dot / peak if peak else None,
                                         "bytes": b_dot}}}
    print(json.dumps(line), flush=True)


def run_stages(args):
    """W + K whole computations of the named workload through the C ABI, each
    with the library's per-stage CUDA events; prints the median stage times.
    Short and deterministic in its launches, so it serves as the program a
    kernel profiler captures."""
    import torch
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream
    w = P.get(args.workload)
    g = dsc.geometry_from_workload(w, sp)
    opts = dsc.compute_opts(w.tau, w.value_dtype, w.h_frac, dsc.DSC_FLAG_TIMING)
    times = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + args.steps):
            r = dsc.dsc_compute_dij(g, opts, sp)
            dsc.dsc_result_wait(r)
            if k >= args.warmup:
                times.append(dsc.dsc_get_stage_times(r))
            v = dsc.dsc_get_csr(r, False)
            pairs, nnz = int(v.pairs), int(v.nnz)
            dsc.dsc_release_result(r)
    dsc.dsc_destroy_geometry(g)
    med = {k: round(statistics.median(t[k] for t in times), 4) for k in times[0]} if times else {}
    print(json.dumps({"workload": w.name, "pairs": pairs, "nnz": nnz, "steps": args.steps, "stage_ms": med}),
          flush=True)


def run_table1(args):
    """The paper's Table 1 water sweep (Section 3.1) as a second workload:
    five coplanar 10 x 10 cm beams on a 30 cm water cube, voxels 0.50-0.25 cm,
    beamlets 0.20-0.50 cm.  Per case: candidate pairs (the paper's N'_voxel),
    kept entries, device ms per computation (median of K graph replays, L2
    flushed between them) and pairs/s; the paper's own N' and C1060 time
    are carried for context."""
    import torch
    from paper_0908_4417_gb300 import build as B
    B.build()
    from paper_0908_4417_gb300 import dsc, phantoms as P
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    sp = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    paper = {1: (0.864e7, 0.06), 2: (1.80e7, 0.10), 3: (3.23e7, 0.18), 4: (5.27e7, 0.30), 5: (4.97e7, 0.29),
             6: (4.70e7, 0.27), 7: (4.39e7, 0.24)}
    cases = []
    n0 = dsc.dsc_launch_count()
    with torch.cuda.stream(stream):
        for c in range(1, 8):
            w = P.table1_water(c)
            g = dsc.geometry_from_workload(w, sp)
            opts = dsc.compute_opts(w.tau, w.value_dtype, w.h_frac, 0)
            for _ in range(max(3, args.warmup)):
                dsc.dsc_release_result(dsc.dsc_compute_dij(g, opts, sp))
            r = dsc.dsc_compute_dij(g, opts, sp)
            v = dsc.dsc_get_csr(r, False)
            pairs, nnz = int(v.pairs), int(v.nnz)
            dsc.dsc_release_result(r)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for k, (a, b) in enumerate(evs):
                flush.fill_(k & 0xff)
                a.record(stream)
                r = dsc.dsc_compute_dij(g, opts, sp)
                b.record(stream)
                dsc.dsc_release_result(r)
            stream.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in evs)
            dsc.dsc_destroy_geometry(g)
            cases.append({"case": c, "voxel_cm": round(w.grid.dx / 10, 4), "beamlet_cm": w.beams[0].a / 10,
                          "grid": w.grid.nx, "beamlets": w.nrows, "pairs": pairs, "nnz": nnz, "ms": round(ms, 4),
                          "pairs_per_s": pairs / (ms / 1e3), "paper_nprime": paper[c][0],
                          "paper_c1060_s": paper[c][1]})
    launches = dsc.dsc_launch_count() - n0
    big = max(cases, key=lambda x: x["pairs"])
    line = {"metric": "voxel-beamlet pairs/s (Table 1 water sweep)", "value": big["pairs_per_s"], "unit": "pairs/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "table1_water", "value_case": big["case"],
                       "l2": "flushed between steps (256 MB write)", "cases": cases},
            "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.stages:
        run_stages(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "table_study":
        run_table_study(args)
    elif args.workload == "superposition":
        run_superposition(args)
    elif args.workload == "table1":
        run_table1(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
