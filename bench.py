#!/usr/bin/env python3
"""Superblock H·v benchmark (direct n-leg DMRG, arXiv 0707.0159).

Workload: the 3-leg Hubbard ladder superblock, t = 1, U = 8, column d = 64,
blocks of m = 256 seeded states (V is 16384 x 16384, dense, no sectors).
One step = one full superblock H·v, Y = H_l V + V H_r^T + H_c V_c, through
dmrg2d_apply_H on inputs already resident in HBM.  value = algorithmic flops
of one H·v x steps x ranks / time.  V (>= 1 GB) is larger than the 129 MB L2,
so no flush is needed between steps.

Also reported: the roofline of the dominant kernel (CUDA events around every
launch of it, from the library's own timing hook), the end-to-end rate through
the same call with the vector staged from/to pinned host memory (pipelined over
three streams), SM clocks sampled during the timed region, the CPU oracle timed
on a bounded sample, the time to the ground energy (residual 1e-7 |E|) of the
mixed-precision solver (--no-tte to skip; --tte-fp64 adds the plain FP64 Lanczos,
which takes over 25 minutes), the H·v of the other workloads (the two m = 1024 sector
superblocks and the small FP64 one with its Lanczos step latency; --no-other-workloads
to skip), and with --sweep the DMRG sweep on a 4 x 12 ladder (--sweep-profile: its
kernel shares under the CUDA profiler).

  python bench.py [--gpus N --steps K --warmup W] [--precision tf32|bf16|fp32|fp64]
  python bench.py --impl reference     # the CPU oracle on the same workload
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

METRIC = "superblock H·v TFLOP/s & time to ground energy at 1e-8 rel. vs plain FP64"

# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture of
# this workload (dram__bytes_read.sum + dram__bytes_write.sum), keyed by tile
# configuration name and dtype.  They hold only for the kernel code they were taken on:
# `traffic` is reported as null when the device part of csrc/hv_tc.cu (everything before
# its host-side section) together with csrc/tc_ptx.cuh no longer has this SHA-256.
NCU_TRAFFIC = {
    "kernel sha256": "d49bf130d81d1a0bdd43a4515dc1382c9e7a80cca9432f14a5533abd182f5af8",
    "bytes": {
        "CTA-pair kernel 256x256 (8x8-tile blocked raster), phase-2 V in one 3-D copy|tf32":
            15.21e9 + 1.07e9,
        "dense kernel 128x256 (8x8-tile blocked raster), phase-2 V in one 3-D copy|bf16":
            6.81e9 + 1.06e9,
    },
}


def kernel_digest():
    """SHA-256 of the tensor-core kernels' source: csrc/hv_tc.cu up to its host-side
    section, then csrc/tc_ptx.cuh."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_0707_0159_gb300", "csrc")
    with open(os.path.join(csrc, "hv_tc.cu"), "rb") as f:
        hv = f.read()
    with open(os.path.join(csrc, "tc_ptx.cuh"), "rb") as f:
        ptx = f.read()
    cut = hv.find(b"// ---- host side")
    return hashlib.sha256((hv if cut < 0 else hv[:cut]) + ptx).hexdigest()


def ncu_traffic(config_name, dtype):
    if kernel_digest() != NCU_TRAFFIC["kernel sha256"]:
        return None
    return NCU_TRAFFIC["bytes"].get(f"{config_name}|{dtype}")
WORKLOAD = "ladder3_hubbard_d64_m256_dense"
# the synthetic superblocks of the benchmark: name -> (builder, H·v precision by default,
# configuration keys of the JSON line)
WORKLOADS = {
    "ladder3_hubbard_d64_m256_dense": (
        lambda synth: synth.workload_ladder3_hubbard_m256(), "tf32",
        {"m": 256, "d": 64, "n_legs": 3, "t": 1.0, "U": 8.0}),
    "ladder3_hubbard_d64_m128_dense": (   # the same model at m = 128 (V 8192^2, 256 MB)
        lambda synth: synth.workload_ladder3_hubbard_m256(m=128), "tf32",
        {"m": 128, "d": 64, "n_legs": 3, "t": 1.0, "U": 8.0}),
    "ladder2_hubbard_d16_m512_dense": (   # a reduced superblock for the CTA-pair kernel
        lambda synth: (synth.model("hubbard", 2, t=1.0, U=8.0), synth.hubbard_block(512, 2, 10),
                       synth.hubbard_block(512, 2, 11), None), "tf32",
        {"m": 512, "d": 16, "n_legs": 2, "t": 1.0, "U": 8.0}),
    "ladder4_heisenberg_d16_m1024_sectors": (
        lambda synth: synth.workload_ladder4_heisenberg_sectors(), "bf16",
        {"m": 1024, "d": 16, "n_legs": 4, "J": 1.0, "sectors": "S^z_tot = 0, 7 block sectors"}),
    "ladder3_hubbard_d64_m1024_sectors": (
        lambda synth: synth.workload_ladder3_hubbard_sectors(), "tf32",
        {"m": 1024, "d": 64, "n_legs": 3, "t": 1.0, "U": 8.0,
         "sectors": "(N_up, N_dn) = (15, 15), 25 block sectors"}),
    "ladder2_heisenberg_d4_m64": (
        lambda synth: synth.workload_ladder2_heisenberg_m64(), "fp64",
        {"m": 64, "d": 4, "n_legs": 2, "J": 1.0}),
}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds: float = 15.0, workload: str = WORKLOAD):
    """The oracle's H·v on the same workload, timed on a bounded slab of its outputs.

    The slab is rows i1 < r of every tile in the first i3-column of V; its
    algorithmic work is the fraction (r/m1)(1/d) of one H·v.  The oracle applies the
    dense superblock (it has no sector layout): for a sector workload the rate is that of
    the dense form of the same blocks.
    """
    from oracle.superblock import Superblock
    from paper_0707_0159_gb300 import synth
    mdl, left, right, _ = WORKLOADS[workload][0](synth)
    sb = Superblock(mdl, left, right)
    v = synth.start_vector(sb.n_vec, 12)
    t0 = time.perf_counter()
    sb.apply_slab(v, [0], [0])
    t1 = time.perf_counter() - t0
    r = int(max(1, min(sb.m1, seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    sb.apply_slab(v, list(range(r)), [0])
    dt = time.perf_counter() - t0
    frac = (r / sb.m1) * (1.0 / sb.d)
    flops = _flops_dense_structure(sb) * frac
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": _cpu_threads(),
            "kind": "oracle",
            "sample": f"oracle 4-index H·v restricted to i1 < {r} and i3 = 0 "
                      f"({frac:.2e} of one H·v), {dt:.1f} s, numpy FP64"}


def _cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        return max(i.get("num_threads", 1) for i in threadpool_info()) or os.cpu_count()
    except Exception:
        return os.cpu_count()


def _flops_dense_structure(sb):
    """Algorithmic flops of one H·v counted from the oracle's term structure (CPU only)."""
    import numpy as np
    d, m1, m4 = sb.d, sb.m1, sb.m4
    posL = np.eye(d, dtype=bool)
    for _, X, _ in sb.terms_l[2:]:
        posL |= X != 0
    posR = np.eye(d, dtype=bool)
    for _, X, _ in sb.terms_r[2:]:
        posR |= X != 0
    Hc = sb.col.H
    eye = np.eye(d, dtype=bool)
    offL = (Hc != 0) & ~posL & ~eye
    offR = (Hc != 0) & ~posR & ~eye
    S = (sb.H_center() != 0) | np.kron(eye, offL) | np.kron(offR, eye)
    return (2.0 * posL.sum() * m1 * m1 * d * m4 + 2.0 * posR.sum() * m4 * m4 * m1 * d
            + 2.0 * S.sum() * m1 * m4)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(seconds=3.0, workload=args.workload)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(seconds=float(args.ref_seconds), workload=args.workload))
    total = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded blocks, numpy default_rng)",
            "config": {"workload": args.workload, **WORKLOADS[args.workload][2]},
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's time (every rank gets it); x itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse_cpulist(text: str) -> set:
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_near_gpu(index: int):
    """Restrict this process to the CPUs the GPU's PCI device reports as local (sysfs
    local_cpulist), so pinned host buffers allocated afterwards land in the memory next
    to the GPU's host link.  Returns (previous affinity, bound CPUs) or None when the
    topology is not readable or shares no CPU with the current affinity."""
    import torch
    try:
        p = torch.cuda.get_device_properties(index)
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bdf}/local_cpulist") as f:
            local = parse_cpulist(f.read())
        prev = os.sched_getaffinity(0)
        use = local & prev
        if not use or use == prev:
            return None
        os.sched_setaffinity(0, use)
        return prev, sorted(use)
    except (AttributeError, OSError, ValueError):
        return None


def job_tflops(flops_per_rank_step: float, ms: float, world: int) -> float:
    """Whole-job throughput: every rank does one H·v of its own replica per step, the job
    step takes the slowest rank's time."""
    return world * flops_per_rank_step / (ms * 1e-3) / 1e12


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_0707_0159_gb300 import dmrg2d, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    prec = dmrg2d.PRECISION[args.precision]

    build, _, wl_config = WORKLOADS[args.workload]
    mdl, left, right, target = build(synth)
    ops = dmrg2d.build_ops(mdl, left, right, target=target)
    info = ops.info
    n, flops = info["n_vec"], info["flops_per_apply"]
    pad = dmrg2d.sector_dense_index(ops) < 0 if target is not None else None
    if prec in (dmrg2d.TF32, dmrg2d.BF16) and not info["tc_ok"]:
        raise RuntimeError("tensor-core path unavailable for this workload")
    in_dt = {dmrg2d.FP64: torch.float64, dmrg2d.FP32: torch.float32, dmrg2d.TF32: torch.float32,
             dmrg2d.BF16: torch.bfloat16}[prec]
    out_dt = torch.float64 if prec == dmrg2d.FP64 else torch.float32
    v_np = synth.start_vector(n, 12 + rank)
    if pad is not None:
        v_np[pad] = 0.0   # padding rows of a sector layout are zero on input
    v_host = torch.from_numpy(v_np).to(in_dt)
    v = v_host.to(dev)
    y = torch.empty(n, dtype=out_dt, device=dev)
    stream = torch.cuda.current_stream()
    tune = None
    if prec in (dmrg2d.TF32, dmrg2d.BF16) and args.tile_config is not None:
        dmrg2d.set_tile_config(ops, prec, args.tile_config)
        tune = {"chosen": args.tile_config, "name": dmrg2d.tile_config_name(args.tile_config),
                "ms": None}
    elif prec in (dmrg2d.TF32, dmrg2d.BF16):
        # tile configuration chosen by the library's autotuner (outside the timed region)
        best, tms = dmrg2d.autotune(ops, prec)
        tune = {"chosen": best, "name": dmrg2d.tile_config_name(best),
                "ms": [round(t, 4) for t in tms]}

    def barrier():
        if world > 1:
            dist.barrier()

    # inputs and outputs larger than L2 (129 MB) need no flush; smaller ones get an L2
    # flush (a 512 MB write) between timed H·v, each H·v timed on its own
    io_bytes = v.numel() * v.element_size() + y.numel() * y.element_size()
    flush = io_bytes < 2 * 129 * 2 ** 20
    l2_note = ("inputs larger than L2 (no flush)" if not flush else
               "L2 flushed (512 MB write) between timed H·v, each timed on its own")
    scratch = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev) if flush else None
    for _ in range(args.warmup):
        dmrg2d.apply_H(ops, v, y, prec)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    dmrg2d.profile_start(ops, args.steps)
    if not flush:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            dmrg2d.apply_H(ops, v, y, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / args.steps
    else:
        evs = []
        for _ in range(args.steps):
            scratch.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dmrg2d.apply_H(ops, v, y, prec)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        step_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    k_ms, k_n = dmrg2d.profile_stop(ops)
    clocks = clk.stop()
    barrier()
    ms = max_over_ranks(step_ms, dev)
    value = job_tflops(flops, ms, world)

    # ---- end to end through the same call: pinned host -> device -> H·v -> host ----
    # Every step uploads its input from pinned host memory, runs dmrg2d_apply_H and reads
    # the result back.  Steps are pipelined the way a caller streams work through the
    # library: uploads on one stream, H·v on another, downloads on a third, two buffer
    # sets, so step i+1's upload and step i-1's download overlap step i's H·v.
    near = bind_near_gpu(local)
    vh = v_host.pin_memory()
    yh = [torch.empty(n, dtype=out_dt).pin_memory() for _ in range(2)]
    # host-link bandwidth alone, one buffer each way (context for the e2e figure)
    link = {}
    for name, (dst, src) in (("h2d_gbs", (v, vh)), ("d2h_gbs", (yh[0], y))):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dst.copy_(src, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        link[name] = src.numel() * src.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9
    vd = [v, torch.empty_like(v)]
    yd = [y, torch.empty_like(y)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_steps(count):
        for i in range(count):
            b = i % 2
            s_in.wait_event(ev_cmp[b])            # vd[b] no longer read by step i-2
            with torch.cuda.stream(s_in):
                vd[b].copy_(vh, non_blocking=True)
            ev_in[b].record(s_in)
            s_cmp.wait_event(ev_in[b])
            s_cmp.wait_event(ev_out[b])           # yd[b] already copied out by step i-2
            dmrg2d.apply_H(ops, vd[b], yd[b], prec, stream=s_cmp)
            ev_cmp[b].record(s_cmp)
            s_out.wait_event(ev_cmp[b])
            with torch.cuda.stream(s_out):
                yh[b].copy_(yd[b], non_blocking=True)
            ev_out[b].record(s_out)

    torch.cuda.synchronize()
    e2e_steps(2)
    torch.cuda.synchronize()
    barrier()
    ke = max(4, args.steps // 2)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(s_in)
    e2e_steps(ke)
    for st_ in (s_in, s_cmp):
        s_out.wait_stream(st_)
    e3.record(s_out)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3) / ke, dev)
    e2e = {"value": job_tflops(flops, ms_e2e, world), "unit": "TFLOP/s",
           "h2d_bytes_per_step": vh.numel() * vh.element_size(),
           "d2h_bytes_per_step": yh[0].numel() * yh[0].element_size(),
           "ms_per_step": ms_e2e, "pipelined": "upload / H·v / download on three streams",
           "host_link": link,
           "cpus_bound": f"{len(near[1])} GPU-local CPUs" if near else "unchanged"}
    if near:
        os.sched_setaffinity(0, near[0])

    out_dtype = {dmrg2d.FP64: "f64", dmrg2d.FP32: "f32", dmrg2d.TF32: "tf32",
                 dmrg2d.BF16: "bf16"}[prec]
    # ---- roofline of the dominant kernel ----
    pk = peaks()
    kernel_ms = k_ms / max(k_n, 1)
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    if prec == dmrg2d.BF16:
        peak, pnote = pk.get("bf16_tflops", 1900.0), "measured bf16 (MEASURED_PEAKS.json)"
        bound = "tensor"
    elif prec == dmrg2d.TF32:
        peak = pk.get("bf16_tflops", 1900.0) * 1.1 / 2.25
        pnote = "measured bf16 x nominal tf32/bf16 ratio 1.1/2.25"
        bound = "tensor"
    elif prec == dmrg2d.FP64:
        peak, pnote, bound = 1.25, "nominal GB300 FP64 1.25 TFLOP/s", "alu"
    else:
        peak, pnote, bound = 2 * 152 * 128 * 2.07e9 / 1e12, "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz", "alu"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (ncu_traffic(tune["name"], out_dtype)
                        if tune and args.workload == WORKLOAD else None),
            "peak_source": pnote,
            "kernel_ms": kernel_ms, "kernel_launches": k_n}

    out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": out_dtype,
           "data": "synthetic (seeded blocks and vector, numpy default_rng)",
           "config": {"workload": args.workload, **wl_config,
                      "n_vec": n, "flops_per_hv": flops, "parallelism": f"replicas{world}",
                      "l2": l2_note, "tile_config": tune},
           "clocks": clocks, "e2e": e2e,
           "gpu_launches": k_n * kernels_per_hv(tune, prec, target is not None),
           "roofline": roof}

    if args.tte and rank == 0 and prec != dmrg2d.FP64:
        out["time_to_energy"] = time_to_energy(ops, n, prec, args, dev)
    if prec == dmrg2d.FP64 and rank == 0:   # the small superblock: latency per H·v and step
        out["latency"] = {"us_per_hv": ms * 1e3, **lanczos_latency(ops, n, dev)}
    if args.link_probe and rank == 0:
        out["host_link_probe"] = link_probe(dev)
    if args.other_workloads and rank == 0 and world == 1 and args.workload == WORKLOAD:
        out["other_workloads"] = other_workloads(args, dev)
    if args.sweep and rank == 0:
        out["dmrg_sweep"] = dmrg_sweep_run(args)
    if args.sweep_profile and rank == 0:
        out["dmrg_sweep_kernel_profile"] = sweep_kernel_profile(args)
    if args.precond_study and rank == 0:
        out["precond_study"] = precond_study(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(seconds=float(args.ref_seconds),
                                           workload=args.workload)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


SWEEP_LATTICES = {
    # name: (model, columns, sector filling, default --sweep-m, description)
    "heisenberg4x12": (lambda synth: synth.model("heisenberg", 4, J_leg=1.0, J_rung=1.0), 12,
                       {}, "128,512,512,1024,1024",
                       "4x12 open Heisenberg ladder, J=1, S^z_tot = 0 sector"),
    # the paper's Fig. 3b system: 3 x 10 Hubbard ladder, U/t = 10, 14 up + 14 down
    "hubbard3x10": (lambda synth: synth.model("hubbard", 3, t=1.0, U=10.0), 10,
                    {"n_up": 14, "n_dn": 14}, "128,256,256",
                    "3x10 open Hubbard ladder, t=1, U=10, (N_up, N_dn) = (14, 14)"),
}


def dmrg_sweep_run(args):
    """The DMRG sweep around the path on --sweep-lattice (default: the 4 x 12 open
    Heisenberg ladder, J = 1, in the S^z_tot = 0 sector; or the 3 x 10 Hubbard ladder at
    U = 10 with 14 + 14 electrons), warm-up with --sweep-m-warmup states, then finite
    sweeps with the --sweep-m schedule, superblock ground states in --precision with FP64
    refinement; energies per sweep, the time split and the observables of the last sweep."""
    from paper_0707_0159_gb300 import dmrg2d, synth
    build, L, filling, m_default, desc = SWEEP_LATTICES[args.sweep_lattice]
    mdl = build(synth)
    ms = [int(m) for m in (args.sweep_m or m_default).split(",")]
    prec = args.sweep_precision or args.precision
    net = dmrg2d.MLP(hidden=256, seed=7) if args.sweep_precond == "mlp" else None
    out = dmrg2d.sweep(mdl, L, m_warmup=args.sweep_m_warmup, m_sweeps=ms,
                       precision=prec, tol=1e-9, max_iter=600, krylov_dim=80,
                       sectors=True, solver=args.sweep_solver, precond=args.sweep_precond,
                       mlp=net, mlp_train_sweeps=args.sweep_mlp_train_sweeps,
                       mlp_epochs=args.sweep_mlp_epochs, **filling)
    e, sw = out["energy"], out["sweep"]
    per = {str(s): min(e[i] for i in range(len(e)) if sw[i] == s) for s in sorted(set(sw))}
    last = max(sw)
    # leg-bond energies between lattice columns x and x + 1 along the last sweep (the
    # paper's h(x, y) profile), and <S_tot^2> at the end of each sweep (Lieb-Mattis)
    profile = {}
    for i in range(len(e)):
        if sw[i] == last:
            profile[str(out["l"][i])] = out["leg_bond"][i]
    s2 = {str(sw[i]): out["s2"][i] for i in range(len(e)) if out["s2"][i] == out["s2"][i]}
    extra = {}
    if filling:
        # hole density h(x, y) and S(x) of the central columns x = l, l + 1 of each step of
        # the last sweep (the paper's Hubbard observables; the end columns are never central)
        hole, smax = {}, {}
        for i in range(len(e)):
            if sw[i] == last:
                for c in range(2):
                    x = str(out["l"][i] + c)
                    hole[x] = [float(v) for v in out["h"][i][c]]
                    smax[x] = float(out["S"][i][c])
        extra = {"hole_density_last_sweep": hole, "S_last_sweep": smax}
    return {"lattice": desc, **extra,
            "m_warmup": args.sweep_m_warmup, "m_sweeps": ms,
            "precision": prec, "solver": args.sweep_solver,
            "precond": args.sweep_precond if args.sweep_solver == "davidson" else None,
            "mlp_train_sweeps": args.sweep_mlp_train_sweeps if net is not None else None,
            "steps": out["n_steps"],
            "energy_min_per_sweep": per, "energy_last": e[-1], "max_trunc": max(out["trunc"]),
            "max_trunc_per_sweep": {str(s_): max(out["trunc"][i] for i in range(len(e))
                                                  if sw[i] == s_) for s_ in sorted(set(sw))},
            "solver_steps": sum(out["iters"]),
            "solver_steps_per_sweep": {str(s_): sum(out["iters"][i] for i in range(len(e))
                                                    if sw[i] == s_) for s_ in sorted(set(sw))},
            "seconds": out["seconds"], "train_seconds": out["train_seconds"],
            "transform_seconds": out["transform_seconds"],
            "solve_seconds": out["solve_seconds"], "build_seconds": out["build_seconds"],
            "density_matrix_seconds": out["dm_seconds"], "renorm_seconds": out["renorm_seconds"],
            "observables_seconds": out["obs_seconds"], "s2_per_sweep": s2,
            **({} if filling else {"leg_bond_profile_last_sweep": profile})}


def link_probe(dev):
    """Host-link bandwidth with 1 GiB pinned buffers: host to device, device to host, and
    both at once, each copy split into 1, 2, 4 or 8 chunks on separate streams."""
    import torch
    n = 2 ** 28
    h_in = torch.empty(n, dtype=torch.float32).pin_memory()
    h_out = torch.empty(n, dtype=torch.float32).pin_memory()
    d_in = torch.empty(n, dtype=torch.float32, device=dev)
    d_out = torch.empty(n, dtype=torch.float32, device=dev)
    streams = [torch.cuda.Stream() for _ in range(8)]

    def run(k, up, down, reps=5):
        ch = n // k
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for i in range(k):
                if up:
                    with torch.cuda.stream(streams[i % 4]):
                        d_in[i * ch:(i + 1) * ch].copy_(h_in[i * ch:(i + 1) * ch],
                                                        non_blocking=True)
                if down:
                    with torch.cuda.stream(streams[4 + i % 4]):
                        h_out[i * ch:(i + 1) * ch].copy_(d_out[i * ch:(i + 1) * ch],
                                                         non_blocking=True)
        torch.cuda.synchronize()
        return 4 * n / ((time.perf_counter() - t0) / reps) / 1e9

    return {str(k): {"h2d_gbs": run(k, True, False), "d2h_gbs": run(k, False, True),
                     "both_each_gbs": run(k, True, True)} for k in (1, 2, 4, 8)}


def other_workloads(args, dev):
    """H·v of the other workloads on the same GPU (outside the headline's timed region):
    the two sector-restricted m = 1024 superblocks in their precisions (tile configuration
    by the autotuner) and the small FP64 superblock with its Lanczos step latency.  Each
    H·v timed alone by CUDA events; the small one with an L2 flush (512 MB write) before
    each H·v, the large ones with inputs larger than L2."""
    import torch
    from paper_0707_0159_gb300 import dmrg2d, synth
    pk = peaks()
    res = {}
    for name in ("ladder4_heisenberg_d16_m1024_sectors", "ladder3_hubbard_d64_m1024_sectors",
                 "ladder2_heisenberg_d4_m64"):
        build, pname, _ = WORKLOADS[name]
        prec = dmrg2d.PRECISION[pname]
        mdl, left, right, target = build(synth)
        ops = dmrg2d.build_ops(mdl, left, right, target=target)
        n, flops = ops.info["n_vec"], ops.info["flops_per_apply"]
        v_np = synth.start_vector(n, 12)
        if target is not None:
            v_np[dmrg2d.sector_dense_index(ops) < 0] = 0.0
        in_dt = {dmrg2d.FP64: torch.float64, dmrg2d.TF32: torch.float32,
                 dmrg2d.BF16: torch.bfloat16}[prec]
        v = torch.from_numpy(v_np).to(in_dt).to(dev)
        y = torch.empty(n, dtype=torch.float64 if prec == dmrg2d.FP64 else torch.float32,
                        device=dev)
        tune = None
        if prec != dmrg2d.FP64:
            best, _ = dmrg2d.autotune(ops, prec)
            tune = {"chosen": best, "name": dmrg2d.tile_config_name(best)}
        small = prec == dmrg2d.FP64
        scratch = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev) if small else None
        for _ in range(3):
            dmrg2d.apply_H(ops, v, y, prec)
        torch.cuda.synchronize()
        evs = []
        for _ in range(10):
            if small:
                scratch.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dmrg2d.apply_H(ops, v, y, prec)
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
        tf = flops / (ms * 1e-3) / 1e12
        if prec == dmrg2d.BF16:
            peak = pk.get("bf16_tflops", 1900.0)
        elif prec == dmrg2d.TF32:
            peak = pk.get("bf16_tflops", 1900.0) * 1.1 / 2.25
        else:
            peak = 1.25
        res[name] = {"precision": pname, "n_vec": n, "flops_per_hv": flops, "ms_per_hv": ms,
                     "tflops": tf, "frac_of_peak": tf / peak, "tile_config": tune}
        if small:
            res[name]["latency"] = {"us_per_hv": ms * 1e3, **lanczos_latency(ops, n, dev)}
        del ops, v, y, scratch
    return res


def sweep_kernel_profile(args):
    """Where the sweep's device time goes: the 4 x 12 sweep with the --sweep-profile-m
    schedule run once under the CUDA profiler (CUPTI, through torch.profiler), kernels
    grouped by name.  Times under the profiler are not benchmark values: only the shares
    are reported as evidence."""
    from torch.profiler import ProfilerActivity, profile
    from paper_0707_0159_gb300 import dmrg2d, synth
    mdl = synth.model("heisenberg", 4, J_leg=1.0, J_rung=1.0)
    ms = [int(m) for m in args.sweep_profile_m.split(",")]
    prec = args.sweep_precision or args.precision
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        out = dmrg2d.sweep(mdl, 12, m_warmup=args.sweep_m_warmup, m_sweeps=ms,
                           precision=prec, tol=1e-9, max_iter=600, krylov_dim=80, sectors=True)
    rows = []
    for e in prof.key_averages():
        t = getattr(e, "device_time_total", None)
        if t is None:
            t = getattr(e, "cuda_time_total", 0.0)
        if t > 0 and not e.key.startswith("Memcpy") and not e.key.startswith("Memset"):
            rows.append((t, e.count, e.key))
    rows.sort(reverse=True)
    tot = sum(r[0] for r in rows) or 1.0

    def group(name):
        if "sytrd" in name:
            return "cuSOLVER tridiagonalisation (sytrd)"
        if "stedc" in name or "laed" in name or "steqr" in name or "larft" in name \
                or "ormtr" in name or "transpose<sytrd" in name:
            return "cuSOLVER other (eigenvectors, back-transformation)"
        if "d884gemm" in name or "d884syrk" in name or "syherk" in name or "gemm" in name.lower():
            return "cuBLAS FP64 GEMM / SYRK"
        if "hv_" in name:
            return "H·v kernels (this library)"
        if "dmrg2d" in name:
            return "other kernels of this library"
        return "other"
    groups = {}
    for t, c, k in rows:
        g = groups.setdefault(group(k), [0.0, 0])
        g[0] += t
        g[1] += c
    return {"schedule": {"m_warmup": args.sweep_m_warmup, "m_sweeps": ms}, "precision": prec,
            "steps": out["n_steps"], "note": "device time under the CUDA profiler; shares only",
            "groups": {k: {"share": v[0] / tot, "launches": v[1]}
                       for k, v in sorted(groups.items(), key=lambda kv: -kv[1][0])},
            "top_kernels": [{"name": k[:120], "launches": c, "share": t / tot}
                            for t, c, k in rows[:15]]}


def precond_study(args):
    """The learned Davidson preconditioner against Jacobi on the 3-leg Hubbard sector
    superblock (the structure of the m = 1024 workload: blocks of 12 sites, 25 (N_up, N_dn)
    sectors, the 3 x 10 lattice at 15 up + 15 down) at m = --precond-m.  The network (2 hidden
    layers of 256) is trained on logged Jacobi-Davidson steps of seeds 0 .. N-1 (FP64
    Davidson to 1e-10), then both preconditioners run through the mixed Davidson path (TF32
    H·v, FP64 outer loop to ||r|| <= 1e-7 |E|) on the unseen seeds 32 .. 39 from the same
    start vectors (the low-precision Davidson stage to a residual of 1e-3 |E|, above TF32's
    floor): iterations, H·v counts and time to energy of each."""
    import numpy as np
    import torch
    from paper_0707_0159_gb300 import dmrg2d, synth
    dev = torch.device("cuda", 0)
    m = args.precond_m
    case = lambda seed: synth.workload_ladder3_hubbard_sectors(m=m, seed=seed)
    net = dmrg2d.MLP(hidden=256, seed=7)
    rng = np.random.default_rng(11)
    cap, batch, epochs = 40, 8192, 4
    t_train = time.perf_counter()
    losses = []
    for seed in range(args.precond_train):
        mdl, left, right, target = case(seed)
        ops = dmrg2d.build_ops(mdl, left, right, target=target)
        n = ops.info["n_vec"]
        pad = dmrg2d.sector_dense_index(ops) < 0
        v0 = synth.start_vector(n, seed + 100)
        v0[pad] = 0.0
        xl = torch.zeros(cap * n, dtype=torch.float64, device=dev)
        rl = torch.zeros(cap * n, dtype=torch.float64, device=dev)
        x = torch.from_numpy(v0).to(dev)
        e, st, code, thetas = dmrg2d.davidson_ground(ops, x, precond="jacobi", tol=1e-10,
                                                     max_iter=600, log=(cap, xl, rl))
        D = torch.empty(n, dtype=torch.float64, device=dev)
        dmrg2d.diagonal(ops, D)
        steps = min(cap, st["iters"]) - 1
        X = torch.empty(batch * 4, dtype=torch.float32, device=dev)
        w = torch.empty(batch, dtype=torch.float32, device=dev)
        T = torch.empty(batch, dtype=torch.float32, device=dev)
        valid = torch.from_numpy(np.flatnonzero(~pad)).to(dev)
        for _ in range(epochs):
            for k in range(steps):
                idx = valid[torch.from_numpy(rng.integers(0, valid.numel(), batch)).to(dev)]
                dmrg2d.mlp_make_batch(ops, xl[k * n:(k + 1) * n], rl[k * n:(k + 1) * n],
                                      thetas[k], x, D, idx, X, w, T)
                losses.append(net.train_step(X, w, T, 3e-4))
        del xl, rl
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    rows = []
    for seed in range(32, 40):
        mdl, left, right, target = case(seed)
        ops = dmrg2d.build_ops(mdl, left, right, target=target)
        n = ops.info["n_vec"]
        pad = dmrg2d.sector_dense_index(ops) < 0
        v0 = synth.start_vector(n, seed + 100)
        v0[pad] = 0.0
        row = {"seed": seed, "n_vec": n}
        for pre in ("jacobi", "mlp"):
            x = torch.from_numpy(v0).to(dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e, st, code = dmrg2d.davidson_ground(
                ops, x, precond=pre, mlp=net if pre == "mlp" else None, precision="tf32",
                refine=1, tol=1e-3, refine_tol=1e-7, max_iter=400, inner_iter=40, outer_max=40)
            torch.cuda.synchronize()
            row[pre] = {"seconds": time.perf_counter() - t0, "energy": e, "status": code,
                        "iters": st["iters"], "n_hv_low": st["n_hv_low"],
                        "n_hv_fp64": st["n_hv_fp64"], "resid": st["resid"]}
        row["energy_rel_diff"] = abs(row["mlp"]["energy"] - row["jacobi"]["energy"]) / abs(
            row["jacobi"]["energy"])
        rows.append(row)
    tot = {pre: {"iters": sum(r[pre]["iters"] for r in rows),
                 "seconds": sum(r[pre]["seconds"] for r in rows)} for pre in ("jacobi", "mlp")}
    return {"m": m, "train_seeds": args.precond_train, "eval_seeds": [32, 39],
            "train_seconds": t_train, "loss_first": losses[0] if losses else None,
            "loss_last": losses[-1] if losses else None, "per_seed": rows, "total": tot}


def kernels_per_hv(tune, prec, sectors):
    """Kernel launches of one dmrg2d_apply_H: the tensor-core configurations launch one
    kernel, or two with the scalar moves in their own kernel (14..19), or three for the
    segment kernels (22: two passes and the moves); the CUDA-core FP64/FP32 H·v one kernel
    on a dense superblock and two (sub-blocks, moves) on a sector layout."""
    if tune is None:
        return 2 if sectors else 1
    c = tune["chosen"]
    return 3 if c == 22 else (2 if 14 <= c < 20 else 1)


def lanczos_latency(ops, n, dev, steps=200):
    """Plain FP64 Lanczos, fixed steps, from a seeded start: wall time per step (H·v, the
    recurrence, two Gram-Schmidt passes and the tridiagonal eigenpair at the end)."""
    import torch
    from paper_0707_0159_gb300 import dmrg2d, synth
    x = torch.from_numpy(synth.start_vector(n, 2)).to(dev)
    dmrg2d.lanczos_ground(ops, x.clone(), max_iter=steps, krylov_dim=steps, fixed_steps=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e, st, code = dmrg2d.lanczos_ground(ops, x, max_iter=steps, krylov_dim=steps, fixed_steps=1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"steps": steps, "us_per_step": dt / steps * 1e6, "energy": e, "status": code,
            "hv_us_per_step": st["hv_ms"] / steps * 1e3}


def time_to_energy(ops, n, prec, args, dev):
    """Ground energy to a residual of tol*|E| from the same start vector: the mixed
    solver (low-precision H·v + an outer Rayleigh-Ritz loop whose H·v is FP64 emulated
    with float pairs, and again with true FP64 H·v there) and, with --tte-fp64, plain
    FP64 Lanczos."""
    import torch
    from paper_0707_0159_gb300 import dmrg2d, synth
    v0 = torch.from_numpy(synth.start_vector(n, 3)).to(dev)
    res = {"tol_rel_residual": args.tte_tol}
    runs = (("mixed", "fp64x"), ("mixed_fp64_refine", "fp64"))
    for key, rprec in runs:
        x = v0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_mp, st_mp, c_mp = dmrg2d.lanczos_ground(ops, x, precision=prec, refine=1,
                                                  tol=args.tte_tol, inner_iter=300,
                                                  krylov_dim=40, outer_max=40,
                                                  refine_precision=rprec)
        torch.cuda.synchronize()
        res[key] = {"precision": args.precision, "refine_precision": rprec,
                    "seconds": time.perf_counter() - t0, "energy": e_mp, "status": c_mp, **st_mp}
    e_mp = res["mixed"]["energy"]
    if args.tte_fp64:
        # the plain FP64 method: thick-restart Lanczos, FP64 H·v and FP64 vectors throughout
        x = v0.clone()
        clk = Clocks(dev.index or 0)
        clk.start()
        t0 = time.perf_counter()
        e64, st64, c64 = dmrg2d.lanczos_ground(ops, x, precision=dmrg2d.FP64, tol=args.tte_tol,
                                               max_iter=args.tte_fp64_max_iter,
                                               krylov_dim=args.tte_fp64_kdim,
                                               thick_keep=args.tte_fp64_keep, check_every=5)
        torch.cuda.synchronize()
        res["fp64"] = {"seconds": time.perf_counter() - t0, "energy": e64, "status": c64,
                       "method": f"thick-restart Lanczos, krylov_dim {args.tte_fp64_kdim}, "
                                 f"{args.tte_fp64_keep} Ritz vectors kept", **st64,
                       "clocks": clk.stop()}
        res["energy_rel_diff"] = abs(e_mp - e64) / abs(e64)
        res["speedup"] = res["fp64"]["seconds"] / res["mixed"]["seconds"]
        if args.tte_ref_tol > 0:
            # the same FP64 solve continued from its own vector to a tighter residual: the
            # reference energy both solvers are compared with (not part of either time)
            t0 = time.perf_counter()
            e_ref, st_ref, c_ref = dmrg2d.lanczos_ground(
                ops, x, precision=dmrg2d.FP64, tol=args.tte_ref_tol,
                max_iter=args.tte_fp64_max_iter, krylov_dim=args.tte_fp64_kdim,
                thick_keep=args.tte_fp64_keep, check_every=5)
            torch.cuda.synchronize()
            res["fp64_reference"] = {"seconds": time.perf_counter() - t0, "energy": e_ref,
                                     "status": c_ref, **st_ref}
            res["mixed_vs_reference_rel"] = {k: abs(res[k]["energy"] - e_ref) / abs(e_ref)
                                             for k in ("mixed", "mixed_fp64_refine", "fp64")
                                             if k in res}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="synthetic superblock (default: the dense 3-leg Hubbard, m = 256)")
    ap.add_argument("--precision", default=os.environ.get("DMRG2D_BENCH_PREC"),
                    choices=["tf32", "bf16", "fp32", "fp64"],
                    help="H·v precision (default: the workload's)")
    ap.add_argument("--tte", action="store_true", default=True,
                    help="time the mixed-precision ground-state solve (default on)")
    ap.add_argument("--no-tte", dest="tte", action="store_false")
    ap.add_argument("--tte-fp64", action="store_true", help="with --tte: also the plain FP64 solve")
    ap.add_argument("--tte-tol", type=float, default=1e-7)
    ap.add_argument("--tte-fp64-max-iter", type=int, default=3000)
    ap.add_argument("--tte-fp64-kdim", type=int, default=48,
                    help="plain FP64 Lanczos: basis vectors before a thick restart")
    ap.add_argument("--tte-fp64-keep", type=int, default=12,
                    help="plain FP64 Lanczos: Ritz vectors kept at a thick restart")
    ap.add_argument("--tte-ref-tol", type=float, default=1e-10,
                    help="with --tte-fp64: continue the FP64 solve to this residual for the "
                         "reference energy (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true", help="also run the DMRG sweep (4 x 12 ladder)")
    ap.add_argument("--sweep-lattice", default="heisenberg4x12", choices=sorted(SWEEP_LATTICES))
    ap.add_argument("--sweep-m", default=None,
                    help="states kept per finite sweep (default: the lattice's schedule)")
    ap.add_argument("--sweep-m-warmup", type=int, default=128)
    ap.add_argument("--sweep-precision", default=None, choices=["tf32", "bf16", "fp64"],
                    help="ground-state H·v precision of the sweep (default: --precision)")
    ap.add_argument("--other-workloads", action="store_true", default=True,
                    help="also time the sector-restricted and small workloads' H·v (default "
                         "on, with the default workload at N = 1)")
    ap.add_argument("--no-other-workloads", dest="other_workloads", action="store_false")
    ap.add_argument("--link-probe", action="store_true",
                    help="also measure the host link (one way and both ways, chunked copies)")
    ap.add_argument("--sweep-profile", action="store_true",
                    help="also run the sweep once under the CUDA profiler: kernel shares")
    ap.add_argument("--sweep-profile-m", default="128,1024",
                    help="states kept per finite sweep in the profiled run")
    ap.add_argument("--sweep-solver", default="lanczos", choices=["lanczos", "davidson"])
    ap.add_argument("--sweep-precond", default="jacobi", choices=["none", "jacobi", "mlp"],
                    help="Davidson preconditioner of the sweep (mlp: trained in the sweep)")
    ap.add_argument("--sweep-mlp-train-sweeps", type=int, default=1,
                    help="the warm-up and sweeps below this index train the network")
    ap.add_argument("--sweep-mlp-epochs", type=int, default=2)
    ap.add_argument("--precond-study", action="store_true",
                    help="also train and evaluate the learned Davidson preconditioner")
    ap.add_argument("--precond-m", type=int, default=256)
    ap.add_argument("--precond-train", type=int, default=32)
    ap.add_argument("--tile-config", type=int, default=None,
                    help="tensor-core tile configuration index instead of the autotuner")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.precision is None:
        args.precision = WORKLOADS[args.workload][1]
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
