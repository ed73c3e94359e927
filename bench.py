"""Benchmark of the Galerkin-assembly hot path on one GB300 (or N replicas).

Step = one pass of the hot path over the 2D diffusion workload (P1
triangles, 1024 x 1024 jittered grid, Hilbert element order, lognormal kappa
at 3 points per element, c = 1, f ~ U(-1, 1) per node; 2,097,152 elements),
FP32: the linear system in one pass (stiffness CSR values and load vector,
fused Map + deterministic Reduce), and the backward assembly for an upstream
gradient of the values (grad kappa, grad coords, grad c).  Inputs live in HBM before timing; L2 is
flushed between steps (outside the per-step CUDA events).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload instead.  Under torchrun every rank runs its own
replica (no data-path collective: weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import meshgen as mg  # noqa: E402

METRIC = "elements assembled/sec and achieved HBM GB/s (fwd, fwd+bwd, batched vs looped)"
WORKLOAD = ("2D diffusion, P1 triangles, 1024x1024 grid jittered +-0.2h, Hilbert element order, "
            "kappa lognormal at 3 points per element, c=1, f~U(-1,1) per node")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / elasticity / batched breakdown")
    ap.add_argument("--extras-only", choices=["diffusion", "residual", "facets", "batch", "elasticity", "small"],
                    default=None,
                    help="run only this part of the breakdown (short runs, e.g. for profiling one kernel)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_max(x, world, device):
    """The maximum of a per-rank scalar over all ranks (the slowest replica's
    time); x itself on a single rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, ms_max):
    """Whole-job throughput of N independent replicas: every rank's units over
    the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------------ workload
def workload(n=1024):
    cfg = mg.diffusion2d(n)
    m = cfg["mesh"]
    return m, cfg


def alg_bytes(kind, E, N, nnz, s, nv=3, Q=3, d=2):
    """Compulsory bytes: read cells, coords and coefficients once, write outputs once."""
    if kind == "fwd":
        return E * nv * 4 + N * d * s + E * Q * s + nnz * s
    if kind == "system":  # forward and load together: cells and coords read once
        return E * nv * 4 + N * d * s + E * Q * s + N * s + nnz * s + N * s
    if kind == "load":
        return E * nv * 4 + N * d * s + N * s + N * s
    if kind == "bwd":
        return E * nv * 4 + N * d * s + E * Q * s + nnz * s + E * Q * s + N * d * s
    if kind == "residual":  # read cells, coords, kappa, x, f, the Dirichlet mask; write y
        return E * nv * 4 + N * d * s + E * Q * s + N * s + N * s + N + N * s
    if kind == "residual_bwd":  # dL/dx = K g, then the adjoint backward (lam = g, U = x) and the load backward
        return (E * nv * 4 + N * d * s + E * Q * s + N * s + N + N * s  # K g
                + E * nv * 4 + N * d * s + E * Q * s + 2 * N * s + E * Q * s + N * d * s  # kappa, coords
                + E * nv * 4 + N * d * s + 2 * N * s + N * d * s)  # f, coords (accumulated)
    if kind == "elastic":
        return E * 4 * 4 + N * 3 * s + 2 * E * s + nnz * s
    if kind == "elastic_bwd":  # + read grad_vals, write grad_lam, grad_mu, grad_coords
        return E * 4 * 4 + N * 3 * s + 2 * E * s + nnz * s + 2 * E * s + N * 3 * s
    raise ValueError(kind)


# Algorithmic floating-point operations per element of the minimal
# formulation of each assembly (an FMA counts as two, a division as one; the
# counts are derived in the design notes): the roof that FP64 runs meet on
# the FP64 pipe, next to the HBM roof.
ALU_FLOPS = {"fwd": 46, "system": 55, "bwd": 111, "elastic": 453}


def two_roofs(ms, bytes_, flops, hbm_gbs, fp64_flops):
    """Achieved fractions of the HBM roof, of the FP64 ALU roof, and of the
    lower of the two (the binding bound: max of the two times over the
    measured time)."""
    t_hbm = bytes_ / (hbm_gbs * 1e9)
    t_alu = flops / fp64_flops
    t = ms * 1e-3
    return {"hbm_frac": t_hbm / t, "alu_frac": t_alu / t, "frac_min_roof": max(t_hbm, t_alu) / t,
            "flops_per_launch": flops, "alu_tflops": flops / t / 1e12, "bound": "alu" if t_alu > t_hbm else "hbm"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# translation units and headers each timed kernel is built from
_FWD_SRC = ["forward.cu", "fan.cuh", "blk_bilinear.cuh", "gather.cuh", "elements.cuh", "blocks.cuh", "async.cuh",
            "tg_internal.cuh"]
KERNEL_SOURCES = {
    "system": _FWD_SRC, "fwd": _FWD_SRC, "load": _FWD_SRC,
    "bwd": ["backward.cu", "fan.cuh", "blk_bilinear.cuh", "gather.cuh", "elements.cuh", "blocks.cuh", "async.cuh",
            "tg_internal.cuh"],
}


def source_hash(kernel_key):
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2602_05052_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES[kernel_key]):
        p = os.path.join(cs, f)
        if os.path.exists(p):
            with open(p, "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """DRAM bytes (read + write) per launch from the committed ncu summary, or
    None when the kernel's sources changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    k = d.get("kernels", {}).get(kernel_key)
    if k is None or k.get("source_hash") != source_hash(kernel_key):
        return None
    return k.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ the CPU oracle
def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_model():
    """The host CPU's model name as lscpu reports it (None if unavailable)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return None
    for line in out.splitlines():
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    return None


def f32_host(a):
    """An input as the FP32 GPU run reads it, promoted back to FP64 for the oracle."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def oracle_for(m, cfg, threads, G=None):
    """The chunked FP64 oracle on the workload with FP32-rounded inputs (the
    inputs of the FP32 GPU run), so one oracle pass serves both the CPU
    timing and the FP32 error; G the upstream gradient of the values."""
    from oracle.chunked import ChunkedOracle
    return ChunkedOracle(m.cells, f32_host(m.coords), f32_host(cfg["kappa"]), f32_host(cfg["f"]), cfg["c"], threads,
                         seed=1, G=G)


def time_oracle(orc, reps):
    """Seconds per pass of the oracle over its workload (after one untimed
    pass), and that pass's results."""
    res = orc.step()
    t0 = time.perf_counter()
    for _ in range(reps):
        orc.step()
    return (time.perf_counter() - t0) / reps, res


def run_reference(args):
    """The reference arm: the FP64 oracle on all host cores (elements in
    contiguous chunks, one process each, partial results added in chunk
    order), a full pass over the workload per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    m, cfg = workload()
    cores = host_cores()
    orc = oracle_for(m, cfg, cores)
    try:
        for _ in range(max(args.warmup, 1)):
            orc.step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            orc.step()
        dt = time.perf_counter() - t0
    finally:
        orc.close()
    v = m.n_elems * args.steps / dt
    sample = (f"each step: the full workload ({m.n_elems} elements, {m.n_nodes} nodes); forward DOK scatter-add, "
              f"load and backward by the FP64 oracle in {cores} processes of contiguous element chunks, partial "
              f"results added in chunk order")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": m.n_elems, "nodes": m.n_nodes},
        "cpu_baseline": {"value": v, "unit": "elements/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    import paper_2602_05052_gb300 as tg
    from paper_2602_05052_gb300 import build
    build.build_library()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    barrier = lambda: replica_barrier(world)
    max_over_ranks = lambda x: replica_max(x, world, dev)

    dt = torch.float32
    s = 4
    m, cfg = workload()
    E, N = m.n_elems, m.n_nodes
    d = lambda a, t=dt: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
    p = tg.tg_build_pattern(d(m.cells, torch.int32), N, tg.P1_TRI)
    nnz = p.nnz
    coords, kappa, f = d(m.coords), d(cfg["kappa"]), d(cfg["f"])
    gvals = d(np.random.default_rng(1).normal(size=nnz))
    vals = torch.empty(nnz, dtype=dt, device=dev)
    F = torch.empty(N, dtype=dt, device=dev)
    gk, gx, gc = torch.empty_like(kappa), torch.empty_like(coords), torch.empty(1, dtype=dt, device=dev)
    flush = L2Flush(torch, dev)
    c = cfg["c"]

    def step(ev=None):
        if ev:
            ev[0].record()
        # the linear system (K, F) in one pass: fused Map + Reduce of both
        tg.tg_assemble_system(p, coords, kappa, tg.PER_QP, c, f, tg.PER_NODE, vals=vals, F=F)
        if ev:
            ev[1].record()
        tg.tg_assemble_backward(p, coords, kappa, tg.PER_QP, c, grad_vals=gvals, grad_kappa=gk, grad_coords=gx,
                                grad_c=gc)
        if ev:
            ev[2].record()

    launches_per_step = 2  # system (K and F in one kernel), backward (its global sums finish in-kernel)
    for _ in range(max(args.warmup, 3)):
        flush()
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush()
            step(evs[k])
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - w0
    clocks = clk.summary()
    t_sys = [e[0].elapsed_time(e[1]) for e in evs]
    t_bwd = [e[1].elapsed_time(e[2]) for e in evs]
    t_step = [a + b for a, b in zip(t_sys, t_bwd)]
    ms = max_over_ranks(sum(t_step) / args.steps)
    value = replica_throughput(E, world, ms)
    st, bad = tg.tg_get_device_status(p)
    if st != 0:
        raise RuntimeError(f"device status {st} at element {bad}")

    peak, peak_src = load_peaks()
    kern = {"system": (statistics.mean(t_sys), alg_bytes("system", E, N, nnz, s)),
            "bwd": (statistics.mean(t_bwd), alg_bytes("bwd", E, N, nnz, s))}
    dom = max(kern, key=lambda k: kern[k][0])
    names = {"system": "k_bilinear_fan<float,UB,load>", "bwd": "k_backward_fan<float,gvals,UB>"}
    ach = kern[dom][1] / (kern[dom][0] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": ncu_traffic(dom), "peak_source": f"{peak_src} (copy, burst)",
                "algorithmic_bytes_per_launch": kern[dom][1]}
    per_kernel = {k: {"ms": v[0], "alg_GBps": v[1] / (v[0] * 1e-3) / 1e9, "frac_of_peak": v[1] / (v[0] * 1e-3) / 1e9 / peak,
                      "elements_per_s": E / (v[0] * 1e-3)} for k, v in kern.items()}

    # ---------------- the same step, median of 30, and with the outputs' write-back inside the events
    # The L2 flush between steps only reads, so a timed step ends with its
    # outputs still dirty in L2.  A second read of the flush buffer right
    # after the step, inside the events, evicts them (their write-back lands
    # there); the same read timed alone on a clean L2 is subtracted.
    def median_of(n, evict):
        ts = []
        for _ in range(n):
            flush()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            step()
            if evict:
                flush(spin_us=0)
            a1.record()
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        return statistics.median(ts)

    def evict_alone(n):
        ts = []
        for _ in range(n):
            flush()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            flush(spin_us=0)
            a1.record()
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        return statistics.median(ts)

    ms_med = max_over_ranks(median_of(30, False))
    ms_wb = max_over_ranks(median_of(30, True) - evict_alone(30))

    # ---------------- end to end: pinned host inputs -> C-ABI calls -> host results
    # Every step copies all of its inputs host -> device and all of its
    # outputs device -> host.  Steps are pipelined over two device buffer
    # sets and three streams (copy in, compute, copy out), so that one step's
    # copies overlap the neighbouring steps' work; the dependencies (events)
    # keep each buffer set's reuse ordered.
    names_in, names_out = ("coords", "kappa", "f", "gvals"), ("vals", "F", "gk", "gx", "gc")
    dev_in = [[coords, kappa, f, gvals], [t.clone() for t in (coords, kappa, f, gvals)]]
    dev_out = [[vals, F, gk, gx, gc], [torch.empty_like(t) for t in (vals, F, gk, gx, gc)]]
    h_in = [t.cpu().pin_memory() for t in (coords, kappa, f, gvals)]
    h_out = [[torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in dev_out[0]] for _ in range(2)]
    bi = sum(t.numel() * t.element_size() for t in h_in)
    bo = sum(t.numel() * t.element_size() for t in h_out[0])
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "cmp", "out")}
    started = [False, False]

    def e2e_step(k):
        b = k % 2
        ci, cd, ho = dev_in[b], dev_out[b], h_out[b]
        with torch.cuda.stream(s_in):
            if started[b]:
                s_in.wait_event(ev["cmp"][b])  # the last compute on this set has read its inputs
            for hd, dd in zip(h_in, ci):
                dd.copy_(hd, non_blocking=True)
            ev["in"][b].record(s_in)
        s_cmp.wait_event(ev["in"][b])
        if started[b]:
            s_cmp.wait_event(ev["out"][b])  # the last copy-out of this set is done
        tg.tg_assemble_system(p, ci[0], ci[1], tg.PER_QP, c, ci[2], tg.PER_NODE, vals=cd[0], F=cd[1], stream=s_cmp)
        tg.tg_assemble_backward(p, ci[0], ci[1], tg.PER_QP, c, grad_vals=ci[3], grad_kappa=cd[2], grad_coords=cd[3],
                                grad_c=cd[4], stream=s_cmp)
        ev["cmp"][b].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev["cmp"][b])
            for hd, dd in zip(ho, cd):
                hd.copy_(dd, non_blocking=True)
            ev["out"][b].record(s_out)
        started[b] = True

    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(args.steps):
        e2e_step(k)
    e1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    # the results read back equal the device-resident run's
    e2e_ok = bool(torch.equal(h_out[(args.steps - 1) % 2][0], vals.cpu()))

    out = {"metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "elements": E, "nodes": N, "nnz": nnz,
                      "step": "system (K values and load vector F in one pass) + backward (grad kappa, grad "
                              "coords, grad c) for an upstream gradient of the values",
                      "l2": "flushed between steps by reading a 512 MB buffer (leaves L2 clean), outside the "
                            "per-step CUDA events",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "ms_per_step_median30": ms_med, "value_median30": replica_throughput(E, world, ms_med),
           "ms_per_step_with_writeback": ms_wb,
           "writeback_how": "median of 30 steps, each followed inside its events by a 512 MB read that evicts the "
                            "step's outputs from L2 (their DRAM write-back included), minus the median of 30 such "
                            "reads alone on a clean L2",
           "wall_s_timed_region": wall, "gpu_launches": launches_per_step * args.steps,
           "roofline": roofline, "kernels": per_kernel,
           "e2e": {"value": replica_throughput(E, world, e2e_ms), "unit": "elements/s", "h2d_bytes_per_step": bi,
                   "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms, "results_match_device_run": e2e_ok,
                   "how": "pinned host buffers; per step all inputs copied in and all outputs copied out; steps "
                          "pipelined over two device buffer sets on copy-in, compute and copy-out streams"},
           "clocks": clocks}

    if args.extras_only and rank == 0:
        if args.extras_only == "diffusion":
            out["breakdown"] = diffusion_extras(tg, torch, dev, m, cfg, p, peak, flush)
        elif args.extras_only == "residual":
            out["breakdown"] = residual_extras(tg, torch, dev, m, cfg, p, peak, flush)
        elif args.extras_only == "facets":
            out["breakdown"] = facet_extras(tg, torch, dev, m, p, flush)
        elif args.extras_only == "elasticity":
            out["breakdown"] = elasticity_extras(tg, torch, dev, peak, flush)
        elif args.extras_only == "small":
            out["breakdown"] = small_configs(tg, torch, dev)
        else:
            out["breakdown"] = batch_extras(tg, torch, dev, peak, flush)
    elif not args.no_extras and rank == 0:
        out["breakdown"] = extras(tg, torch, dev, m, cfg, p, peak, flush)
    for k in list(out.get("breakdown", {})):
        if k.startswith("fp32_err_"):
            out.setdefault("fp32_err", {})[k[len("fp32_err_"):]] = out["breakdown"].pop(k)
    if not args.no_cpu_baseline and rank == 0:
        # the FP64 oracle on the FP32-rounded inputs of this run: its timing
        # on all host cores and on one, and the FP32 error of the step
        G = f32_host(np.random.default_rng(1).normal(size=nnz))
        cores = host_cores()
        orc = oracle_for(m, cfg, cores, G)
        try:
            sec_n, (rv, rF, rk, rx, rc) = time_oracle(orc, 3)
        finally:
            orc.close()
        orc = oracle_for(m, cfg, 1, G)
        try:
            sec_1, _ = time_oracle(orc, 1)
        finally:
            orc.close()
        step()
        torch.cuda.synchronize()
        rel = lambda got, want: float(np.linalg.norm(np.asarray(got, np.float64).ravel() - np.ravel(want))
                                      / np.linalg.norm(np.ravel(want)))
        out.setdefault("fp32_err", {})["diffusion2d_1024"] = {
            "vals": rel(vals.cpu().numpy(), rv), "F": rel(F.cpu().numpy(), rF),
            "grad_kappa": rel(gk.cpu().numpy(), rk), "grad_coords": rel(gx.cpu().numpy(), rx),
            "grad_c": rel(gc.cpu().numpy(), [rc]),
            "how": "relative Frobenius error of the step's FP32 outputs against the FP64 oracle fed the same "
                   "FP32-rounded inputs, every entry"}
        out["cpu_baseline"] = {
            "value": E / sec_n, "unit": "elements/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"the full workload ({E} elements: forward DOK scatter-add, load, backward), FP64, in {cores} "
                      f"processes of contiguous element chunks with partial results added in chunk order; mean of "
                      f"3 passes ({sec_n:.2f} s each)",
            "single_core": {"value": E / sec_1, "cores": 1,
                            "sample": f"the same pass in one process, 1 pass ({sec_1:.2f} s)"}}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


class L2Flush:
    """Evict L2 by reading a buffer 4x its size: the evicted lines (the last
    step's outputs) are written back here, outside the timed events, and the
    cache is left holding clean lines only."""

    def __init__(self, torch, dev, mb=512):
        self.buf = torch.ones(mb * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        self.acc = torch.empty((), dtype=torch.float32, device=dev)
        self.torch = torch

    def __call__(self, spin_us=400):
        self.torch.sum(self.buf, dim=0, out=self.acc)
        # Keep the GPU busy while the host enqueues the timed calls, so the
        # start event is not followed by idle time waiting for the launch.
        if spin_us:
            self.torch.cuda._sleep(int(spin_us * 2000))


def timed(torch, fn, flush, reps=10, warm=3, spin_us=400):
    """Median of per-call CUDA-event times, L2 flushed before each call (and
    the GPU kept busy for spin_us while the host enqueues the call)."""
    for _ in range(warm):
        flush()
        fn()
    ts = []
    for _ in range(reps):
        flush(spin_us)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def extras(tg, torch, dev, m, cfg, p, peak, flush):
    """Breakdown: FP64, atomic comparison, elasticity, batched vs looped."""
    out = diffusion_extras(tg, torch, dev, m, cfg, p, peak, flush)
    fp64 = out["fp64_fma_peak_tflops"] * 1e12
    out.update(residual_extras(tg, torch, dev, m, cfg, p, peak, flush))
    out.update(facet_extras(tg, torch, dev, m, p, flush))
    out.update(elasticity_extras(tg, torch, dev, peak, flush, fp64))
    out.update(batch_extras(tg, torch, dev, peak, flush))
    out.update(small_configs(tg, torch, dev))
    return out


def diffusion_extras(tg, torch, dev, m, cfg, p, peak, flush):
    """The 2D diffusion kernels one by one in FP32 and FP64 (forward, atomic
    comparison, backward, load, system), with the FP64 ALU roof."""
    out = {}
    E, N, nnz = m.n_elems, m.n_nodes, p.nnz
    fp64 = tg.tg_diag_fma_rate(torch.float64)
    out["fp64_fma_peak_tflops"] = fp64 / 1e12
    out["fp32_fma_peak_tflops"] = tg.tg_diag_fma_rate(torch.float32) / 1e12
    for dtn, dt, s in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        d = lambda a, t=dt: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
        x, k, f = d(m.coords), d(cfg["kappa"]), d(cfg["f"])
        v = torch.empty(nnz, dtype=dt, device=dev)
        gv = d(np.random.default_rng(1).normal(size=nnz))
        ms_f = timed(torch, lambda: tg.tg_assemble_bilinear(p, x, k, tg.PER_QP, 1.0, v), flush)
        ms_a = timed(torch, lambda: tg.tg_assemble_bilinear_atomic(p, x, k, tg.PER_QP, 1.0, v), flush)
        ms_b = timed(torch, lambda: tg.tg_assemble_backward(p, x, k, tg.PER_QP, 1.0, grad_vals=gv), flush)
        ms_l = timed(torch, lambda: tg.tg_assemble_load(p, x, f, tg.PER_NODE), flush)
        F_ = torch.empty(N, dtype=dt, device=dev)
        ms_s = timed(torch, lambda: tg.tg_assemble_system(p, x, k, tg.PER_QP, 1.0, f, tg.PER_NODE, vals=v, F=F_), flush)
        bf, bb = alg_bytes("fwd", E, N, nnz, s), alg_bytes("bwd", E, N, nnz, s)
        out[f"diffusion2d_{dtn}"] = {
            "fwd_ms": ms_f, "fwd_elements_per_s": E / ms_f * 1e3, "fwd_alg_GBps": bf / ms_f / 1e6,
            "fwd_frac_hbm": bf / ms_f / 1e6 / peak,
            "atomic_fwd_ms": ms_a, "gather_vs_atomic_speedup": ms_a / ms_f,
            "bwd_ms": ms_b, "bwd_alg_GBps": bb / ms_b / 1e6, "bwd_frac_hbm": bb / ms_b / 1e6 / peak,
            "fwd_plus_bwd_elements_per_s": E / (ms_f + ms_b) * 1e3, "load_ms": ms_l,
            "system_ms": ms_s, "system_alg_GBps": alg_bytes("system", E, N, nnz, s) / ms_s / 1e6}
        if dt == torch.float64:
            out[f"diffusion2d_{dtn}"]["roofs"] = {
                "fwd": two_roofs(ms_f, bf, ALU_FLOPS["fwd"] * E, peak, fp64),
                "system": two_roofs(ms_s, alg_bytes("system", E, N, nnz, s), ALU_FLOPS["system"] * E, peak, fp64),
                "bwd": two_roofs(ms_b, bb, ALU_FLOPS["bwd"] * E, peak, fp64),
                "fp64_peak_tflops": fp64 / 1e12}
    return out


def elasticity_extras(tg, torch, dev, peak, flush, fp64=None):
    """Vector P1 elasticity on 64^3 Kuhn tetrahedra: forward and backward for
    an upstream gradient of the values, FP32 and FP64."""
    out = {}
    ce = mg.elasticity3d(64)
    me = ce["mesh"]
    pe = tg.tg_build_pattern(torch.as_tensor(me.cells, device=dev), me.n_nodes, tg.P1_TET_VEC3)
    for dtn, dt, s in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        d = lambda a, t=dt: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
        x, lam, mu = d(me.coords), d(ce["lam"]), d(ce["mu"])
        v = torch.empty(pe.nnz, dtype=dt, device=dev)
        ms_e = timed(torch, lambda: tg.tg_assemble_elasticity(pe, x, lam, mu, tg.PER_ELEMENT, v), flush)
        be = alg_bytes("elastic", me.n_elems, me.n_nodes, pe.nnz, s)
        gv = d(np.random.default_rng(7).normal(size=pe.nnz))
        gl, gm, gx = torch.empty_like(lam), torch.empty_like(mu), torch.empty_like(x)
        ms_eb = timed(torch, lambda: tg.tg_assemble_elasticity_backward(pe, x, lam, mu, tg.PER_ELEMENT, grad_vals=gv,
                                                                        grad_lam=gl, grad_mu=gm, grad_coords=gx), flush)
        bb = alg_bytes("elastic_bwd", me.n_elems, me.n_nodes, pe.nnz, s)
        out[f"elasticity3d_{dtn}"] = {"ms": ms_e, "elements_per_s": me.n_elems / ms_e * 1e3,
                                      "alg_GBps": be / ms_e / 1e6, "frac_hbm": be / ms_e / 1e6 / peak,
                                      "bwd_ms": ms_eb, "bwd_alg_GBps": bb / ms_eb / 1e6,
                                      "bwd_frac_hbm": bb / ms_eb / 1e6 / peak}
        if dt == torch.float64 and fp64:
            out[f"elasticity3d_{dtn}"]["roofs"] = {"fwd": two_roofs(ms_e, be, ALU_FLOPS["elastic"] * me.n_elems,
                                                                    peak, fp64), "fp64_peak_tflops": fp64 / 1e12}
        if dt == torch.float32:
            tg.tg_assemble_elasticity(pe, x, lam, mu, tg.PER_ELEMENT, v)
            out["fp32_err_elasticity3d_64"] = elasticity_sample_err(pe, me, ce, v)
    del pe
    return out


def elasticity_sample_err(pe, me, ce, v, n_rows=2048, seed=12):
    """FP32 error of the elasticity values on sampled node rows: the FP64
    oracle (fed the FP32-rounded inputs) assembles the elements incident to
    2,048 random nodes, which complete those nodes' rows; relative Frobenius
    error over the sampled rows' 3 x 3 blocks."""
    import oracle as O
    g = np.random.default_rng(seed)
    nodes = np.sort(g.choice(me.n_nodes, size=n_rows, replace=False))
    hit = np.isin(me.cells, nodes).any(axis=1)
    R = O.assemble_elasticity(me.cells[hit], f32_host(me.coords), f32_host(ce["lam"][hit]), f32_host(ce["mu"][hit]),
                              O.PER_ELEMENT)
    rows = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    rp = pe.row_ptr.cpu().numpy().astype(np.int64)
    vals = v.cpu().numpy().astype(np.float64)
    got = np.concatenate([vals[rp[r]:rp[r + 1]] for r in rows])
    want = np.concatenate([R.val[R.row_ptr[r]:R.row_ptr[r + 1]] for r in rows])
    return {"vals": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
            "how": f"relative Frobenius error over the complete rows of {n_rows} random nodes (3 DoF rows each, "
                   f"{len(want)} entries) against the FP64 oracle on the elements incident to them, FP32-rounded "
                   f"inputs"}


def batch_extras(tg, torch, dev, peak, flush):
    """Batched P2: 256 instances, one persistent launch against 256 launches
    (plain and graph-captured)."""
    out = {}
    insts = mg.batched_p2(256, seed=4)
    dt = torch.float32
    pats, xs, ks, vs = [], [], [], []
    tot_e = tot_b = 0
    for ins in insts:
        mi = ins["mesh"]
        pi = tg.tg_build_pattern(torch.as_tensor(mi.cells, device=dev), mi.n_nodes, tg.P2_TRI)
        pats.append(pi)
        xs.append(torch.as_tensor(mi.coords, dtype=dt, device=dev))
        ks.append(torch.as_tensor(ins["kappa"], dtype=dt, device=dev))
        vs.append(torch.empty(pi.nnz, dtype=dt, device=dev))
        tot_e += mi.n_elems
        tot_b += alg_bytes("fwd", mi.n_elems, mi.n_nodes, pi.nnz, 4, nv=6, Q=6)
    b = tg.tg_batch_create(pats)
    cs = [0.0] * len(pats)
    tune_ms = tg.tg_batch_autotune(b, xs, ks, tg.PER_QP, cs, vs, reps=3)
    # the host marshals and checks 768 tensors per batched call (about 0.5 ms
    # in Python): a longer spin keeps that out of the device time
    ms_b = timed(torch, lambda: tg.tg_batch_assemble(b, xs, ks, tg.PER_QP, cs, vs), flush, spin_us=2000)

    def looped():
        for pi, xi, ki, vi in zip(pats, xs, ks, vs):
            tg.tg_assemble_bilinear(pi, xi, ki, tg.PER_QP, 0.0, vi)

    ms_l = timed(torch, looped, flush, reps=5)
    g_b, g_l = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g_b, stream=st):
        tg.tg_batch_assemble(b, xs, ks, tg.PER_QP, cs, vs, stream=st)
    with torch.cuda.graph(g_l, stream=st):
        for pi, xi, ki, vi in zip(pats, xs, ks, vs):
            tg.tg_assemble_bilinear(pi, xi, ki, tg.PER_QP, 0.0, vi, stream=st)
    torch.cuda.synchronize()
    ms_bg = timed(torch, g_b.replay, flush)
    ms_lg = timed(torch, g_l.replay, flush)
    ref = [v.clone() for v in vs]
    looped()
    same = all(torch.equal(a, b_) for a, b_ in zip(ref, vs))
    # FP32 error of 8 instances (every 32nd) against the FP64 oracle on their FP32-rounded inputs
    import oracle as O
    num = den = 0.0
    for j in range(0, len(insts), 32):
        mi = insts[j]["mesh"]
        R = O.assemble_bilinear(O.P2_TRI, mi.cells, f32_host(mi.coords), f32_host(insts[j]["kappa"]), O.PER_QP, 0.0)
        got = ref[j].cpu().numpy().astype(np.float64)
        num += float(np.sum((got - R.val) ** 2))
        den += float(np.sum(R.val ** 2))
    out["fp32_err_batched_p2"] = {"vals": (num / den) ** 0.5,
                                  "how": "relative Frobenius error of the batched launch's values of 8 of the 256 "
                                         "instances (every 32nd, all entries) against the FP64 oracle fed the "
                                         "FP32-rounded inputs"}
    out["batched_p2_f32"] = {
        "instances": len(pats), "elements": tot_e, "alg_bytes": tot_b, "schedule": b.schedule(),
        "autotune_best_ms": tune_ms,
        "batched_ms": ms_b, "batched_graph_ms": ms_bg, "looped_ms": ms_l, "looped_graph_ms": ms_lg,
        "batched_elements_per_s": tot_e / ms_b * 1e3, "batched_alg_GBps": tot_b / ms_b / 1e6,
        "batched_frac_hbm": tot_b / ms_b / 1e6 / peak, "speedup_vs_looped": ms_l / ms_b,
        "speedup_vs_looped_graph": ms_lg / ms_bg, "bitwise_equal_to_looped": same}
    del b, pats, xs, ks, vs
    return out


def residual_extras(tg, torch, dev, m, cfg, p, peak, flush):
    """Matrix-free residual y = K x - F and loss ||y||^2 of Eq. (res1) on the
    1024^2 workload (x random, u = 0 rows on the boundary), and its reverse
    mode: dL/dx = K g, dL/dkappa and dL/dcoords (lam = g, U = x), dL/df."""
    out = {}
    E, N = m.n_elems, m.n_nodes
    mask = torch.as_tensor(m.boundary.astype(np.uint8), device=dev)
    for dtn, dt, s in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        d = lambda a, t=dt: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
        X, k, f = d(m.coords), d(cfg["kappa"]), d(cfg["f"])
        x = d(np.random.default_rng(9).uniform(-1, 1, N))
        y, loss = torch.empty(N, dtype=dt, device=dev), torch.empty(1, dtype=dt, device=dev)
        fwd = lambda: tg.tg_residual(p, X, k, tg.PER_QP, 1.0, x, f, tg.PER_NODE, mask, y=y, loss=loss)
        ms = timed(torch, fwd, flush)
        fwd()
        g = 2.0 * y  # dL/dy of L = ||y||^2 (zero on the Dirichlet rows)
        gx_in, gk, gX, gf = (torch.empty_like(x), torch.empty_like(k), torch.empty_like(X), torch.zeros_like(f))
        ng = -g

        def bwd():
            tg.tg_residual(p, X, k, tg.PER_QP, 1.0, g, y=gx_in, loss=False)
            tg.tg_assemble_backward(p, X, k, tg.PER_QP, 1.0, lam=g, U=x, grad_kappa=gk, grad_coords=gX, grad_c=False)
            tg.tg_assemble_load_backward(p, X, f, tg.PER_NODE, 1, ng, grad_f=gf, grad_coords=gX, accumulate=True)

        ms_b = timed(torch, bwd, flush)
        b, bb = alg_bytes("residual", E, N, 0, s), alg_bytes("residual_bwd", E, N, 0, s)
        out[f"residual2d_{dtn}"] = {
            "ms": ms, "elements_per_s": E / ms * 1e3, "alg_GBps": b / ms / 1e6, "frac_hbm": b / ms / 1e6 / peak,
            "bwd_ms": ms_b, "bwd_alg_GBps": bb / ms_b / 1e6, "bwd_frac_hbm": bb / ms_b / 1e6 / peak,
            "loss": float(loss.item()),
            "note": "y = K x - F without storing K, Dirichlet rows zeroed, loss = ||y||^2 in FP64; backward = "
                    "K g (matrix-free) + adjoint backward (lam = g, U = x) + load backward, 3 launches"}
        # Allen-Cahn backward-Euler step residual (method of lines): (1/dt) M (U1 - U0) + a^2 K U1 + N(U1),
        # N the load of eps^2 (u^3 - u); its x-gradient action K g + J(U1) g
        r = [0.0, -0.3, 0.0, 0.3]
        u0 = d(np.random.default_rng(10).uniform(-1, 1, N)) / 1e-3
        a2 = d([0.01])
        ac = lambda: tg.tg_semilinear_residual(p, X, a2, tg.PER_QP if a2.numel() > 1 else tg.CONSTANT, 1e3, x, r, u0,
                                               tg.PER_NODE, dirichlet=mask, y=y, loss=loss)
        ms_ac = timed(torch, ac, flush)
        acj = lambda: tg.tg_semilinear_residual(p, X, a2, tg.CONSTANT, 1e3, g, r, x_react=x, y=gx_in, loss=False)
        ms_acj = timed(torch, acj, flush)
        ba = E * 3 * 4 + N * 2 * s + 3 * N * s + N  # cells, coords, x, U0 / dt, y, mask (constant a^2)
        out[f"allen_cahn2d_{dtn}"] = {"step_residual_us": ms_ac * 1e3, "jacobian_action_us": ms_acj * 1e3,
                                      "elements_per_s": E / ms_ac * 1e3, "alg_GBps": ba / ms_ac / 1e6,
                                      "frac_hbm": ba / ms_ac / 1e6 / peak,
                                      "note": "one launch each; constant a^2, nodal U0 / dt, mask and loss"}
    return out


def facet_extras(tg, torch, dev, m, p, flush):
    # (the boundary is 0.4% of the nodes: a latency-bound launch, reported in microseconds)
    """Robin matrix term and Neumann/Robin load on the 4,096 boundary edges
    of the 1024^2 workload, added onto assembled values (one launch)."""
    fac = mg.boundary_facets(m)
    fc = tg.tg_build_facets(p, torch.as_tensor(fac, device=dev))
    out = {}
    for dtn, dt in (("f32", torch.float32), ("f64", torch.float64)):
        X = torch.as_tensor(m.coords, dtype=dt, device=dev)
        al = torch.as_tensor(np.random.default_rng(3).uniform(0.5, 2, len(fac) * 2), dtype=dt, device=dev)
        g = torch.as_tensor(np.random.default_rng(4).uniform(-1, 1, m.n_nodes), dtype=dt, device=dev)
        v = torch.zeros(p.nnz, dtype=dt, device=dev)
        F = torch.zeros(m.n_nodes, dtype=dt, device=dev)
        ms = timed(torch, lambda: tg.tg_assemble_facets(fc, X, al, tg.PER_QP, g, tg.PER_NODE, v, F), flush)
        es = 4 if dt == torch.float32 else 8
        # facet ids, their nodes' coordinates and g, alpha per point, and a read-modify-write of the touched
        # CSR entries (3 per boundary node) and of F
        fb = len(fac) * 2 * 4 + fc.n_boundary_nodes * (2 * es + es) + len(fac) * 2 * es \
            + fc.n_boundary_nodes * 4 * es * 2
        out[f"facets2d_{dtn}"] = {"facets": len(fac), "boundary_nodes": fc.n_boundary_nodes, "us": ms * 1e3,
                                  "alg_GBps": fb / ms / 1e6,
                                  "note": "Robin alpha per facet point and nodal g, added into CSR values and F"}
    return out


def small_configs(tg, torch, dev):
    """The two small configurations, reported as absolute times (latency- and
    launch-bound at these sizes): the 64^2 Poisson problem (system assembly,
    then CG to 1e-10 on the Dirichlet-condensed system, FP64) and one full
    gradient evaluation of the 48^3 differentiable problem (assembly + CG,
    adjoint CG + backward assembly, FP64)."""
    from paper_2602_05052_gb300 import autograd as A
    out = {}
    d = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=dev)
    cfg = mg.poisson2d(64)
    m = cfg["mesh"]
    p = tg.tg_build_pattern(d(m.cells, torch.int32), m.n_nodes, tg.P1_TRI)
    x, one = d(m.coords), d([1.0])
    mask = d(m.boundary.astype(np.uint8), torch.uint8)
    vals = torch.empty(p.nnz, dtype=torch.float64, device=dev)
    F = torch.empty(m.n_nodes, dtype=torch.float64, device=dev)

    def poisson():
        tg.tg_assemble_system(p, x, one, tg.CONSTANT, 0.0, one, tg.CONSTANT, vals=vals, F=F)
        return tg.tg_cg_solve(p, vals, F, mask, rtol=1e-10)

    for _ in range(3):
        poisson()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 10
    for _ in range(reps):
        _, it, rel = poisson()
    torch.cuda.synchronize()
    ms_sys = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        tg.tg_assemble_system(p, x, one, tg.CONSTANT, 0.0, one, tg.CONSTANT, vals=vals, F=F)
    e1.record()
    torch.cuda.synchronize()
    ms_sys = e0.elapsed_time(e1) / reps
    out["poisson2d_64_f64"] = {"elements": m.n_elems, "system_assembly_us": 1e3 * ms_sys,
                               "assembly_plus_cg_ms": 1e3 * (time.perf_counter() - t0) / reps, "cg_iterations": it,
                               "cg_relres": rel, "note": "host wall time: the CG runs in one cooperative launch"}
    del p
    cfg = mg.differentiable3d(48)
    m = cfg["mesh"]
    p = tg.tg_build_pattern(d(m.cells, torch.int32), m.n_nodes, tg.P1_TET)
    mask = d(m.boundary.astype(np.uint8), torch.uint8)
    x0, f = d(m.coords), d([1.0])
    with torch.no_grad():
        u_t = A.solve_assembled(p, x0, d(cfg["kappa_star"]), tg.PER_ELEMENT, f, tg.CONSTANT, mask, rtol=1e-13)
    k0 = d(cfg["kappa"])

    def grad_eval():
        k = k0.clone().requires_grad_(True)
        x = x0.clone().requires_grad_(True)
        u = A.solve_assembled(p, x, k, tg.PER_ELEMENT, f, tg.CONSTANT, mask, rtol=1e-13)
        L = ((u - u_t) ** 2).sum()
        L.backward()
        return k.grad, x.grad

    grad_eval()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        grad_eval()
    torch.cuda.synchronize()
    t_grad = (time.perf_counter() - t0) / 3
    vals = torch.empty(p.nnz, dtype=torch.float64, device=dev)
    F = torch.empty(m.n_nodes, dtype=torch.float64, device=dev)
    e0.record()
    for _ in range(reps):
        tg.tg_assemble_system(p, x0, k0, tg.PER_ELEMENT, 0.0, f, tg.CONSTANT, vals=vals, F=F)
    e1.record()
    torch.cuda.synchronize()
    out["differentiable3d_48_f64"] = {"elements": m.n_elems, "system_assembly_us": 1e3 * e0.elapsed_time(e1) / reps,
                                      "gradient_evaluation_ms": 1e3 * t_grad,
                                      "note": "gradient evaluation = assembly + CG (1e-13) + adjoint CG + backward "
                                              "assembly + load backward, host wall time"}
    # SIMP cantilever (60 x 30 QUAD4, plane stress): one optimisation iteration's assembly, solve and sensitivity
    cfg = mg.cantilever()
    m = cfg["mesh"]
    p = tg.tg_build_pattern(d(m.cells, torch.int32), m.n_nodes, tg.Q1_QUAD_VEC2)
    X, rho, Fq = d(m.coords), d(cfg["rho"]), d(cfg["F"])
    mask = d(cfg["dirichlet"].astype(np.uint8), torch.uint8)
    law = (cfg["E_min"], cfg["E_max"], cfg["penal"], cfg["nu"])
    vq = torch.empty(p.nnz, dtype=torch.float64, device=dev)
    dc = torch.empty_like(rho)

    def simp_iter():
        tg.tg_assemble_simp(p, X, rho, *law, vals_out=vq)
        u, it, rel = tg.tg_cg_solve(p, vq, Fq, mask, rtol=1e-10, maxit=200000)
        tg.tg_simp_sensitivity(p, X, rho, *law, u, dc_out=dc)
        return it

    simp_iter()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        it = simp_iter()
    torch.cuda.synchronize()
    t_it = (time.perf_counter() - t0) / 3
    u0 = torch.zeros(2 * m.n_nodes, dtype=torch.float64, device=dev)
    e0.record()
    for _ in range(reps):
        tg.tg_assemble_simp(p, X, rho, *law, vals_out=vq)
    e1.record()
    torch.cuda.synchronize()
    t_asm = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        tg.tg_simp_sensitivity(p, X, rho, *law, u0, dc_out=dc)
    e1.record()
    torch.cuda.synchronize()
    out["simp_cantilever_60x30_f64"] = {"elements": m.n_elems, "assembly_us": 1e3 * t_asm,
                                        "sensitivity_us": 1e3 * e0.elapsed_time(e1) / reps,
                                        "iteration_ms": 1e3 * t_it, "cg_iterations": it,
                                        "note": "iteration = SIMP assembly + CG to 1e-10 + sensitivity, host wall "
                                                "time (the CG runs in one cooperative launch)"}
    return out


if __name__ == "__main__":
    main()
