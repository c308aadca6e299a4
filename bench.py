#!/usr/bin/env python3
"""Throughput of the FWHT Pauli-spectrum hot path on GB300.

One step is one sre_mc call in SRE_MC_MARGINAL mode on an N=24 Haar-random
complex64 state (seed 24): normalisation, the exact x-marginal
p(x) = WHT(WHT(|psi|^2)^2)/d and its FP64 CDF, 4096 X-masks drawn from p,
one 2^24-point family transform per X-mask with the fused moment reduction,
and 256 z drawn per family from its spectrum, then the estimators. The metric
counts every Pauli expectation a family transform produces (2^24 per x).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

N > 1 runs one rank per GPU under torchrun (weak scaling: every rank its own
4096 families per step from its own counter range, no data-path collective).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Pauli expectations/s at N=24 (split-BF16 TC vs FP32 SIMT), % HBM roofline"
UNIT = "Pauli expectations/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--N", type=int, default=24)
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--zpx", type=int, default=256)
    ap.add_argument("--x-batch", type=int, default=0)
    ap.add_argument("--radix", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tc", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra workloads (mixed N=24, exact N=18, batched) reported beside the headline")
    ap.add_argument("--workload", default="mc24",
                    choices=["mc24", "batched", "precondition", "mixed", "exact18", "n30"],
                    help="mc24: the headline N=24 MC step; batched: exact M_2/nullity of 4096 T-doped states "
                         "with N ~ U{8..16} in one sre_exact_batched call, against a per-state loop")
    ap.add_argument("--count", type=int, default=4096)
    return ap.parse_args()


TRAFFIC_SOURCES = ("k_pass.cuh", "sre_internal.cuh", "k_pass_f32_multi.cu", "k_pass_dispatch.cuh")


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 over the pass kernel's sources: the
    key under which profiles/traffic.json records a capture."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2601_00761_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(N, dom_pass):
    """ncu DRAM bytes (read + write) per family of pass `dom_pass` at N, from
    profiles/traffic.json (a small-case capture, scaled per family), or None
    when no capture exists for that pass or the kernel's sources changed since
    it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        e = rec["captures"][f"N{N}_pass{dom_pass}"]
        if e["source_sha256_16"] != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_family"]), e
    except Exception:
        return None


def dram_min_bytes(N, dom_pass, npass, fam):
    """Bytes pass `dom_pass` must move through DRAM per launch of `fam`
    families: pass 0 reads psi once per launch (the families of a launch share
    its lines in L2) and writes the 4 B-per-string packed intermediate; a later
    pass reads the intermediate (and writes it again unless it is the last)."""
    d = float(2 ** N)
    if dom_pass == 0:
        return 8.0 * d + 4.0 * d * fam
    return 4.0 * d * fam * (1 if dom_pass == npass - 1 else 2)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak():
    """Dense BF16 tensor rate (TFLOP/s): the measured burst figure, else the
    fallback of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def tc_mma_flop_per_family(pass_bits, N, nsplit=3):
    """Tensor-core FLOPs a family issues in the split-BF16 form: every
    4-bit group of a pass's transformed bits is one H_16 product, 16 MACs (32
    FLOP) per packed point for each BF16 part of the real and of the
    imaginary plane; leftover bits are FP32 butterflies."""
    rounds = sum(b // 4 for b in pass_bits)
    return 2.0 ** (N - 1) * rounds * 32.0 * nsplit * 2


# ------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.p = None
        self.idx = gpu_index
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="sre_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        lines = open(self.path).read().splitlines()
        try:
            os.unlink(self.path)
        except OSError:
            pass
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    N, n_fam, zpx, seed, ctr0 = args
    import oracle
    from paper_2601_00761_gb300 import inputs
    psi = inputs.haar_state(N, 24)
    t0 = time.perf_counter()
    oracle.mc_marginal(psi, n_fam, zpx, seed, ctr0)
    return time.perf_counter() - t0


def oracle_throughput(N, zpx, workers=None, n_fam=2, seed=24, ctr0=0):
    """The oracle as it stands (sre_oracle.c via ctypes, single-threaded C)
    run concurrently in `workers` spawned processes, each on n_fam families of
    the same workload (plus its own x-marginal). Returns (c/s, cores, sample)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    workers = workers or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        times = pool.map(_oracle_worker, [(N, n_fam, zpx, seed, ctr0 + 1000 * i) for i in range(workers)])
    wall = time.perf_counter() - t0
    per = [n_fam * (2 ** N) / t for t in times]
    value = sum(per)
    sample = (f"{workers} processes x {n_fam} families of 2^{N} (each with its own FP64 x-marginal and "
              f"{zpx} z-draws per family), oracle C code single-threaded per process; "
              f"max worker time {max(times):.1f}s, wall {wall:.1f}s")
    return value, workers, sample


# ------------------------------------------------------------ reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    vals = []
    cores = 1
    sample = ""
    for i in range(a.warmup + a.steps):
        v, cores, sample = oracle_throughput(a.N, a.zpx, n_fam=2, ctr0=10_000 * i)
        if i >= a.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    fam_time = 2 * 2 ** a.N / (value / cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": fam_time * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Haar state, N=24)",
            "config": {"workload": f"N={a.N} MC marginal: x ~ p(x), one 2^{a.N}-point family transform per x, "
                                   f"{a.zpx} z per x", "N": a.N, "z_per_x": a.zpx, "seed": 24,
                       "families_per_step": 2 * cores},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ replicas
# bench.py --gpus N under torchrun runs N independent replicas (one GPU each):
# every rank draws from its own Philox counter range, the timed region is
# bracketed by barriers, and the step time is the maximum over ranks.
COUNTER_STRIDE_LOG2 = 40


def counter_base(rank: int) -> int:
    """First Philox counter of a rank's draws (disjoint ranges of 2^40)."""
    return rank << COUNTER_STRIDE_LOG2


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (all ranks call it; barrier, then MAX all-reduce)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dist.barrier()
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- CUDA arm
def run_cuda(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2601_00761_gb300 import build as sre_build
    sre_build.build()
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import inputs

    N, n_x, zpx = a.N, a.nx, a.zpx
    kw = {"x_batch": a.x_batch, "radix_log2": a.radix, "tile_log2": a.tile}
    psi_host = torch.from_numpy(inputs.haar_state(N, 24)).pin_memory()
    psi = psi_host.to(dev)
    ws = torch.empty(sre.sre_workspace_bytes(N, sre.SRE_MC_MARGINAL, n_x, zpx, **kw), dtype=torch.uint8,
                     device=dev)
    xs = torch.empty(n_x, dtype=torch.int64, device=dev)
    zs = torch.empty(n_x * zpx, dtype=torch.int64, device=dev)
    cs = torch.empty(n_x * zpx, dtype=torch.float32, device=dev)
    base_ctr = counter_base(rank)

    def step(i):
        return sre.sre_mc(psi, sre.SRE_MC_MARGINAL, n_x, zpx, seed=24, counter0=base_ctr + i * n_x,
                          workspace=ws, outputs=(xs, zs, cs), **kw)

    for i in range(a.warmup):
        step(i)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = Clocks(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sre.sre_kernel_launches()
    sre.sre_pass_timing(True)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    res = None
    for i in range(a.steps):
        res = step(a.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    timing = sre.sre_pass_timing(False)
    launches = sre.sre_kernel_launches() - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    total_c = world * a.steps * n_x * float(2 ** N)
    value = total_c / (ms / 1e3)

    # dominant kernel of the step: the pass with the largest total time
    hbm, peak_kind = peaks()
    npass = res["n_passes"]
    shares = [timing["ms_sum"][p] for p in range(npass)]
    dom = int(np.argmax(shares))
    avg_ms = timing["ms_sum"][dom] / max(1, timing["launches"][dom])
    algo_bytes = timing["bytes_per_launch"][dom]            # 8 B psi per string per family (+ 4 B out)
    fam_launch = max(1, round(n_x / max(1, timing["launches"][dom] / a.steps)))
    min_bytes = dram_min_bytes(N, dom, npass, fam_launch)
    step_bytes = sum(timing["bytes_per_launch"][p] * timing["launches"][p] for p in range(npass)) / a.steps
    tp = profiled_traffic(N, dom) if not (a.radix or a.tile or a.x_batch) else None
    traffic = tp[0] * fam_launch if tp else None
    # achieved: the bytes DRAM moved per launch (ncu, small-case capture scaled
    # to the launch's families) over the live CUDA-event launch time; without a
    # capture for the current kernel, the DRAM-minimal bytes of the launch
    basis = traffic if traffic is not None else min_bytes
    achieved = basis / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic,
                "achieved_basis": ("ncu dram__bytes_read+write per family (small-case capture, "
                                   "profiles/traffic.json) x families per launch") if traffic is not None else
                                  "DRAM-minimal bytes per launch (no ncu capture for the current kernel sources)",
                "dram_min_bytes_per_launch": min_bytes,
                "frac_dram_min": min_bytes / (avg_ms / 1e3) / 1e9 / hbm,
                "algorithmic_bytes_per_launch": algo_bytes,
                "frac_algorithmic": algo_bytes / (avg_ms / 1e3) / 1e9 / hbm,
                "frac_algorithmic_note": "16 B per string counted with psi read from DRAM by every family; "
                                         "the families of a launch share psi in L2, so this exceeds 1",
                "traffic_capture": tp[1].get("capture") if tp else None,
                "kernel": ["strided pass 0 (reads psi, writes the packed intermediate)",
                           "row pass (reads the intermediate, fused moments)"][min(dom, 1)]
                if npass == 2 else f"pass {dom}",
                "families_per_launch": fam_launch,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "avg_launch_ms": avg_ms,
                "pass_avg_launch_ms": [timing["ms_sum"][p] / max(1, timing["launches"][p]) for p in range(npass)],
                "pass_ms_share": [s_ / sum(shares) for s_ in shares],
                "step_algorithmic_GBps": step_bytes / (ms / a.steps / 1e3) / 1e9}

    # the split-BF16 tensor-core form on the same workload (BF16X3: FP32-level accuracy)
    tc = None
    if not a.no_tc:
        kw_tc = dict(kw, precision=2)
        def step_tc(i):
            return sre.sre_mc(psi, sre.SRE_MC_MARGINAL, n_x, zpx, seed=24, counter0=base_ctr + (1 << 31) + i * n_x,
                              workspace=ws, outputs=(xs, zs, cs), **kw_tc)
        step_tc(0)
        torch.cuda.synchronize()
        sre.sre_pass_timing(True)
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        tc_steps = max(1, min(a.steps, 3))
        for i in range(tc_steps):
            rtc = step_tc(1 + i)
        t1e.record(stream)
        torch.cuda.synchronize()
        tt = sre.sre_pass_timing(False)
        tms = t0e.elapsed_time(t1e)
        if world > 1:
            t = torch.tensor([tms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tms = float(t.item())
        tdom = int(np.argmax([tt["ms_sum"][p] for p in range(npass)]))
        tavg = tt["ms_sum"][tdom] / max(1, tt["launches"][tdom])
        tach = tt["bytes_per_launch"][tdom] / (tavg / 1e3) / 1e9
        mma_tflops = (tc_mma_flop_per_family(sre.sre_make_plan(N, **kw)["pass_bits"], N) * n_x
                      / (tms / tc_steps / 1e3) / 1e12)
        bf16, bf16_kind = bf16_peak()
        tc = {"precision": "split-BF16 x3 (mma.sync m16n8k16, FP32 accumulate)",
              "value": world * tc_steps * n_x * float(2 ** N) / (tms / 1e3), "unit": UNIT,
              "ms_per_step": tms / tc_steps, "dominant_pass": tdom, "achieved_GBps": tach, "frac": tach / hbm,
              "mma_tflops": mma_tflops, "mma_frac": mma_tflops / bf16,
              "mma_peak": {"tflops": bf16, "kind": f"{bf16_kind} dense BF16 (MEASURED_PEAKS.json bf16_tflops)"},
              "pass_ms_share": [tt["ms_sum"][p] / sum(tt["ms_sum"][:npass]) for p in range(npass)],
              "M_rb": rtc["M_rb"], "err_rb": rtc["err_rb"]}

    # end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        xs_h = torch.empty(n_x, dtype=torch.int64).pin_memory()
        zs_h = torch.empty(n_x * zpx, dtype=torch.int64).pin_memory()
        cs_h = torch.empty(n_x * zpx, dtype=torch.float32).pin_memory()
        # Every step uploads its state from pinned host memory and reads its
        # samples back. The upload of step i + 1 runs on a copy stream into the
        # other of two device buffers while step i computes; all of them lie
        # inside the timed region.
        bufs = [torch.empty_like(psi), torch.empty_like(psi)]
        cstream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cstream.wait_event(e0)
        with torch.cuda.stream(cstream):
            bufs[0].copy_(psi_host, non_blocking=True)
            copied[0].record(cstream)
        for i in range(a.steps):
            b = i % 2
            stream.wait_event(copied[b])
            if i + 1 < a.steps:
                cstream.wait_event(used[1 - b])
                with torch.cuda.stream(cstream):
                    bufs[1 - b].copy_(psi_host, non_blocking=True)
                    copied[1 - b].record(cstream)
            sre.sre_mc(bufs[b], sre.SRE_MC_MARGINAL, n_x, zpx, seed=24,
                       counter0=base_ctr + (1 << 30) + i * n_x, workspace=ws, outputs=(xs, zs, cs), **kw)
            used[b].record(stream)
            xs_h.copy_(xs, non_blocking=True)
            zs_h.copy_(zs, non_blocking=True)
            cs_h.copy_(cs, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": total_c / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": psi_host.numel() * psi_host.element_size(),
               "d2h_bytes_per_step": n_x * 8 + n_x * zpx * 12 + 8 * 3}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, cores, sample = oracle_throughput(N, zpx)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    # the other workloads, measured in the same run and reported beside the
    # headline (each as its own bench line would print it)
    extras = None
    if rank == 0 and world == 1 and not a.no_extras:
        extras = {}
        for name, fn, over in (("mixed_n24", measure_mixed, dict(N=24, steps=10, warmup=3)),
                               ("exact_n18", measure_exact18, dict(steps=1, warmup=1)),
                               ("batched", measure_batched, dict(count=4096, steps=2, warmup=1))):
            try:
                extras[name] = fn(argparse.Namespace(**{**vars(a), **over}))
            except Exception as ex:          # reported, not fatal to the headline line
                extras[name] = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Haar state)",
                "config": {"workload": f"N={N} Haar MC marginal: {n_x} x per step from the exact p(x), one "
                                       f"2^{N}-point family transform per x, {zpx} z per x",
                           "N": N, "n_x_per_step": n_x, "z_per_x": zpx, "seed": 24, "precision": "FP32 SIMT",
                           "passes": npass, "l2": "inputs larger than L2: psi is 128 MiB and every step "
                                                  "streams GiBs of intermediate", "parallelism": f"replica x{world}"},
                "roofline": roofline, "tensor_core_form": tc, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(launches),
                "estimates": {"M": res["M"], "err_M": res["err_M"], "M_rb": res["M_rb"], "err_rb": res["err_rb"],
                              "M2_haar_closed_form": math.log2(2 ** N + 3) - 2},
                "extra_workloads": extras}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_batched(a):
    """Uneven batch: count T-doped random Clifford states (N ~ U{8..16},
    eta ~ U{1,2,4,8,32}, n_T ~ U{1..3N}, seeds 4000+i) prepared on the GPU;
    one step = one sre_exact_batched call over all of them. The same states
    through a per-state sre_exact loop are timed beside it."""
    import torch
    from paper_2601_00761_gb300 import build as sre_build
    sre_build.build()
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import inputs
    torch.cuda.set_device(0)
    specs = inputs.workload_batched_specs(count=a.count)
    states = []
    for sp in specs:
        p = torch.zeros(1 << sp["N"], dtype=torch.complex64, device="cuda")
        p[0] = 1
        sre.apply_clifford_tdoped_circuit(p, inputs.batched_gate_list(sp))
        states.append(p)
    total_c = float(sum(4 ** sp["N"] for sp in specs))
    tuned = {}
    for N in sorted({sp["N"] for sp in specs}):
        if sre.sre_make_plan(N)["n_passes"] > 1:
            tuned[N] = sre.sre_autotune(next(p for p, sp in zip(states, specs) if sp["N"] == N))
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        sre.sre_exact_batched(states)
    torch.cuda.synchronize()
    l0 = sre.sre_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        res = sre.sre_exact_batched(states)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    launches = sre.sre_kernel_launches() - l0
    # per-state launch loop on the same states
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    loop = [sre.sre_exact(p, allow_nullity_error=True) for p in states]
    t1.record(stream)
    torch.cuda.synchronize()
    ms_loop = t0.elapsed_time(t1)
    dmax = max(abs(r["M"][1] - q["M"][1]) for r, q in zip(res, loop))
    # every family of every state in one persistent launch (dependency queue), one timed call
    sre.sre_exact_batched(states, batch_queue=1)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    resq = sre.sre_exact_batched(states, batch_queue=1)
    q1.record(stream)
    torch.cuda.synchronize()
    ms_q = q0.elapsed_time(q1)
    dq = max(abs(r["M"][1] - q["M"][1]) for r, q in zip(res, resq))
    line = {"metric": "Pauli expectations/s, batched uneven exact M_2 and nullity", "value": total_c / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded T-doped circuits)",
            "config": {"workload": f"{a.count} T-doped random Clifford states, N ~ U{{8..16}}, one sre_exact_batched call",
                       "states": a.count, "pauli_strings": total_c, "tuned": {str(k): v for k, v in tuned.items()}},
            "per_state_loop": {"value": total_c / (ms_loop / 1e3), "ms": ms_loop},
            "queue_mode": {"value": total_c / (ms_q / 1e3), "ms": ms_q, "max_dM2_vs_default": dq,
                           "what": "batch_queue=1: every family of every state in one persistent launch"},
            "max_dM2_vs_loop": dmax, "gpu_launches": int(launches)}
    return line


def run_batched(a):
    print(json.dumps(measure_batched(a)), flush=True)
    return 0


def run_precondition(a):
    """Clifford preconditioning (main text and SM): the product magic state
    |T>^{N/2}|0>^{N/2}, a random brick-wall Clifford circuit of depth
    N_C = 2N applied on the device (timed: K applications after W warm-up
    applications, each one host call including its gate-table upload), and
    the uniform-x estimator's fluctuation ratio r_2 and M_2 before and after
    (n_x families each)."""
    import torch
    from paper_2601_00761_gb300 import build as sre_build
    sre_build.build()
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import inputs
    torch.cuda.set_device(0)
    N = a.N
    n_x = a.nx if a.nx != 4096 else 20000
    psi = torch.from_numpy(inputs.t_product_state(N, N // 2)).cuda()
    mats, pairs = inputs.brickwall_circuit(N, 2 * N, "clifford", 30 + N)
    before = sre.sre_mc(psi, sre.SRE_MC_UNIFORM, n_x, 1, seed=N)
    scratch = psi.clone()
    for _ in range(a.warmup):
        sre.apply_two_qubit_gates(scratch, mats, pairs)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    l0 = sre.sre_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(a.steps):
        sre.apply_two_qubit_gates(scratch, mats, pairs)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    blocks = (sre.sre_kernel_launches() - l0) // a.steps
    sweep_bytes = blocks * 2 * 8 * 2 ** N          # each fused block reads and writes psi once
    gbps = sweep_bytes / (ms / 1e3) / 1e9
    hbm, peak_kind = peaks()
    # a general two-qubit gate is a 4x4 complex matrix on each of the 2^(N-2)
    # amplitude quartets: 16 complex multiply-adds = 64 real FMA = 128 FLOP
    flop = len(pairs) * 2 ** (N - 2) * 128.0
    tflops = flop / (ms / 1e3) / 1e12
    fp32_peak = fp32_fma_peak_tflops()
    after_state = psi.clone()
    sre.apply_two_qubit_gates(after_state, mats, pairs)
    after = sre.sre_mc(after_state, sre.SRE_MC_UNIFORM, n_x, 1, seed=N)
    m2 = (N // 2) * math.log2(4 / 3)
    # r_2 against the preconditioner's depth N_C (prefixes of the same circuit)
    sweep = []
    n_sweep = min(n_x, 8192)
    for depth in (0, 2, 4, 8, 16, 24, 32, 2 * N):
        st_ = psi.clone()
        if depth:
            mk, pk = inputs.brickwall_circuit(N, depth, "clifford", 30 + N)
            sre.apply_two_qubit_gates(st_, mk, pk)
        r = sre.sre_mc(st_, sre.SRE_MC_UNIFORM, n_sweep, 1, seed=N + 1)
        sweep.append({"layers": depth, "r2": r["r2"], "M2": r["M"][1], "err_M2": r["err_M"][1]})
    line = {"metric": f"brick-wall Clifford preconditioner (depth 2N) on psi at N={N}, two-qubit gates applied per second",
            "value": len(pairs) / (ms / 1e3), "unit": "gates/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (|T>^{N/2}|0>^{N/2}, seeded uniform two-qubit Cliffords)",
            "config": {"workload": f"N={N} product magic state, {len(pairs)} two-qubit Cliffords in {2 * N} "
                                   f"brick-wall layers, then {n_x} uniform-x MC families",
                       "N": N, "gates": int(len(pairs)), "layers": 2 * N, "n_x": n_x},
            "roofline": {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": tflops / fp32_peak, "traffic": None,
                         "kernel": "gate_block_kernel (13-qubit fused blocks, 4x4 complex matrices)",
                         "flop_per_step": flop,
                         "peak_kind": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x max SM clock (MEASURED_PEAKS.json sm_max_mhz)",
                         "hbm": {"bytes_per_step": sweep_bytes, "achieved_GBps": gbps, "frac": gbps / hbm},
                         "blocks_per_circuit": int(blocks)},
            "clocks": clk, "gpu_launches": int(blocks * a.steps),
            "study": {"M2_closed_form": m2,
                      "before": {"r2": before["r2"], "M2": before["M"][1], "err_M2": before["err_M"][1]},
                      "after": {"r2": after["r2"], "M2": after["M"][1], "err_M2": after["err_M"][1]},
                      "r2_closed_form_before": r2_psi_m(N),
                      "r2_vs_layers": {"n_x": n_sweep, "points": sweep}}}
    print(json.dumps(line), flush=True)
    return 0


def measure_mixed(a):
    """SRE of the reduced state of the first N_A = N/2 qubits of an N-qubit
    Haar state (SM, mixed states): one step = one sre_mixed call (Gram matrix
    on the tensor cores, 2^{N_A} family transforms with fused moments,
    totals)."""
    import torch
    from paper_2601_00761_gb300 import build as sre_build
    sre_build.build()
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import inputs
    torch.cuda.set_device(0)
    N = a.N
    NA = N // 2
    psi = torch.from_numpy(inputs.haar_state(N, N)).cuda()
    ws = torch.empty(sre.sre_mixed_workspace_bytes(N, NA), dtype=torch.uint8, device="cuda")
    for _ in range(a.warmup):
        r = sre.sre_mixed(psi, NA, workspace=ws)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    l0 = sre.sre_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(a.steps):
        r = sre.sre_mixed(psi, NA, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    launches = sre.sre_kernel_launches() - l0
    dA, dB = 2 ** NA, 2 ** (N - NA)
    # tensor-core work issued per call (NA >= 7, N - NA >= 5): the upper-triangle
    # 128 x 128 tiles of C, each over d_B / 16 K blocks of 24 BF16 MMAs of
    # 128 x 128 x 16 (4 real products x 6 split-part pairs)
    nt = dA // 128
    tiles = nt * (nt + 1) // 2
    mma_flop = tiles * (dB // 16) * 24 * 2.0 * 128 * 128 * 16
    tflops = mma_flop / (ms / 1e3) / 1e12
    bf16, bf16_kind = bf16_peak()
    line = {"metric": f"Pauli expectations/s on a subsystem: Tr(rho_A P) for all 4^{NA} P on the first {NA} of {N} qubits",
            "value": 4.0 ** NA / (ms / 1e3), "unit": "Pauli expectations/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Haar state)",
            "config": {"workload": f"N={N} Haar state, reduced state of the first {NA} qubits, one sre_mixed call",
                       "N": N, "N_A": NA},
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16, "unit": "TFLOP/s", "frac": tflops / bf16,
                         "traffic": None,
                         "kernel": "Gram matrix Psi Psi^H (gram_tc_kernel: tcgen05 BF16 MMAs over BF16x3-split "
                                   "planes, six part products, FP32 accumulation); achieved = BF16 MMA FLOP issued "
                                   "per call / whole call time (split, diagonal and the 2^N_A family transforms "
                                   "included)",
                         "mma_flop_per_step": mma_flop,
                         "fp32_gemm_equivalent_tflops": 8.0 * dA * dA * dB / (ms / 1e3) / 1e12,
                         "peak_kind": f"{bf16_kind} dense BF16 (MEASURED_PEAKS.json bf16_tflops)"},
            "clocks": clk, "gpu_launches": int(launches),
            "estimates": {"S2": r["S2"], "M": r["M"], "err_M": r["err_M"]}}
    return line


def run_mixed(a):
    print(json.dumps(measure_mixed(a)), flush=True)
    return 0


def measure_exact18(a):
    """Exact enumeration at N = 18 (all 4^18 Pauli expectations of each of the
    twelve T-doped states: eta in {1, 4, 16} x n_T in {0, 8, 32, 64}), FP32 SIMT
    and split-BF16 (x3) tensor-core transforms. One step = sre_exact over all
    twelve states."""
    import torch
    from paper_2601_00761_gb300 import build as sre_build
    sre_build.build()
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import inputs
    torch.cuda.set_device(0)
    specs = inputs.workload_n18_gate_lists()
    states = []
    for sp in specs:
        p = torch.zeros(1 << 18, dtype=torch.complex64, device="cuda")
        p[0] = 1
        sre.apply_clifford_tdoped_circuit(p, sp["gates"])
        states.append(p)
    stream = torch.cuda.current_stream()

    def timed(prec):
        for _ in range(a.warmup):
            for p in states:
                sre.sre_exact(p, allow_nullity_error=True, precision=prec)
        torch.cuda.synchronize()
        l0 = sre.sre_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            res = [sre.sre_exact(p, allow_nullity_error=True, precision=prec) for p in states]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / a.steps, res, sre.sre_kernel_launches() - l0

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, res, launches = timed(0)
    clk = clocks.stop()
    ms_tc, res_tc, _ = timed(2)
    mma_tflops = (tc_mma_flop_per_family(sre.sre_make_plan(18)["pass_bits"], 18) * 2.0 ** 18 * len(states)
                  / (ms_tc / 1e3) / 1e12)
    total_c = len(states) * 4.0 ** 18
    flop = total_c * 30.0        # 18 butterfly adds + ~12 FLOP of phase, squares and moment sums per string
    tflops = flop / (ms / 1e3) / 1e12
    peak = fp32_fma_peak_tflops()
    dm = max(abs(r["M"][k] - q["M"][k]) for r, q in zip(res, res_tc) for k in range(3))
    line = {"metric": "Pauli expectations/s, exact enumeration at N=18 (12 T-doped states)",
            "value": total_c / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded T-doped random Clifford circuits, eta x n_T grid)",
            "config": {"workload": "N=18, eta in {1,4,16} x n_T in {0,8,32,64}, sre_exact per state",
                       "states": len(states), "pauli_strings": total_c},
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                         "traffic": None, "kernel": "strided + row passes (psi and the families live in L2)",
                         "flop_per_step": flop,
                         "peak_kind": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x max SM clock (MEASURED_PEAKS.json sm_max_mhz)"},
            "tensor_core_form": {"precision": "split-BF16 x3", "value": total_c / (ms_tc / 1e3), "ms_per_step": ms_tc,
                                 "max_abs_dM_vs_fp32": dm, "mma_tflops": mma_tflops,
                                 "mma_frac": mma_tflops / bf16_peak()[0]},
            "clocks": clk, "gpu_launches": int(launches),
            "states": [{"eta": sp["eta"], "n_t": sp["n_t"], "M": r["M"], "nullity": r["nullity"]}
                       for sp, r in zip(specs, res)]}
    return line


def run_exact18(a):
    print(json.dumps(measure_exact18(a)), flush=True)
    return 0


def run_n30(a):
    """Large MC with Clifford preconditioning at N = 30 (8 GB state): a T-doped
    random Clifford circuit (eta = 16, n_T = 60: 960 Cliffords + 60 T) from
    |0>, then 2000 random {H, S, CNOT} gates, both applied on the device; then
    the marginal MC, 16 z per x. r_2 is sampled (512 uniform x) before and
    after the preconditioner; a 256-family pilot gives the family count that
    brings the standard errors of M_1 and of M_2 to 1e-3 (reported apart); the
    timed step is one sre_mc call of that many families, at most --nx."""
    import torch
    from paper_2601_00761_gb300 import build as sre_build
    sre_build.build()
    import paper_2601_00761_gb300 as sre
    from paper_2601_00761_gb300 import inputs
    torch.cuda.set_device(0)
    N, zpx = 30, 16
    psi = torch.zeros(1 << N, dtype=torch.complex64, device="cuda")
    psi[0] = 1
    circ = inputs.random_clifford_tdoped_gates(N, 960, 16, 30)
    pre = inputs.random_clifford_gates(N, 2000, 31)
    stream = torch.cuda.current_stream()
    sre.apply_clifford_tdoped_circuit(psi, circ)
    r2_before = sre.sre_mc(psi, sre.SRE_MC_UNIFORM, 512, 1, seed=41)["r2"]
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    sre.apply_clifford_tdoped_circuit(psi, pre)
    g1.record(stream)
    torch.cuda.synchronize()
    ms_gates = g0.elapsed_time(g1)
    r2_after = sre.sre_mc(psi, sre.SRE_MC_UNIFORM, 512, 1, seed=41)["r2"]
    pilot = sre.sre_mc(psi, sre.SRE_MC_MARGINAL, 256, zpx, seed=30, counter0=1 << 40)
    need = [max(pilot["err_rb"][k] / 1e-3, 1.0) ** 2 * 256 for k in (0, 1)]
    n_x = int(min(a.nx, max(256, 256 * math.ceil(max(need) / 256))))    # the timed run stays within a minute
    for _ in range(a.warmup):
        sre.sre_mc(psi, sre.SRE_MC_MARGINAL, 32, zpx, seed=30, counter0=2 << 40)
    torch.cuda.synchronize()
    l0 = sre.sre_kernel_launches()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = sre.sre_mc(psi, sre.SRE_MC_MARGINAL, n_x, zpx, seed=30)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = sre.sre_kernel_launches() - l0
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    rtc = sre.sre_mc(psi, sre.SRE_MC_MARGINAL, 256, zpx, seed=30, precision=2)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_tc = t0.elapsed_time(t1)
    plan = sre.sre_make_plan(N)
    line = {"metric": "Pauli expectations/s, preconditioned MC at N=30 to 1e-3 standard error",
            "value": n_x * 2.0 ** N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded T-doped circuit eta=16, n_T=60, then 2000 random Clifford gates)",
            "config": {"workload": "N=30 T-doped state, 2000-gate Clifford preconditioner, marginal MC",
                       "N": N, "n_x": n_x, "n_x_for_1e-3": {"M1": int(math.ceil(need[0])), "M2_at_least": int(math.ceil(need[1]))},
                       "z_per_x": zpx, "passes": plan["n_passes"],
                       "x_batch": plan["x_batch"], "gates": int(len(circ) + len(pre)), "ms_gates": ms_gates},
            "clocks": clk, "gpu_launches": int(launches),
            "r2_sampled": {"before": r2_before, "after": r2_after, "uniform_x": 512},
            "estimates": {"M": r["M"], "err_M": r["err_M"], "M_rb": r["M_rb"], "err_rb": r["err_rb"],
                          "pilot_err_rb": pilot["err_rb"],
                          "reached_1e-3": {"M1": r["err_rb"][0] <= 1e-3, "M2": r["err_rb"][1] <= 1e-3}},
            "tensor_core_form": {"precision": "split-BF16 x3", "n_x": 256,
                                 "value": 256 * 2.0 ** N / (ms_tc / 1e3), "M_rb": rtc["M_rb"], "err_rb": rtc["err_rb"]}}
    print(json.dumps(line), flush=True)
    return 0


def fp32_fma_peak_tflops():
    """FP32 FMA rate from the unit counts (152 SMs x 128 FP32 lanes, 2 FLOP
    per FMA) and the measured maximum SM clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def r2_psi_m(N):
    """SM closed form of r_2 for |T>^{N/2}|0>^{N/2} (even N)."""
    h = N // 2
    x, y, z = (5 / 4) ** h - 1, 4 ** h - 1, (3 / 2) ** h - 1
    return (8 / 3) ** h * math.sqrt(x / y - z * z / (y * y))


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batched":
        return run_batched(a)
    if a.workload == "precondition":
        return run_precondition(a)
    if a.workload == "mixed":
        return run_mixed(a)
    if a.workload == "exact18":
        return run_exact18(a)
    if a.workload == "n30":
        return run_n30(a)
    return run_cuda(a)


if __name__ == "__main__":
    sys.exit(main())
