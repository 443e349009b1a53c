#!/usr/bin/env python
"""Throughput of batched FiRE local-energy evaluation on GB300.

Metric: walker local-energy evaluations per second at n_el = 180 (zigzag
C26H24, 90 up / 90 down, 4096 walkers per GPU, width 256, 4 MLP layers,
16 determinants, c = 5 bohr), BF16+FP64 form, compared with the plain FP32
form at the E_L errors each shows against the FP64 oracle.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
    python bench.py --op grad            # per-walker d log|Psi|/d theta, C26H24
    python bench.py --op mcmc [--chain k | --scan [--chains 2,8,...]]   # Metropolis sweeps, C_kH_{k+2}

One step = one fire_local_energy call over all walkers of the GPU (neighbour
lists included).  Inputs are resident in HBM for `value`; `e2e` adds the
pinned host->device copy of the positions and the device->host copy of E_L.
L2 is flushed (256 MB write) before every timed step.  With torchrun, every
rank evaluates its own 4096 walkers (weak scaling, no data-path collective).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "walker local-energy evals/sec at n_el=180 (BF16+FP64 vs plain FP32, same E_L error)"
UNIT = "walkers/s"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def simt_peaks(dev):
    """Measured multiply-add rates of the float32 and float64 SIMT pipes
    (fire_selftest_fma_rate: eight independent FMA chains per thread, eight
    256-thread CTAs per SM), best of three launches after a warm-up, in
    TFLOP/s.  These are the peaks of the kernels bound by the FP32 or FP64
    pipe."""
    from paper_2504_06087_gb300 import fire
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    out = {"sm_count": sms}
    for key, dt, iters in (("fp32_tflops", torch.float32, 1 << 20), ("fp64_tflops", torch.float64, 1 << 14)):
        fire.fma_probe(dt, 1024, sms * 8, dev)
        best = 0.0
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = fire.fma_probe(dt, iters, sms * 8, dev)
            e1.record(stream)
            e1.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
        out[key] = best
    return out


# ---------------------------------------------------------------------------
# algorithmic work per stage (for the roofline of the dominant kernel)
# ---------------------------------------------------------------------------

# DRAM bytes (read + write) per walker-determinant of a stage, from an ncu
# capture of that kernel (dram__bytes_read.sum + dram__bytes_write.sum of its
# bucket launches for one determinant of a 32-walker chunk, divided by the 32
# walker-determinants); the capture and its command are summarised in the
# named profiles/ file.  A stage whose kernel changed since its capture has
# no entry.
STAGE_TRAFFIC = {
    # float32 SIMT contraction (FP32 form)
    "contract": (2.1812e7, "ncu capture of one determinant of a 32-walker chunk (profiles/contract_c26h24.md)"),
    # tensor-core contraction (BF16_FP64 form)
    "contract_tc": (1.3585e7, "ncu capture of one four-determinant launch over a 128-walker chunk "
                              "(profiles/contract_tc_c26h24.md)"),
}


def stage_traffic(stage, walker_dets, launches):
    """(bytes per launch, source) of a stage, scaled from its capture by the
    walker-determinants one launch covers; (None, None) without a capture."""
    if stage not in STAGE_TRAFFIC:
        return None, None
    per, src = STAGE_TRAFFIC[stage]
    return per * walker_dets / launches, src + f", scaled to {walker_dets // max(launches, 1)} walker-determinants per launch"


def stage_work(stage, w, info, n_walkers, nbr_sq_sum, nbr_sum=None, precision="bf16"):
    """(flops_total, bytes_total, bound) of one call's stage, from the shapes.

    rows = forward-Laplacian rows of the call (value + Laplacian + 3 tangent
    rows per slot of every electron block); nbr_sum = sum over (walker,
    electron) of |Nbar_n|, nbr_sq_sum of |Nbar_n|^2."""
    a, s = w.arch, w.system
    d, J, n, D, L = a.width, a.jw, s.n_el, a.n_det, a.n_layers
    rows = info["rows_total"]
    if stage == "contract" and precision == "bf16" and nbr_sum is not None:
        # tensor-core contraction, bound by streaming its float32 inputs once
        # per determinant: the three tangent O rows of every (member, tangent
        # electron) pair, the value and Laplacian O rows and the five
        # envelope rows of every electron, and A^T (n floats per row)
        per_det = 4.0 * n * (3 * nbr_sum + n_walkers * n * (2 + 5 + 1))
        return None, per_det * D, "hbm"
    if stage == "mlp_gemm":
        return 2.0 * rows * d * d * L, None, "tensor"
    if stage == "orb_gemm":
        return 2.0 * rows * d * n * D, None, "tensor"
    if stage == "jastrow_mlp":
        return 2.0 * 2 * rows * (d * J + J * J + J), None, "tensor"
    if stage == "att_gemm":
        return 2.0 * rows * d * (a.n_reg + a.n_reg * a.d_reg), None, "tensor"
    if stage == "contract":
        # M_ik,nx for i, k in Nbar_n: 3 |Nbar_n|^2 n MACs per (walker, n, det)
        return 2.0 * 3 * nbr_sq_sum * n * D, None, "alu"
    if stage == "lu":
        return (2.0 / 3.0) * n ** 3 * D * n_walkers, None, "fp64"
    if stage == "inverse":
        return 2.0 * n ** 3 * D * n_walkers, None, "alu"
    return None, None, None


def grad_flops(w):
    """Algorithmic FLOPs of one walker's d log|Psi| / d theta: the value
    forward's multiply-adds (one row per electron; every pair feature within
    the cutoffs counted at the mean neighbour count of the workload), times
    three (forward, input adjoint and weight adjoint of every product), times
    two.  The filters: Gamma's 4 -> 16 -> width layers and the 32 Gaussians
    -> width; the envelopes: N_nuc N_env D n per electron."""
    a, s = w.arch, w.system
    d, J, n, D, L = a.width, a.jw, s.n_el, a.n_det, a.n_layers
    filt = 4 * 16 + 16 * d + 32 * d
    kbar = 24.8 if n == 180 else float(n - 1)
    mac = (n * s.n_nuc * filt            # electron-nucleus filters
           + 3 * n * d * d               # GLU ([W_g | W_v] and W_o)
           + 4 * n * d * d               # message projections
           + n * kbar * filt             # electron-electron filters
           + L * n * d * d               # embedding MLP
           + n * d * D * n               # orbitals
           + n * s.n_nuc * a.n_env * D * n   # envelopes
           + 2 * n * (d * J + J * J + J)     # MLP Jastrows
           + n * d * (a.n_reg + a.n_reg * a.d_reg))   # attention scores and values
    return 2.0 * 3.0 * mac


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fire", choices=["fire", "reference"])
    ap.add_argument("--walkers", type=int, default=4096)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 comparison leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-coords", type=int, default=8,
                    help="second-derivative passes in one oracle sample (of 3 n_el)")
    ap.add_argument("--op", default="local_energy", choices=["local_energy", "grad", "mcmc", "spring", "ecp", "spin"],
                    help="local_energy: the headline metric; grad / mcmc / spring / ecp: the adjoint, the "
                         "sampler, the SPRING update and the non-local pseudopotential")
    ap.add_argument("--global-moves", type=int, default=0, help="--op mcmc: global jumps per sweep")
    ap.add_argument("--chain", type=int, default=26, help="--op mcmc: zigzag chain C_kH_{k+2}")
    ap.add_argument("--scan", action="store_true", help="--op mcmc: every chain k = 2, 8, ..., 44")
    ap.add_argument("--chains", default=None,
                    help="--op mcmc --scan: comma-separated chain lengths k instead of 2, 8, ..., 44")
    ap.add_argument("--sweeps", type=int, default=2, help="--op mcmc: sweeps per timed call")
    ap.add_argument("--no-stages", action="store_true",
                    help="--op mcmc: no extra profiled call for the stage times")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.op != "local_energy":
        return bench_other(args, rank, world, local)

    from paper_2504_06087_gb300 import fire, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)

    from paper_2504_06087_gb300 import replicas
    w = synth.workload("c26h24", args.walkers)
    # every rank evaluates its own block of a global seeded walker set
    r_all, p = synth.make_inputs(w, args.walkers * world)
    w0, _ = replicas.walker_block(args.walkers * world, rank, world)
    r_np = np.ascontiguousarray(r_all[w0:w0 + args.walkers])
    k_cap = 64
    f = fire.Fire(w.system, w.arch, p, args.precision, k_cap=k_cap, device=str(dev))
    r = torch.as_tensor(r_np, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            tdist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for _ in range(max(args.warmup, 0)):
        out = f.local_energy(r)
    torch.cuda.synchronize(dev)

    # timed region: device-resident inputs
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = f.local_energy(r)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    clocks = sampler.stop()
    info = out["info"]
    total_ms = float(sum(times))
    if dist:
        t = torch.tensor([total_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / max(args.steps, 1)
    value = world * args.walkers * args.steps / (total_ms / 1e3)

    # end to end through the public API: pinned host positions in, E_L out
    r_host = torch.as_tensor(r_np).pin_memory()
    e_host = torch.empty(args.walkers, dtype=torch.float64).pin_memory()
    e2e_times = []
    barrier()
    for k in range(max(1, min(args.steps, 2))):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rd = r_host.to(dev, non_blocking=True)
        o2 = f.local_energy(rd)
        e_host.copy_(o2["e_loc"], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = float(np.mean(e2e_times))
    if dist:
        t = torch.tensor([e2e_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": world * args.walkers / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(r_host.numel() * 8), "d2h_bytes_per_step": int(e_host.numel() * 8)}

    # the one cross-rank reduction of a VMC step: E_L moments (float64)
    moments = replicas.energy_moments(out["e_loc"])
    if rank != 0:
        if dist:
            tdist.barrier()
            tdist.destroy_process_group()
        return

    # one profiled call: per-stage device time (CUDA events on the call's stream)
    fire.profile(True)
    outp = f.local_energy(r)
    torch.cuda.synchronize(dev)
    stages = fire.profile_report()
    fire.profile(False)
    nb = f.neighbors(r)
    cnt = nb["cnt"].sum(-1).to(torch.float64)
    nbr_sq_sum = float(((1.0 + cnt) ** 2).sum().item())
    nbr_sum = float((1.0 + cnt).sum().item())
    peaks, peak_src = load_peaks()
    simt = simt_peaks(dev)
    dom = max(stages.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms) = dom
    flops, nbytes, bound = stage_work(dname, w, info, args.walkers, nbr_sq_sum, nbr_sum, args.precision)
    tkey = dname + ("_tc" if bound == "hbm" else "")
    traffic, traffic_src = stage_traffic(tkey, args.walkers * w.arch.n_det, dl)
    roof = {"kernel": dname, "share_of_step": dms / sum(v[1] for v in stages.values()), "launches": dl,
            "traffic": traffic, "traffic_source": traffic_src}
    if nbytes is not None:
        per_launch = nbytes / dl
        achieved = per_launch / (dms / dl / 1e3) / 1e9
        roof.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_source": f"HBM copy bandwidth, {peak_src}",
                     "bytes_per_launch": per_launch, "ms_per_launch": dms / dl})
    elif flops is not None:
        per_launch = flops / dl
        achieved = per_launch / (dms / dl / 1e3) / 1e12
        fp32_note = f"FP32 SIMT, measured in this run (FFMA probe, {simt['sm_count']} SMs)"
        if bound == "tensor":
            peak, pnote = peaks["bf16_tflops_sustained"], f"bf16 dense sustained, {peak_src}"
            if args.precision != "bf16":
                peak, pnote = simt["fp32_tflops"], fp32_note
        elif bound == "fp64":
            peak, pnote = simt["fp64_tflops"], f"FP64 SIMT, measured in this run (DFMA probe, {simt['sm_count']} SMs)"
        else:
            peak, pnote = simt["fp32_tflops"], fp32_note
        roof.update({"bound": "tensor" if bound == "tensor" else "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": pnote,
                     "flops_per_launch": per_launch, "ms_per_launch": dms / dl})
    roof["stages_ms"] = {k: round(v[1], 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1][1])}

    # accuracy of this form and of plain FP32 against the stored FP64 oracle values
    comparison = {}
    gpath = os.path.join(ROOT, "tests", "golden", "c26h24_oracle.json")
    forms = [args.precision] + ([] if args.no_compare or args.precision == "fp32" else ["fp32"])
    if os.path.exists(gpath):
        g = json.load(open(gpath))
        rg, pg = synth.make_inputs(w, g["n_walkers"])
        for prec in forms:
            fo = fire.Fire(w.system, w.arch, pg, prec, k_cap=k_cap, device=str(dev))
            oo = fo.local_energy(rg)
            e = oo["e_loc"].cpu().numpy()
            la = oo["logabs"].cpu().numpy()
            ref = np.asarray(g["e_loc"])
            comparison[prec] = {"e_loc_rel_err_max": float(np.max(np.abs(e - ref) / np.maximum(np.abs(ref), 1))),
                                "logabs_rel_err_max": float(np.max(np.abs(la - np.asarray(g["logabs"])) /
                                                                   np.maximum(np.abs(np.asarray(g["logabs"])), 1))),
                                "oracle_walkers": g["n_walkers"]}
    if not args.no_compare and args.precision != "fp32":
        f32 = fire.Fire(w.system, w.arch, p, "fp32", k_cap=k_cap, device=str(dev))
        f32.local_energy(r)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        f32.local_energy(r)
        e1.record(stream)
        e1.synchronize()
        comparison.setdefault("fp32", {})["value"] = args.walkers / (e0.elapsed_time(e1) / 1e3)
        del f32
    comparison.setdefault(args.precision, {})["value"] = value / world

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_baseline(w, args.oracle_coords)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16+f32+f64", "fp32": "f32", "fp64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"zigzag C26H24, n_el=180 (90 up/90 down), {args.walkers} walkers per GPU, "
                               "width 256, 4 MLP layers, 16 determinants, c=5 bohr, c_n=20 bohr, k_cap=64",
                   "precision": {"bf16": "bf16_fp64", "fp32": "fp32", "fp64": "fp64"}[args.precision],
                   "walkers_per_gpu": args.walkers, "l2": "flushed before every step (256 MB write)",
                   "parallelism": f"replicas x{world} (walker blocks, no data-path collective; one float64 "
                                  f"all-reduce of E_L moments after the timed calls)"},
        "e2e": e2e, "gpu_launches": int(info["n_launches"]) * args.steps,
        "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "comparison": comparison,
        "simt_peaks": simt,
        "diag": {"e_loc_moments_all_ranks": moments, "rows_total": info["rows_total"], "mean_neighbors": info["mean_neighbors"],
                 "k_required": info["k_required"], "n_chunks": info["n_chunks"], "n_nodes": info["n_nodes"],
                 "launches_per_step": info["n_launches"], "step_ms": times},
    }
    print(json.dumps(line), flush=True)
    if dist:
        tdist.barrier()
        tdist.destroy_process_group()


def oracle_sample(w, r1, p, coords):
    """One bounded sample of the oracle local energy on one walker: forward,
    gradient and `coords` of the 3 n_el second-derivative passes of its
    Laplacian.  Returns (seconds, seconds scaled to the full walker)."""
    from oracle import fire_oracle as O
    n = w.system.n_el
    pt = O.params_to_torch(p)
    t0 = time.perf_counter()
    r = torch.as_tensor(r1).clone().requires_grad_(True)
    la, _ = O.logpsi(w.system, w.arch, pt, r)
    (g,) = torch.autograd.grad(la.sum(), r, create_graph=True)
    t1 = time.perf_counter()
    lap = 0.0
    for q in range(coords):
        i, x = q // 3, q % 3
        (gg,) = torch.autograd.grad(g[:, i, x].sum(), r, retain_graph=True)
        lap += float(gg[0, i, x])
    with torch.no_grad():
        O.potential(w.system, r.detach())
    t2 = time.perf_counter()
    full = (t1 - t0) + (t2 - t1) * (3 * n) / coords
    return t2 - t0, full


def oracle_baseline(w, coords):
    from paper_2504_06087_gb300 import synth
    torch.set_num_threads(os.cpu_count() or 1)
    r1, p = synth.make_inputs(w, 1)
    oracle_sample(w, r1, p, 1)          # warm-up: thread pool, allocator, first graph build
    spent, full = oracle_sample(w, r1, p, coords)
    return {"value": 1.0 / full, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"1 walker of the same workload: forward, gradient and {coords} of the {3 * w.system.n_el} "
                      f"second-derivative passes of the FP64 dense oracle ({spent:.1f} s measured), time scaled "
                      f"to the full Laplacian"}


def reference_arm(args, rank, world):
    """The oracle, as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_2504_06087_gb300 import synth
    torch.set_num_threads(os.cpu_count() or 1)
    w = synth.workload("c26h24", args.walkers)
    r1, p = synth.make_inputs(w, 1)
    for _ in range(args.warmup):
        oracle_sample(w, r1, p, args.oracle_coords)
    tot = spent = 0.0
    for _ in range(args.steps):
        sp, full = oracle_sample(w, r1, p, args.oracle_coords)
        spent += sp
        tot += full
    value = args.steps / tot
    cpu = {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
           "sample": f"per step 1 walker: forward, gradient and {args.oracle_coords} of {3 * w.system.n_el} "
                     f"second-derivative passes ({1e3 * spent / args.steps:.0f} ms measured per step); the "
                     f"value scales the passes to the full Laplacian ({1e3 * tot / args.steps:.0f} ms per walker)"}
    # ms_per_step is the timed sample itself (what ran in each step); value is
    # the throughput of whole walkers extrapolated from it
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * spent / args.steps,
            "ms_per_walker_extrapolated": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "zigzag C26H24, n_el=180 (90 up/90 down), width 256, 4 MLP layers, "
                                   "16 determinants, c=5 bohr (FP64 dense CPU oracle)",
                       "precision": "fp64"},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



# ---------------------------------------------------------------------------
# the adjoint and the sampler (not the headline metric)
# ---------------------------------------------------------------------------

def _timed(fn, steps, warmup, dev):
    for _ in range(max(warmup, 0)):
        fn()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    times, outs = [], []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs.append(fn())
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, outs


def bench_other(args, rank, world, local):
    from paper_2504_06087_gb300 import fire, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    base = {"n_gpus": world, "steps": args.steps, "warmup": args.warmup, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    if args.op == "spring":
        return bench_spring(args, rank, dev, base)
    if args.op == "ecp":
        return bench_ecp(args, rank, dev, base)
    if args.op == "spin":
        return bench_spin(args, rank, dev, base)
    if args.op == "grad":
        w = synth.workload("c26h24", args.walkers)
        r_np, p = synth.make_inputs(w, args.walkers)
        f = fire.Fire(w.system, w.arch, p, "fp32", k_cap=64, device=str(dev))
        r = torch.as_tensor(r_np, device=dev)
        sampler = ClockSampler(local)
        sampler.start()
        times, outs = _timed(lambda: f.grad_logpsi(r)["info"], args.steps, args.warmup, dev)
        clocks = sampler.stop()
        fire.profile(True)
        f.grad_logpsi(r)
        torch.cuda.synchronize(dev)
        stages = fire.profile_report()
        fire.profile(False)
        ms = float(np.mean(times))
        simt = simt_peaks(dev)
        flops = grad_flops(w) * args.walkers
        out_bytes = 4.0 * args.walkers * f.n_params
        peaks, peak_src = load_peaks()
        achieved = flops / (ms / 1e3) / 1e12
        roof = {"kernel": "whole call (value forward with intermediates + adjoint)", "bound": "alu",
                "achieved": achieved, "peak": simt["fp32_tflops"], "unit": "TFLOP/s",
                "frac": achieved / simt["fp32_tflops"],
                "peak_source": f"FP32 SIMT, measured in this run (FFMA probe, {simt['sm_count']} SMs)",
                "flops_per_walker": grad_flops(w),
                "output_bytes": out_bytes, "output_write_ms_at_hbm_peak": out_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3,
                "note": "algorithmic FLOPs = 3x the multiply-adds of the value forward (forward, input adjoint, "
                        "weight adjoint of every product) x 2; every weight-gradient product runs on the SIMT pipe"}
        line = dict(base, metric="per-walker d log|Psi|/d theta evaluations/sec at n_el=180 (FP32 adjoint)",
                    value=args.walkers / (ms / 1e3), unit="walkers/s", ms_per_step=ms, higher_is_better=True,
                    dtype="f32+f64", config={"workload": f"zigzag C26H24, n_el=180, {args.walkers} walkers, "
                                                         f"{f.n_params} parameters, output [W, P] float32",
                                             "precision": "fp32 (float64 LU)"},
                    gpu_launches=int(outs[-1]["n_launches"]), clocks=clocks, roofline=roof,
                    stages_ms={k: round(v[1], 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1][1])})
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    chains = [args.chain]
    if args.scan:
        chains = [int(k) for k in args.chains.split(",")] if args.chains else [2, 8, 14, 20, 26, 32, 38, 44]
    pts = []
    for k in chains:
        w = synth.workload(f"sample_k{k}", args.walkers)
        r_np, p = synth.make_inputs(w, args.walkers)
        f = fire.Fire(w.system, w.arch, p, "fp32", k_cap=64, device=str(dev))
        r = torch.as_tensor(r_np, device=dev).contiguous()
        ctr = [0]

        def call():
            o = f.mcmc_step(r, 0.3, args.sweeps, refresh_every=32, seed=2504, counter=ctr[0],
                            n_global=args.global_moves, sigma_global=2.0)
            ctr[0] = o["counter"]
            return {kk: o[kk] for kk in ("n_accepted", "max_drift", "info", "walker_drift")}
        sampler = ClockSampler(local)
        sampler.start()
        times, outs = _timed(call, args.steps, args.warmup, dev)
        clocks = sampler.stop()
        stages = {}
        if not args.no_stages:
            fire.profile(True)
            call()
            torch.cuda.synchronize(dev)
            stages = fire.profile_report()
            fire.profile(False)
        n = w.system.n_el
        ms = float(np.mean(times))
        sweeps_s = args.sweeps / (ms / 1e3)
        acc = sum(o["n_accepted"] for o in outs) / (len(outs) * args.walkers * n * args.sweeps)
        drift = max(o["max_drift"] for o in outs)
        wd = torch.stack([o["walker_drift"] for o in outs]).max(0).values.cpu().numpy()
        dq = {"p50": float(np.percentile(wd, 50)), "p99": float(np.percentile(wd, 99)),
              "p999": float(np.percentile(wd, 99.9)), "max": float(wd.max()),
              "walkers_above_1e-2": int((wd > 1e-2).sum())}
        pts.append((n, 1.0 / sweeps_s))
        line = dict(base, metric=f"Metropolis sweeps/sec, zigzag C{k}H{k + 2} (n_el={n}), {args.walkers} walkers",
                    value=sweeps_s, unit="sweeps/s", ms_per_step=ms, higher_is_better=True, dtype="f32+f64",
                    config={"workload": f"zigzag C{k}H{k + 2}, n_el={n}, {args.walkers} walkers, width 256, 4 MLP "
                                        f"layers, 16 determinants, c=5 bohr, sigma=0.3 bohr single-electron moves, "
                                        f"float64 refresh every 32 moves; one step = one fire_mcmc_step call of "
                                        f"{args.sweeps} sweeps (with its start and end rebuilds)",
                            "precision": "fp32 state, float64 LU / ratios / refresh"},
                    s_per_sweep=1.0 / sweeps_s, acceptance=acc, max_drift=drift, drift_quantiles=dq,
                    gpu_launches=int(outs[-1]["info"]["n_launches"]), clocks=clocks,
                    stages_ms={kk: round(v[1], 3) for kk, v in sorted(stages.items(), key=lambda kv: -kv[1][1])})
        if rank == 0:
            print(json.dumps(line), flush=True)
        del f, r
        torch.cuda.empty_cache()
    if len(pts) > 2 and rank == 0:
        x = np.log([q[0] for q in pts])
        y = np.log([q[1] for q in pts])
        slope = float(np.polyfit(x, y, 1)[0])
        print(json.dumps({"metric": "fit: seconds per sweep ~ n_el^a", "a": slope,
                          "points": [{"n_el": q[0], "s_per_sweep": q[1]} for q in pts]}), flush=True)

def bench_spring(args, rank, dev, base):
    """One SPRING update (fire_spring_step) on the C26H24 workload: the
    gradient rows of 4096 walkers (fire_grad_logpsi, float32, 5.1 M
    parameters) and their local energies, computed once before timing."""
    from paper_2504_06087_gb300 import fire, synth
    w = synth.workload("c26h24", args.walkers)
    r_np, p = synth.make_inputs(w, args.walkers)
    r = torch.as_tensor(r_np, device=dev)
    f = fire.Fire(w.system, w.arch, p, "fp32", k_cap=64, device=str(dev))
    O = f.grad_logpsi(r)["grad"]
    del f
    torch.cuda.empty_cache()
    fb = fire.Fire(w.system, w.arch, p, "bf16", k_cap=64, device=str(dev))
    e = fb.local_energy(r)["e_loc"]
    del fb
    torch.cuda.empty_cache()
    N, P = O.shape
    d0 = torch.zeros(P, dtype=torch.float32, device=dev)
    state = {"d": d0}

    def step():
        out = fire.spring_step(O, e, state["d"], 0.99, 1e-3)
        state["d"] = out["delta"]
        return out["status"]
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    times, _ = _timed(step, args.steps, args.warmup, dev)
    clocks = sampler.stop()
    fire.profile(True)
    step()
    torch.cuda.synchronize(dev)
    stages = fire.profile_report()
    fire.profile(False)
    ms = float(np.mean(times))
    peaks, src = load_peaks()
    gram_flops = 2.0 * N * N * P
    line = dict(base, metric="SPRING updates/sec, C26H24 gradient rows (4096 walkers x 5.1 M parameters)",
                value=1e3 / ms, unit="updates/s", ms_per_step=ms, higher_is_better=True, dtype="f32+f64",
                config={"workload": f"zigzag C26H24, {N} walkers, {P} parameters, O [N, P] float32 from "
                                    f"fire_grad_logpsi, lambda=1e-3, eta=0.99",
                        "precision": "Gram matrix as six split-bf16 products (FP32 accumulation), float64 solve"},
                roofline={"kernel": "tc_gemm (Gram)", "bound": "tensor",
                          "achieved": gram_flops / (ms / 1e3) / 1e12,
                          "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                          "frac": gram_flops / (ms / 1e3) / 1e12 / peaks["bf16_tflops_sustained"],
                          "note": "algorithmic 2 N^2 P of the whole update time; the tensor cores execute six "
                                  f"split products of it; peak: bf16 dense sustained, {src}"},
                clocks=clocks, gpu_launches=None,
                stages_ms={k: round(v[1], 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1][1])})
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_ecp(args, rank, dev, base):
    """Non-local pseudopotential energy (fire_ecp_nonlocal) on C26H24 with a
    synthetic semi-local pseudopotential on every carbon (N_quad = 4,
    r_cut = 1.2 bohr, s and d channels)."""
    from paper_2504_06087_gb300 import fire, synth
    w = synth.workload("c26h24", args.walkers)
    r_np, p = synth.make_inputs(w, args.walkers)
    r = torch.as_tensor(r_np, device=dev)
    ecp = [{"n_quad": 4, "r_cut": 1.2, "terms": [[(4.0, 0, 1.0)], [], [(1.5, 0, 0.6)]]} if z == 6.0 else None
           for z in w.system.nuc_charge]
    f = fire.Fire(w.system, w.arch, p, "fp32", k_cap=64, device=str(dev))
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    times, outs = _timed(lambda: f.ecp_nonlocal(r, ecp, seed=5)["info"], args.steps, args.warmup, dev)
    clocks = sampler.stop()
    ms = float(np.mean(times))
    n = w.system.n_el
    line = dict(base, metric=f"non-local pseudopotential evaluations/sec, zigzag C26H24 (n_el={n}), "
                             f"{args.walkers} walkers, N_quad=4 on carbons",
                value=args.walkers / (ms / 1e3), unit="walkers/s", ms_per_step=ms, higher_is_better=True,
                dtype="f32+f64", config={"workload": f"zigzag C26H24, {args.walkers} walkers, synthetic "
                                                     "pseudopotential on the 26 carbons (s and d channels), "
                                                     f"{n} x 4 virtual single-electron moves per call",
                                         "precision": "fp32 state, float64 lemma and exact ratios"},
                s_per_virtual_move=ms / 1e3 / (n * 4), gpu_launches=int(outs[-1]["n_launches"]), clocks=clocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_spin(args, rank, dev, base):
    """S+ swap ratios (fire_spin_ratios) on C26H24: the last spin-down electron
    swapped with each of the 90 spin-up electrons, every walker."""
    from paper_2504_06087_gb300 import fire, synth
    w = synth.workload("c26h24", args.walkers)
    r_np, p = synth.make_inputs(w, args.walkers)
    r = torch.as_tensor(r_np, device=dev)
    f = fire.Fire(w.system, w.arch, p, "fp32", k_cap=64, device=str(dev))
    beta = w.system.n_el - 1
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    times, outs = _timed(lambda: f.spin_ratios(r, beta)["info"], args.steps, args.warmup, dev)
    clocks = sampler.stop()
    ms = float(np.mean(times))
    nu = w.system.n_up
    line = dict(base, metric=f"S+ swap-ratio evaluations/sec, zigzag C26H24 (n_el={w.system.n_el}), "
                             f"{args.walkers} walkers, {nu} swaps per walker",
                value=args.walkers / (ms / 1e3), unit="walkers/s", ms_per_step=ms, higher_is_better=True,
                dtype="f32+f64", config={"workload": f"zigzag C26H24, {args.walkers} walkers, beta = electron "
                                                     f"{beta}, {nu} two-electron swaps per walker",
                                         "precision": "fp32 state, float64 lemma and exact ratios"},
                s_per_swap=ms / 1e3 / nu, gpu_launches=int(outs[-1]["n_launches"]), clocks=clocks)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
