"""Benchmark of the semistochastic local-energy path on the H50-shaped chain.

One step = one nqs_local_energy call over the whole batch (environments,
enumeration and Slater-Condon H_nm, the eps split, Philox draws, amplitudes
of every deterministic and drawn determinant, the E_loc sums). Inputs are
synthetic (seeded), resident in HBM before the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the CPU oracle, bounded sample per step

Prints one JSON line (rank 0).
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

from paper_2507_19276_gb300 import shard  # noqa: E402
from paper_2507_19276_gb300 import workloads as W  # noqa: E402

METRIC = "E_loc samples/s (H50 shape)"
UNIT = "samples/s"

# workload -> (generator(n_samples, seed_offset), default samples per GPU,
# default precision, metric)
WORKLOADS = {
    "h50": (lambda n, o: W.h50_chain(n_samples=n, seed_offset=o), 4096, "mixed", METRIC),
    "k8": (lambda n, o: W.small_chain(n_samples=n, seed_offset=o), 256, "fp64",
           "E_loc samples/s (K8 chain, D=8, plain FP64)"),
    "fe2s2": (lambda n, o: W.fe2s2_dense(n_samples=n, seed_offset=o), 8192, "mixed",
              "E_loc samples/s (Fe2S2 shape, D=256)"),
    "h18": (lambda n, o: W.h18_graph(n_samples=n, seed_offset=o), 16384, "mixed",
            "E_loc samples/s (H18 graph, D=32)"),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def measured_ceilings(device, args):
    """L2 read and gather rates and CUDA-core FMA rates, measured on this GPU
    before the timed region (paper_2507_19276_gb300/peaks): the denominators of
    the enumeration and FP64 rooflines, which MEASURED_PEAKS.json does not hold."""
    if getattr(args, "no_peaks", False):
        return None
    from paper_2507_19276_gb300.peaks import probe
    return probe.measure(device)


def with_overrides(sys_, args):
    """The workload with the command line's eps / N_eps / uniform counts."""
    import dataclasses
    ch = {}
    if getattr(args, "eps", None) is not None:
        ch["eps"] = args.eps
    if getattr(args, "draws", None) is not None:
        ch["n_draws"] = args.draws
    if getattr(args, "uniform_counts", False):
        ch["counts"] = np.ones(len(sys_.samples))
    return dataclasses.replace(sys_, **ch) if ch else sys_


def time_gradient(ctx, sys_, samples, counts, prec, tol, base, dev):
    """The backward pass on the bench's batch (device buffers): the VJP alone
    (nqs_grad_log_psi_vjp with fixed weights) and the energy gradient
    (nqs_energy_gradient: E_loc, the weights on the device, the VJP), each
    timed once after one untimed call, with CUDA events; plus the VJP with the
    environments formed 1024 samples at a time (nqs_options.grad_chunk)."""
    import torch
    from paper_2507_19276_gb300 import nqs
    Ns = int(samples.shape[0])
    u = torch.from_numpy(np.random.default_rng(1).normal(size=Ns)).to(dev)
    NH, K, D, E = sys_.n_hidden, sys_.K, sys_.D, sys_.n_edges
    gT = torch.empty((E, 4, D, D), dtype=torch.float64, device=dev)
    gW = torch.empty((NH, 2 * K), dtype=torch.float64, device=dev) if NH else None
    gb = torch.empty(NH, dtype=torch.float64, device=dev) if NH else None
    st = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a.record(st)
        fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    out = {}
    for chunk in (0, 1024):
        ctx.set_precision(prec, timing=False, sample_index_base=base, energy_tolerance=tol, grad_chunk=chunk)
        out[f"vjp_ms{'_chunk1024' if chunk else ''}"] = timed(
            lambda: nqs.nqs_grad_log_psi_vjp(ctx.h, samples, u, Ns, gT, gW, gb))
    ctx.set_precision(prec, timing=False, sample_index_base=base, energy_tolerance=tol)
    e = torch.empty(Ns, dtype=torch.float64, device=dev)
    out["energy_gradient_ms"] = timed(lambda: nqs.nqs_energy_gradient(
        ctx.h, samples, counts, Ns, sys_.eps, sys_.n_draws, sys_.seed, 0, gT, gW, gb, None, e))
    out["vjp_samples_per_s"] = Ns / (out["vjp_ms"] / 1e3)
    # FP64 outer-product work of the site-tensor gradient: 2 D^2 per sample and edge
    out["vjp_flops"] = 2.0 * D * D * E * Ns
    return out


def enum_bytes(K, na, nb, n_samples, n_det):
    """Algorithmic bytes of the enumeration stage (Slater-Condon elements of
    every connected determinant, the eps split, the deterministic lists): per
    element the integral reads of its rule -- 8 B for a single (one Fock
    element per sample), 16 B for a same-spin double ((ai|bj) and (aj|bi)),
    8 B for an alpha-beta double -- and 12 B (rank + H) per listed entry."""
    c2 = lambda x: x * (x - 1) // 2
    singles = na * (K - na) + nb * (K - nb)
    same = c2(na) * c2(K - na) + c2(nb) * c2(K - nb)
    ab = na * (K - na) * nb * (K - nb)
    return n_samples * (8.0 * singles + 16.0 * same + 8.0 * ab) + 12.0 * n_det


# DRAM bytes (read + write) per evaluated amplitude of the amplitude stage,
# summed over its kernels, from ncu counters on the H50 shape (D = 64) with
# 512 samples; the stage's traffic grows in proportion to the amplitudes
# evaluated. None where not measured, or where the stage's kernels changed
# after the counters were taken (the mixed form's correlator factors, marks
# and row kernel have since; 328.5 B per amplitude was the earlier figure).
STAGE_TRAFFIC_PER_AMP = {"mixed": None, "fp64_shared": None}

DTYPES = {"mixed": "f16x3 tensor-core products (f32 accumulate) + f32 gathers; f64 H, ratios, sums; "
                   "psi(n) in double-f32; heaviest samples re-evaluated (f64, tables in double-f32) "
                   "to the energy tolerance",
          "fp64_shared": "f64", "fp64": "f64"}


THROTTLE_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def summarize_clocks(lines):
    """Median SM clock, the largest max clock and the throttle reasons seen in
    nvidia-smi CSV lines (index, clocks.sm, clocks.max.sm, power.draw,
    reasons.active, then the four reasons of THROTTLE_REASONS)."""
    sm, mx, reasons = [], [], set()
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(THROTTLE_REASONS, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
            "samples": len(sm)}


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        self.t.join(timeout=2)
        return summarize_clocks(self.lines)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(sys_, n_samples, threads):
    """The oracle, as it stands, on the first n_samples of the batch."""
    from oracle import oracle as O
    P = O.Problem(sys_.subset(range(n_samples)))
    t0 = time.perf_counter()
    O.local_energy(P, threads=threads)
    dt = time.perf_counter() - t0
    return n_samples / dt, dt


def workload_config(sys_, precision, ws=1, energy_tol=0.0):
    kind = "graph" if sys_.pred_ptr is not None else "chain"
    return {"workload": f"{sys_.name} {kind} K={sys_.K} {sys_.n_alpha}a+{sys_.n_beta}b D={sys_.D} "
                        f"N_h={sys_.n_hidden} Ns={len(sys_.samples)} per GPU eps={sys_.eps:g} "
                        f"N_eps={sys_.n_draws}",
            "K": sys_.K, "D": sys_.D, "n_hidden": sys_.n_hidden,
            "samples_per_gpu": len(sys_.samples), "global_batch": ws * len(sys_.samples),
            "eps": sys_.eps, "n_draws": sys_.n_draws, "precision": precision,
            "energy_tolerance_ha": energy_tol,
            "l2": "inputs > L2 (deterministic lists and shared-prefix tables exceed 129 MB)"
            if sys_.K >= 20 else "small case: working set may sit in L2"}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    if args.workload == "uneven":
        # the first samples of the first systems, one oracle call per system
        systems = [s.subset(range(2)) for s in W.uneven_batch()[:max(1, cores // 2)]]
        metric, sys_ = BATCH_METRIC, systems[0]
        per_step = sum(len(s.samples) for s in systems)

        def one_step():
            return sum(cpu_oracle_rate(s, len(s.samples), cores)[1] for s in systems)
    else:
        if args.workload == "h50_rnn":
            # the oracle has its own sampler; its E_loc is timed on uniform samples
            gen, n_def, metric = (lambda n, o: W.h50_rnn(n_samples=n, seed_offset=o)), 64, RNN_METRIC
        else:
            gen, n_def, _, metric = WORKLOADS[args.workload]
        sys_ = with_overrides(gen(args.samples or n_def, 0), args)
        per_step = min(len(sys_.samples), max(2, cores))

        def one_step():
            return cpu_oracle_rate(sys_, per_step, cores)[1]
    for _ in range(args.warmup):
        one_step()
    t = 0.0
    for _ in range(args.steps):
        t += one_step()
    v = per_step * args.steps / t
    line = {"impl": "reference", "metric": metric, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(sys_, "fp64-oracle"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} samples per step (the first of the workload's "
                                       f"batch{'es' if args.workload == 'uneven' else ''})"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run(args):
    import torch
    from paper_2507_19276_gb300 import nqs

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    live = measured_ceilings(local, args)
    # weak scaling: one batch of args.samples unique samples per GPU, split
    # contiguously; each shard's draws are keyed by global sample position
    gen, n_def, _, metric = WORKLOADS[args.workload]
    total = (args.samples or n_def) * ws
    lo, hi = shard.shard_range(total, ws, rank)
    sys_ = with_overrides(gen(total, 0), args).subset(range(lo, hi))
    Ns = len(sys_.samples)
    ctx = nqs.Context(local)
    ctx.set_system(sys_)
    prec = {"mixed": nqs.NQS_PREC_MIXED, "fp64": nqs.NQS_PREC_FP64,
            "fp64_shared": nqs.NQS_PREC_FP64_SHARED}[args.precision]
    tol = args.energy_tol if prec == nqs.NQS_PREC_MIXED else 0.0
    ctx.set_precision(prec, timing=True, sample_index_base=lo, energy_tolerance=tol,
                      tile_blocks_per_sm=args.tile_bps, table_mb=args.table_mb)

    samples = torch.from_numpy(sys_.samples.view(np.int64)).to(dev)
    counts = torch.from_numpy(sys_.counts).to(dev)
    e_loc = torch.empty(Ns, dtype=torch.float64, device=dev)

    def step(summary=None):
        if ws > 1 and summary is None:
            summary = nqs.EnergySummary()
        nqs.nqs_local_energy(ctx.h, samples, counts, Ns, sys_.eps, sys_.n_draws, sys_.seed, e_loc,
                             summary)
        if ws > 1:
            # the one exchange of the method: the weighted-energy sums
            return shard.allreduce(summary.as_dict(), device=dev)
        return None

    summ = nqs.EnergySummary()
    for _ in range(args.warmup):
        step(summ)
    torch.cuda.synchronize()
    ctx.stage_times()   # reset counters

    stream = torch.cuda.current_stream(dev)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)     # nvidia-smi's start-up (NVML init) stays outside the timed region
    barrier(ws)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        step()
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    ms = start.elapsed_time(stop)
    stages = ctx.stage_times()
    ms = max_over_ranks(ms, ws, dev)
    value = total * args.steps / (ms / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside
    hs = torch.from_numpy(sys_.samples.view(np.int64)).pin_memory()
    hc = torch.from_numpy(sys_.counts).pin_memory()
    he = torch.empty(Ns, dtype=torch.float64).pin_memory()
    nqs.nqs_local_energy(ctx.h, hs, hc, Ns, sys_.eps, sys_.n_draws, sys_.seed, he, None)
    torch.cuda.synchronize()
    ctx.stage_times()
    barrier(ws)
    t0 = time.perf_counter()
    start.record(stream)
    for _ in range(args.steps):
        nqs.nqs_local_energy(ctx.h, hs, hc, Ns, sys_.eps, sys_.n_draws, sys_.seed, he, None)
    stop.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max(start.elapsed_time(stop), 1e3 * (time.perf_counter() - t0))
    e2e_ms = max_over_ranks(e2e_ms, ws, dev)
    ctx.stage_times()

    # roofline of the amplitude contraction (the dominant stage)
    peaks, src = _peaks()
    work = summ.as_dict()
    n_amp = work["n_amplitudes"]
    D = sys_.D
    amp_ms = sum(stages[k][0] for k in ("tables", "amp_det", "amp_draw")) / args.steps
    amp_launches = sum(stages[k][1] for k in ("tables", "amp_det", "amp_draw")) / args.steps
    # the method's work per amplitude: one D x D product per site of the span
    # between the first and last changed site, plus the closing dot product
    # chains: D x D products over each amplitude's span; graphs: per in-edge
    # of every recomputed vertex (the plain form's matvecs)
    mv_alg = work["span_sites"] if sys_.pred_ptr is None else work["matvecs"]
    flops = 2.0 * D * D * mv_alg + 2.0 * D * n_amp
    executed = 2.0 * D * D * work["matvecs"] + 2.0 * D * n_amp
    achieved = flops / (amp_ms / 1e3) / 1e12
    graph = sys_.pred_ptr is not None
    if prec == nqs.NQS_PREC_MIXED:
        roof = {"bound": "tensor", "unit": "TFLOP/s", "achieved": achieved,
                "peak": peaks["bf16_tflops_sustained"],
                "peak_source": f"{src} dense bf16 (sustained; f16 has the same nominal rate)",
                "kernel": ("k_graph_tiles (tcgen05, 128-row tiles re-running the vertices from "
                           "each row's first change)" if graph else
                           "amplitude stage: k_fam_mark, k_fam_compact, k_site_boundary, "
                           "k_site_build, k_site_tiles_pipe (tcgen05), k_fam_rbm, k_fam_rows")}
    else:
        roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": achieved,
                "peak": live["fma64_tflops"] if live else 1.056,
                "peak_source": ("FP64 FMA rate measured before the timed region (peaks probe)" if live
                                else "FP64 FMA rate of an earlier peaks-probe run on a GB300"),
                "kernel": ("amplitude stage (shared prefixes, FP64)" if prec == nqs.NQS_PREC_FP64_SHARED
                           else "k_amp_chain_fp64 / k_amp_graph_fp64 (one amplitude per row)")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the same stage against the work the shared-prefix form executes
    roof["executed_frac"] = executed / (amp_ms / 1e3) / 1e12 / roof["peak"]
    # the row kernel (k_fam_rows, the largest share of the mixed step) against the
    # on-chip rate it is bound by: per row it gathers the left and right vectors
    # (D floats each) and, with a correlator, one factor row per side (N_h
    # rounded up to 4, plus the P - 1 group: 4 more floats)
    roof_rows = None
    if live and prec == nqs.NQS_PREC_MIXED and not graph:
        rows_ms = (stages["amp_det"][0] + stages["amp_draw"][0]) / args.steps
        NH = sys_.n_hidden
        per_row = 4.0 * (2 * D + (2 * (((NH + 3) // 4) * 4 + 4) if NH else 0))
        l2 = max(live["l2_read_gbs"].values())
        ach = per_row * n_amp / (rows_ms / 1e3) / 1e9
        roof_rows = {"bound": "l2", "unit": "GB/s", "achieved": ach, "peak": l2, "frac": ach / l2,
                     "peak_source": "L2 streaming read rate measured before the timed region (peaks probe)",
                     "kernel": "k_fam_rows (gathers of the left/right vectors and correlator rows)",
                     "bytes_per_row": per_row, "stage_ms_per_step": rows_ms, "traffic": None}
    # enumeration stage (count pass, write pass, draws): algorithmic integral
    # bytes against the measured L2 rates (the integral table is L2-resident)
    enum_ms = sum(stages[k][0] for k in ("count", "write", "draw")) / args.steps
    eb = enum_bytes(sys_.K, sys_.n_alpha, sys_.n_beta, Ns, work["n_det"])
    roof_enum = None
    if live and enum_ms > 0:
        eri_mb = 8 * sys_.K ** 4 / 2 ** 20
        l2 = max(live["l2_read_gbs"].values())
        g8 = live["gather8_gbs"]["64" if eri_mb > 32 else "32"]
        ach = eb / (enum_ms / 1e3) / 1e9
        roof_enum = {"bound": "l2", "unit": "GB/s", "achieved": ach, "peak": l2, "frac": ach / l2,
                     "peak_source": "L2 streaming read rate measured before the timed region "
                                    "(peaks probe, best over 16..96 MB)",
                     "gather8_peak": g8, "frac_of_gather8": ach / g8,
                     "hbm_peak": peaks["hbm_gbs"], "frac_of_hbm": ach / peaks["hbm_gbs"],
                     "traffic": None, "algorithmic_bytes_per_step": eb, "stage_ms_per_step": enum_ms,
                     "kernel": "enumeration stage: k_enum (count), k_write_dets, k_draws, k_dedup",
                     "eri_mb": eri_mb}
    key = args.precision if args.workload == "h50" else None
    roof["traffic"] = STAGE_TRAFFIC_PER_AMP.get(key, None)
    if roof["traffic"] is not None:
        roof["traffic"] *= n_amp
    roof.update({"algorithmic_flops_per_step": flops, "executed_flops_per_step": executed,
                 "stage_ms_per_step": amp_ms, "launches_per_step": amp_launches,
                 "span_sites_per_step": work["span_sites"], "matvecs_per_step": work["matvecs"]})

    # the FP64 GPU form on the same batch: its throughput and the energy difference
    fp64 = None
    if not args.no_fp64_compare and prec == nqs.NQS_PREC_MIXED:
        e_mixed = e_loc.clone()
        # the FP64 form of the same evaluation order: shared prefixes for chains,
        # the plain form for graphs
        cmp_name = "fp64" if graph else "fp64_shared"
        ctx.set_precision(nqs.NQS_PREC_FP64 if graph else nqs.NQS_PREC_FP64_SHARED, timing=False,
                          sample_index_base=lo)
        s64 = nqs.EnergySummary()
        step(s64)
        torch.cuda.synchronize()
        start.record(stream)
        step(s64)
        stop.record(stream)
        torch.cuda.synchronize()
        ms64 = start.elapsed_time(stop)
        d = (e_loc - e_mixed).abs()
        e64 = s64.as_dict()["e_mean"]
        # the mixed form without the FP64 re-evaluation: its energy error and time
        ctx.set_precision(nqs.NQS_PREC_MIXED, timing=False, sample_index_base=lo, energy_tolerance=0.0)
        s0 = nqs.EnergySummary()
        step(s0)
        torch.cuda.synchronize()
        start.record(stream)
        step(s0)
        stop.record(stream)
        torch.cuda.synchronize()
        ms0 = start.elapsed_time(stop)
        fp64 = {"precision": cmp_name, "value": total / (ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64,
                "e_mean_diff_ha": abs(e64 - work["e_mean"]),
                "e_mean_diff_unrefined_ha": abs(e64 - s0.as_dict()["e_mean"]),
                "mixed_unrefined_ms_per_step": ms0,
                "max_abs_diff_ha": float(d.max().item()),
                "median_abs_diff_ha": float(d.median().item()),
                "max_rel_diff": float((d / e_loc.abs().clamp_min(1e-300)).max().item())}

    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic", "config": workload_config(sys_, args.precision, ws, tol),
            "connected_dets_per_s": value * work["n_conn"],
            "amplitudes_per_s": ws * n_amp * args.steps / (ms / 1e3),
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "roofline": roof,
            "roofline_enum": roof_enum,
            "roofline_rows": roof_rows,
            "measured_ceilings": live,
            "fp64_gpu": fp64,
            "e2e": {"value": total * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": Ns * 16 + Ns * 8, "d2h_bytes_per_step": Ns * 8},
            "clocks": clk,
            "gpu_launches": int(sum(v[1] for v in stages.values())),
            "summary": {"e_mean": work["e_mean"], "n_det": work["n_det"],
                        "n_draw_unique": work["n_draw_unique"], "n_refined": work["n_refined"],
                        "e_error_bound_ha": work["e_error_bound"], "n_audited": work["n_audited"],
                        "audit_rel_error": work["audit_rel_error"], "error_factor": work["error_factor"]}}
    if args.grad:
        line["gradient"] = time_gradient(ctx, sys_, samples, counts, prec, tol, lo, dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n_cpu = max(2, min(cores, 16))
        rate, dt = cpu_oracle_rate(sys_, n_cpu, cores)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {n_cpu} of {Ns} samples ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


RNN_METRIC = "E_loc samples/s (H50 shape, BDG(1)-RNN chi=10, autoregressive samples)"


def run_rnn(args):
    """The paper's H50 setting of Fig. 3a (Sec. 4.1): the normalised BDG(1)-RNN
    readout at chi = 10, eps = 0.01, N_eps = 100. One step = nqs_sample of
    N_s draws (autoregressive, breadth first) + nqs_local_energy (FP64) over
    the unique samples with their counts; device buffers throughout."""
    import torch
    from paper_2507_19276_gb300 import nqs

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    live = measured_ceilings(local, args)
    sys_ = with_overrides(W.h50_rnn(n_samples=2, seed_offset=rank), args)
    n_draw = args.samples or 4096
    ctx = nqs.Context(local)
    ctx.set_system(sys_)
    ctx.set_precision(nqs.NQS_PREC_FP64, timing=True)
    smp = torch.empty((n_draw, 2), dtype=torch.int64, device=dev)
    cnt = torch.empty(n_draw, dtype=torch.float64, device=dev)
    e_loc = torch.empty(n_draw, dtype=torch.float64, device=dev)

    def step(k, summ=None):
        nu = nqs.nqs_sample(ctx.h, n_draw, sys_.seed + k, smp, cnt, n_draw)
        nqs.nqs_local_energy(ctx.h, smp, cnt, nu, sys_.eps, sys_.n_draws, sys_.seed, e_loc, summ)
        return nu

    summ = nqs.EnergySummary()
    for k in range(args.warmup):
        step(k, summ)
    torch.cuda.synchronize()
    ctx.stage_times()
    st = torch.cuda.current_stream(dev)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    barrier(ws)
    torch.cuda.synchronize()
    start.record(st)
    uniq = 0
    for k in range(args.steps):
        uniq += step(1000 + k)
    stop.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    ms = max_over_ranks(start.elapsed_time(stop), ws, dev)
    stages = ctx.stage_times()
    value = ws * uniq / (ms / 1e3)
    nu = step(0, summ)
    torch.cuda.synchronize()
    work = summ.as_dict()
    ctx.stage_times()
    # FP64 work of the amplitudes: per recomputed vertex four candidate cells
    # (2 D^2 each) and their weights (2 D each), plus the sampler's per-node cells
    D = sys_.D
    amp_ms = (stages["amp_det"][0] + stages["amp_draw"][0]) / args.steps
    flops = work["span_sites"] * (4 * 2.0 * D * D + 4 * 3.0 * D)
    peak = live["fma64_tflops"] if live else 1.056
    roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": flops / (amp_ms / 1e3) / 1e12, "peak": peak,
            "peak_source": "FP64 FMA rate measured before the timed region (peaks probe)" if live
            else "FP64 FMA rate of an earlier probe run on this pool's GB300",
            "kernel": "k_rnn_amp (normalised readout, FP64, one warp per row)", "traffic": None,
            "algorithmic_flops_per_step": flops, "stage_ms_per_step": amp_ms}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # end to end: the same step with host-side outputs (samples back to the host,
    # then E_loc through host buffers)
    hs = np.empty((n_draw, 2), np.uint64)
    hc = np.empty(n_draw, np.float64)
    he = np.empty(n_draw, np.float64)
    t0 = time.perf_counter()
    ue = 0
    for k in range(args.steps):
        n_u = nqs.nqs_sample(ctx.h, n_draw, sys_.seed + 2000 + k, hs, hc, n_draw)
        nqs.nqs_local_energy(ctx.h, hs[:n_u], hc[:n_u], n_u, sys_.eps, sys_.n_draws, sys_.seed, he, None)
        ue += n_u
    e2e_s = time.perf_counter() - t0
    line = {"metric": RNN_METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"h50_rnn chain K={sys_.K} {sys_.n_alpha}a+{sys_.n_beta}b BDG(1)-RNN "
                                   f"chi={D}, {n_draw} autoregressive draws per step, eps={sys_.eps:g} "
                                   f"N_eps={sys_.n_draws}",
                       "draws_per_step": n_draw, "unique_per_step": uniq / args.steps,
                       "l2": "inputs > L2 (deterministic lists exceed 129 MB)"},
            "draws_per_s": ws * n_draw * args.steps / (ms / 1e3),
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "roofline": roof, "measured_ceilings": live,
            "e2e": {"value": ws * ue / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 24 * n_draw,
                    "d2h_bytes_per_step": 32 * n_draw},
            "clocks": clk, "gpu_launches": int(sum(v[1] for v in stages.values())),
            "summary": {"e_mean": work["e_mean"], "n_det": work["n_det"], "unique": nu}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        hs0 = np.empty((n_draw, 2), np.uint64)
        hc0 = np.empty(n_draw, np.float64)
        n_u = nqs.nqs_sample(ctx.h, n_draw, sys_.seed, hs0, hc0, n_draw)
        sub = dataclasses_replace(sys_, samples=hs0[:min(4, n_u)].copy(), counts=hc0[:min(4, n_u)].copy())
        rate, dt = cpu_oracle_rate(sub, len(sub.samples), cores)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{len(sub.samples)} sampled determinants ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def dataclasses_replace(obj, **kw):
    import dataclasses
    return dataclasses.replace(obj, **kw)


BATCH_METRIC = "E_loc samples/s (64-system uneven batch, one call)"


def run_batch(args):
    """64 independent chains (K 12..40, D 16/32/64, 512..4096 samples each) in
    one nqs_local_energy_batch call per step, each system on its own context
    and stream. The step is timed with CUDA events on the current stream; the
    call returns only after every system's stream has finished."""
    import torch
    from paper_2507_19276_gb300 import nqs

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    systems = W.uneven_batch(seed_offset=rank)
    prec = {"mixed": nqs.NQS_PREC_MIXED, "fp64": nqs.NQS_PREC_FP64,
            "fp64_shared": nqs.NQS_PREC_FP64_SHARED}[args.precision]
    tol = args.energy_tol if prec == nqs.NQS_PREC_MIXED else 0.0
    streams, ctxs, dargs, hargs = [], [], [], []
    for s in systems:
        st = torch.cuda.Stream(dev)
        c = nqs.Context(local, stream=st.cuda_stream)
        c.set_system(s)
        c.set_precision(prec, timing=True, energy_tolerance=tol)
        streams.append(st)
        ctxs.append(c)
        common = {"eps": s.eps, "n_draws": s.n_draws, "seed": s.seed}
        dargs.append(dict(common, samples=torch.from_numpy(s.samples.view(np.int64)).to(dev),
                          counts=torch.from_numpy(s.counts).to(dev),
                          out=torch.empty(len(s.samples), dtype=torch.float64, device=dev)))
        hargs.append(dict(common, samples=s.samples, counts=s.counts,
                          out=np.empty(len(s.samples), np.float64)))
    n_total = sum(len(s.samples) for s in systems)

    # schedule and tiles from the autotuner (cached per workload signature)
    tuned = None
    if not args.no_autotune:
        from paper_2507_19276_gb300 import autotune
        cfg, entry = autotune.tune(ctxs, dargs, systems, prec, tol)
        args.workers = cfg["workers"]
        tuned = {"config": cfg, "trials": entry.get("trials", [])}
        for c in ctxs:
            c.set_precision(prec, timing=True, energy_tolerance=tol,
                            tile_blocks_per_sm=cfg["tile_blocks_per_sm"], table_mb=cfg["table_mb"])

    def step(a):
        return nqs.local_energy_batch(ctxs, a, n_workers=args.workers)

    res = None
    for _ in range(args.warmup):
        res = step(dargs)
    torch.cuda.synchronize()
    for c in ctxs:
        c.stage_times()
    stream = torch.cuda.current_stream(dev)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    barrier(ws)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(args.steps):
        res = step(dargs)
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    ms = max_over_ranks(start.elapsed_time(stop), ws, dev)
    stages = {}
    launches = 0
    for c in ctxs:
        for k, (t, n) in c.stage_times().items():
            stages[k] = stages.get(k, 0.0) + t / args.steps
            launches += n
    value = ws * n_total * args.steps / (ms / 1e3)

    # end to end with host buffers
    step(hargs)
    torch.cuda.synchronize()
    for c in ctxs:
        c.stage_times()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(hargs)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), ws, dev)
    for c in ctxs:
        c.stage_times()

    # energy gradient of every system in the same batch call (Eq. egrad)
    grad = None
    if args.grad:
        gargs = [dict(a, grad=True) for a in hargs]
        nqs.local_energy_batch(ctxs, gargs, n_workers=args.workers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nqs.local_energy_batch(ctxs, gargs, n_workers=args.workers)
        torch.cuda.synchronize()
        grad = {"ms_per_step": 1e3 * (time.perf_counter() - t0),
                "what": "E_loc + u_n on the device + FP64 VJP of every system, host buffers"}
        for c in ctxs:
            c.stage_times()

    # the FP64 shared-prefix form on the same batch: per-system weighted-energy differences
    fp64 = None
    if not args.no_fp64_compare and prec == nqs.NQS_PREC_MIXED:
        for c in ctxs:
            c.set_precision(nqs.NQS_PREC_FP64_SHARED)
        r64 = step(hargs)
        torch.cuda.synchronize()
        for c in ctxs:
            c.set_precision(nqs.NQS_PREC_MIXED, energy_tolerance=0.0)
        r0 = step(hargs)
        torch.cuda.synchronize()
        d = [abs(a[1]["e_mean"] - b[1]["e_mean"]) for a, b in zip(res, r64)]
        d0 = [abs(a[1]["e_mean"] - b[1]["e_mean"]) for a, b in zip(r0, r64)]
        fp64 = {"precision": "fp64_shared", "e_mean_diff_ha_max_over_systems": max(d),
                "e_mean_diff_ha_median": float(np.median(d)),
                "e_mean_diff_unrefined_ha_max": max(d0), "e_mean_diff_unrefined_ha_median": float(np.median(d0)),
                "n_refined_total": int(sum(r[1]["n_refined"] for r in res))}

    peaks, src = _peaks()
    flops = sum(2.0 * s.D * s.D * r[1]["span_sites"] + 2.0 * s.D * r[1]["n_amplitudes"]
                for s, r in zip(systems, res))
    executed = sum(2.0 * s.D * s.D * r[1]["matvecs"] + 2.0 * s.D * r[1]["n_amplitudes"]
                   for s, r in zip(systems, res))
    achieved = flops / (ms / args.steps / 1e3) / 1e12
    roof = {"bound": "tensor", "unit": "TFLOP/s", "achieved": achieved,
            "peak": peaks["bf16_tflops_sustained"],
            "peak_source": f"{src} dense bf16 (sustained; f16 has the same nominal rate)",
            "kernel": "whole batch step (all stages of 64 systems, overlapped on streams)",
            "frac": achieved / peaks["bf16_tflops_sustained"], "traffic": None,
            "algorithmic_flops_per_step": flops, "executed_flops_per_step": executed}
    Ks = [s.K for s in systems]
    line = {"metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": f"uneven_batch: 64 chains K {min(Ks)}..{max(Ks)}, D 16/32/64, "
                                   f"{n_total} samples per GPU, eps=1e-3, N_eps=1024",
                       "systems": len(systems), "samples_per_gpu": n_total,
                       "precision": args.precision, "energy_tolerance_ha": tol,
                       "workers": args.workers,
                       "l2": "inputs > L2 (deterministic lists exceed 129 MB)"},
            "connected_dets_per_s": ws * args.steps * sum(
                len(s.samples) * r[1]["n_conn"] for s, r in zip(systems, res)) / (ms / 1e3),
            "amplitudes_per_s": ws * args.steps * sum(r[1]["n_amplitudes"] for r in res) / (ms / 1e3),
            "stage_ms_per_step_summed_over_systems": stages,
            "roofline": roof,
            "e2e": {"value": ws * n_total * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": 24 * n_total, "d2h_bytes_per_step": 8 * n_total},
            "clocks": clk, "gpu_launches": int(launches),
            "autotune": tuned, "fp64_gpu": fp64, "energy_gradient": grad,
            "summary": {"n_refined": int(sum(r[1]["n_refined"] for r in res)),
                        "audit_rel_error_max": max(r[1]["audit_rel_error"] for r in res)}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sub_ = [s.subset(range(2)) for s in systems[:8]]
        t = sum(cpu_oracle_rate(s, 2, cores)[1] for s in sub_)
        line["cpu_baseline"] = {"value": 2 * len(sub_) / t, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": f"first 2 samples of the first "
                                                            f"{len(sub_)} systems ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="h50", choices=sorted(WORKLOADS) + ["uneven", "h50_rnn"],
                    help="h50 (default), k8, fe2s2, h18, uneven (64 systems in one batch call) or "
                         "h50_rnn (normalised BDG(1)-RNN, autoregressive samples)")
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64", "fp64_shared"],
                    help="default: the workload's (mixed for chains with D %% 16 == 0, fp64 otherwise)")
    ap.add_argument("--samples", type=int, default=None, help="samples per GPU (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--workers", type=int, default=8, help="host worker threads (uneven batch)")
    ap.add_argument("--energy-tol", type=float, default=1e-6,
                    help="mixed form: bound (Ha) on the weighted-energy error, met by "
                         "re-evaluating the heaviest samples in FP64 (0: none)")
    ap.add_argument("--eps", type=float, default=None,
                    help="deterministic threshold (default: the workload's; the paper's runs use 0.01)")
    ap.add_argument("--draws", type=int, default=None,
                    help="stochastic draws per sample (default: the workload's; the paper's runs use 100)")
    ap.add_argument("--uniform-counts", action="store_true",
                    help="every sample count 1 instead of the workload's Zipf counts")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the L2 / FMA ceilings measured before the timed region")
    ap.add_argument("--no-autotune", action="store_true",
                    help="uneven batch: default schedule instead of the autotuner's")
    ap.add_argument("--tile-bps", type=int, default=0,
                    help="site-tile blocks per SM (schedule only; 0: the library's default)")
    ap.add_argument("--table-mb", type=int, default=0,
                    help="cap (MiB) on one sample batch's shared-prefix tables (schedule only; 0: default)")
    ap.add_argument("--grad", action="store_true",
                    help="also time the energy gradient (uneven batch; h18 / h50_rnn workloads)")
    ap.add_argument("--peaks", action="store_true",
                    help="print the measured ceilings (L2 read, random gathers, FMA) and exit")
    args = ap.parse_args()
    if args.peaks:
        from paper_2507_19276_gb300.peaks import probe
        print(json.dumps(probe.measure(0)), flush=True)
        return
    if args.precision is None:
        args.precision = {"uneven": "mixed", "h50_rnn": "fp64"}.get(args.workload) or \
            WORKLOADS[args.workload][2]
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_batch(args)
    elif args.workload == "h50_rnn":
        run_rnn(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
