"""Benchmark of the Lanczos / mTPQ hot path on one GB300 (or N independent replicas).

Default workload: the spin-1/2 Heisenberg model (J = 1) on the 6x6 periodic square lattice in
its S^z = 0 sector, dimension C(36,18) = 9,075,135,300 (more rows than 2^32), fp64 vectors.  One
benchmark step is one hphi_lanczos_run of 20 Lanczos steps from a seeded random start
(section 3.4: start vector, fused H v + vector-update steps, fp64 tridiagonal eigensolve,
energies on the host); the workload's own run has 100 steps (`--lanczos-steps 100`).  Metric:
H v throughput of the Lanczos loop in Gelem/s (rows x Lanczos steps per second), with Lanczos
steps/s, the roofline of the fused H v group against HBM and against the fp64 pipe, the same
run through the public API with the start vector copied from pinned host memory (e2e), the
mixed form (fp32 vectors, fp64 reductions, fp64 Ritz vector + Rayleigh-quotient refinement)
against fp64, and the 4x4 Hubbard Lanczos line.

Timing: W untimed warm-up steps, then K steps between CUDA events on the launching stream,
barrier + synchronize on both sides, max over ranks.  Vectors (73 GB each) exceed the 129 MB L2,
so no flush is needed.  `--impl reference` times the CPU oracle instead (the only other place
this file runs oracle code), on a bounded sample of rows of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "H·v Gelem/s & %HBM peak; Lanczos/mTPQ steps/s, FP64 vs mixed+batched at ΔE"
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per fused H v launch group from an ncu capture of the current
# kernels, with where they come from; absent where no capture of the current kernels exists
MEASURED_TRAFFIC = {("heisenberg_6x6_sz0", "fp64"): (1_001_300_000_000, "ncu capture at full size (1-pass DRAM "
                                                       "counters): k_sec_hi + k_sec_lo of one step after the "
                                                       "first, split (15, 2), 1 KB pass-H stripes")}
# fp64 FMA throughput of this machine's GB300 from a throughput probe (thread-level T op/s); the
# chip issues fp64 at 1/64 of its fp32 rate
FP64_PEAK_TOPS = 0.50


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
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
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if os.environ.get("HPHI_BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Replicas: every rank processes the same units; the job's rate is all units over the
    slowest rank's time (seconds = max over ranks), in giga-units per second."""
    return world * units_per_rank / seconds / 1e9


def l2_note(vector_bytes: int) -> str:
    if vector_bytes > 129e6:
        return f"vectors ({vector_bytes / 1e9:.2f} GB) exceed the 129 MB L2; no flush"
    return f"vectors ({vector_bytes / 1e6:.2f} MB) fit in L2: on-chip workload, no flush"


def hv_group_name(spec, m, prec, nvec, what):
    """The kernels of one fused H v launch group, as the library picks them."""
    import paper_1703_03637_gb300 as hp
    kind = "spin" if spec.kind == wl.SPIN else "hubbard"
    if kind == "hubbard" and not m.is_complex:
        ks = "k_maxexp + k_quant + k_hub_dn + k_hub_up_q" if prec == hp.FP64 else "k_hub_dn + k_hub_up"
    elif kind == "spin" and spec.basis == wl.BASIS_FULL and nvec in (32, 64, 128, 256):
        ks = "k_maxexp_cols + k_quant_cols + k_hv_batch" if prec == hp.FP64 else "k_hv_batch"
    else:
        ks = "k_hv_hub" if kind == "hubbard" else "k_hv_spin"
    return f"{ks} ({what})"


# ----------------------------------------------------------------------------- CPU oracle timing
def oracle_rows_per_s(spec, target_s: float = 12.0, max_rows: int = 4_000_000):
    """Oracle H v over a slice of rows of the workload, all host cores; rows per second."""
    import oracle
    D = oracle.dim(spec)
    rng = np.random.default_rng(0)
    v = np.empty(D, dtype=np.complex128)
    v.real = rng.standard_normal(D)
    v.imag = 0.0
    n = min(20000, D)
    max_rows = min(max_rows, D)
    t0 = time.perf_counter()
    oracle.apply_H_slice(spec, v, 0, n)
    dt = time.perf_counter() - t0
    n2 = int(min(max_rows, max(n, n * target_s / max(dt, 1e-6))))
    r0 = (D - n2) // 2
    t0 = time.perf_counter()
    oracle.apply_H_slice(spec, v, r0, n2)
    dt2 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    return n2 / dt2, n2, dt2, cores


def oracle_sampled_rows_per_s(spec, target_s: float = 12.0, max_rows: int = 2_000_000, seed: int = 777):
    """Oracle H v on randomly sampled rows of a workload too large for a host copy of the vector:
    every input element a row needs is regenerated from its Philox index (the oracle's
    or_apply_H_rows_philox), all host cores; rows per second."""
    import oracle
    D = oracle.dim(spec)
    rng = np.random.default_rng(1)
    n = 20000
    rows = np.sort(rng.integers(0, D, size=n)).astype(np.uint64)
    t0 = time.perf_counter()
    oracle.apply_H_rows_philox(spec, rows, seed, False)
    dt = time.perf_counter() - t0
    n2 = int(min(max_rows, max(n, n * target_s / max(dt, 1e-6))))
    rows = np.sort(rng.integers(0, D, size=n2)).astype(np.uint64)
    t0 = time.perf_counter()
    oracle.apply_H_rows_philox(spec, rows, seed, False)
    dt2 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    return n2 / dt2, n2, dt2, cores


def oracle_baseline(spec, target_s: float = 12.0):
    """CPU baseline of one H v row in Gelem/s with the sample it was measured on."""
    import oracle
    D = oracle.dim(spec)
    if D * 16 <= 16e9:
        rps, n, dt, cores = oracle_rows_per_s(spec, target_s)
        sample = (f"oracle H v on {n} contiguous rows of the same basis ({dt:.1f} s, OpenMP over {cores} host "
                  f"threads); a Lanczos step is one such H v per row")
    else:
        rps, n, dt, cores = oracle_sampled_rows_per_s(spec, target_s)
        sample = (f"oracle H v on {n} randomly sampled rows, input elements regenerated from the Philox "
                  f"definition of the start vector ({dt:.1f} s, OpenMP over {cores} host threads); a Lanczos "
                  f"step is one such H v per row")
    return {"value": round(rps / 1e9, 6), "unit": "Gelem/s", "cores": cores, "kind": "oracle", "sample": sample}


# ----------------------------------------------------------------------------- main
def pinned_gaussian(D, seed, complex_=False, chunk=1 << 27):
    """A seeded Gaussian start vector in pinned host memory, drawn on the device chunk by chunk
    (torch's generator; any Gaussian vector serves as a Lanczos start) and copied out."""
    import torch
    dt = torch.complex128 if complex_ else torch.float64
    host = torch.empty(D, dtype=dt, pin_memory=True)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for c in range(0, D, chunk):
        n = min(chunk, D - c)
        host[c:c + n].copy_(torch.randn(n, dtype=dt, device="cuda", generator=g))
    torch.cuda.synchronize()
    return host


def run_e2e_lanczos(m, D, seed, steps, prec, args, world, v0_host=None):
    """The same Lanczos run through the public API with the start vector in pinned host memory:
    every step copies it in (the library's own copy into its first Lanczos vector, so no device
    copy of it is held beside the workspace) and reads the energies and coefficients back;
    rows x steps per second."""
    import torch
    if v0_host is None:
        v0_host = pinned_gaussian(D, seed, m.is_complex)
    m.lanczos(steps, prec=prec, v0=v0_host, v0_on_host=True)  # untimed: the host-copy path warm
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        r = m.lanczos(steps, prec=prec, v0=v0_host, v0_on_host=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    out = {"value": round(whole_job_rate(D * steps * e2e_steps, world, e2e_s), 4), "unit": "Gelem/s",
           "h2d_bytes_per_step": int(v0_host.numel() * v0_host.element_size()),
           "d2h_bytes_per_step": int(8 * (2 * steps + 8 + 4)), "steps": e2e_steps, "e0": r["eig"][0],
           "start": "pinned host vector copied in by hphi_lanczos_run (v0_on_host)"}
    del v0_host
    return out


# Lanczos steps per benchmark step where the workload's own run is too long for a few-minute
# benchmark (the 6x6 sector's 100-step fp64 run takes about a minute)
BENCH_LANCZOS_STEPS = {"heisenberg_6x6_sz0": 20}
# fp64-pipe operations per row of the fused Lanczos pass 1 of the split-row fp64 path, counted
# from k_sec_lo's folded epilogue with an integral diagonal (the Heisenberg workloads): the
# int64 -> fp64 conversion of the element and the update c1 hv - c2 P (one multiply, one FMA);
# the element itself and <C, H C> are integer arithmetic
SEC_FP64_OPS_PER_ROW = 3


def host_ram_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError, AttributeError):
        return 0


def timed_lanczos(m, steps, prec, seed, args, world, local, rank, refine=False, n=None, profile=True):
    """W warm-up runs then n timed runs (CUDA events on the current stream, barrier + sync on both
    sides, max over ranks); eager launches with an event pair around every fused H v group, or
    (profile=False: runs whose whole recurrence is one kernel) graph launches, the per-step
    device time then being the run's device time over its steps."""
    import torch
    n = n or args.steps
    for _ in range(args.warmup):
        m.lanczos(steps, prec=prec, seed=seed, profile=profile, refine=refine)
    stream = torch.cuda.current_stream()
    clk = Clocks(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hv_ms, hv_n, launches, res = 0.0, 0, 0, None
    e0.record(stream)
    for _ in range(n):
        res = m.lanczos(steps, prec=prec, seed=seed, profile=profile, refine=refine)
        if profile:
            hv_ms += res["hv_ms"]
            hv_n += res["hv_launches"]
        else:
            hv_ms += res["ms"]
            hv_n += res["steps"]
        launches += res["launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop() if clk else None
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    return dict(ms=ms, hv_avg_ms=hv_ms / max(hv_n, 1), launches=launches, res=res, clocks=clocks, n=n)


def run_ours(args, world, rank, local):
    import torch
    import paper_1703_03637_gb300 as hp

    torch.cuda.set_device(local)
    W = wl.workload(args.workload)
    spec = W["model"]
    steps = args.lanczos_steps or BENCH_LANCZOS_STEPS.get(args.workload, W["steps"])
    prec = hp.FP64 if args.prec == "fp64" else hp.FP32
    seed = wl.START_SEED + rank
    m = hp.Model.from_spec(spec)
    D = m.dim
    esz = (8 if prec == hp.FP64 else 4) * (2 if m.is_complex else 1)
    # end-to-end input: a start vector in pinned host memory, made before the workspace exists
    host_v0 = None
    e2e_note = None
    if args.e2e:
        need = D * 8 * (2 if m.is_complex else 1)
        if need * 1.3 < host_ram_bytes():
            host_v0 = pinned_gaussian(D, seed, m.is_complex)
            torch.cuda.empty_cache()
        else:
            e2e_note = f"not run: a {need / 1e9:.0f} GB pinned start vector does not fit the host memory"
    # untimed set-up: the launch shapes of both precisions
    tune = None
    if args.split:
        L, K = (int(x) for x in args.split.split(","))
        m.set_sector_split(prec, L, K)
    elif args.autotune:
        tune = {"fp64" if prec == hp.FP64 else "fp32": m.autotune(prec)}
        if args.mixed and prec == hp.FP64:
            tune["fp32"] = m.autotune(hp.FP32)
    m.release_workspace()
    # a real spin model of at most 32,768 rows runs the whole recurrence in one thread-block
    # cluster (k_lz_cl), which only graph-launched (unprofiled) runs take
    one_cluster = prec == hp.FP64 and spec.kind == wl.SPIN and not m.is_complex and D <= 32768
    t = timed_lanczos(m, steps, prec, seed, args, world, local, rank, profile=not one_cluster)
    t["one_cluster"] = one_cluster
    ms_step = t["ms"] / t["n"]
    res = t["res"]
    value = whole_job_rate(D * steps * t["n"], world, t["ms"] / 1e3)
    e2e = None
    if host_v0 is not None:
        e2e = run_e2e_lanczos(m, D, seed, steps, prec, args, world, host_v0)
        del host_v0
    # mixed precision (fp32 vectors, fp64 reductions) + fp64 Ritz vector and Rayleigh quotient
    mixed = None
    if args.mixed and prec == hp.FP64:
        m.release_workspace()
        a = argparse.Namespace(**vars(args))
        a.warmup = 1
        tm = timed_lanczos(m, steps, hp.FP32, seed, a, world, local, rank, refine=True, n=1)
        rm = tm["res"]
        e64 = float(res["eig"][0])
        ms_mix = tm["ms"]
        mixed = {"value": round(whole_job_rate(D * steps, world, ms_mix / 1e3), 4), "unit": "Gelem/s",
                 "ms_per_step": round(ms_mix, 3), "lanczos_steps_per_s": round(steps / (ms_mix / 1e3), 3),
                 "includes": "fp32 Lanczos + fp64 Ritz vector (stored basis if it fits in 60% of free HBM, "
                             "else a replayed second pass), fp64 H x, Rayleigh quotient, residual",
                 "e_refined": rm["e_refined"], "e_fp64": e64, "e_fp32_ritz": float(rm["eig"][0]),
                 "rel_energy_diff_vs_fp64": abs(rm["e_refined"] - e64) / abs(e64),
                 "residual": rm["residual"], "speedup_vs_fp64": round(ms_step / ms_mix, 3),
                 "fused_hv_ms": round(tm["hv_avg_ms"], 3)}
    m.release_workspace()
    m.close()
    torch.cuda.empty_cache()
    sub = run_hubbard_sub(args, world, local, rank) if (args.sub and args.workload != "hubbard_4x4_8u8d") else None
    if rank != 0:
        return None
    out = assemble_lanczos_line(args, world, spec, D, steps, prec, esz, value, ms_step, t, e2e, e2e_note, mixed, tune)
    if sub is not None:
        out["hubbard_4x4_8u8d"] = sub
    return out


def hv_group_kernels(spec, m, prec):
    """The kernels of one fused Lanczos pass-1 launch group, as the library picks them."""
    import paper_1703_03637_gb300 as hp
    if spec.kind == wl.SPIN and spec.basis == wl.BASIS_SZ and not m.is_complex:
        if prec == hp.FP64:
            return ("k_sec_hi + k_sec_lo (split-row H v fused with Lanczos pass 1, on the int64 copy that the "
                    "previous pass 2 wrote; k_maxexp + k_quant in the first step only)")
        return "k_sec_hi + k_sec_lo (split-row H v fused with Lanczos pass 1)"
    if spec.kind == wl.HUBBARD and not m.is_complex and prec == hp.FP64:
        return ("k_hub_dn + k_hub_up_q (two-pass H v fused with Lanczos pass 1, on the int64 copy that the "
                "previous pass 2 wrote; k_maxexp + k_quant in the first step only)")
    return hv_group_name(spec, m, prec, 1, "Lanczos pass 1")


def assemble_lanczos_line(args, world, spec, D, steps, prec, esz, value, ms_step, t, e2e, e2e_note, mixed, tune):
    import paper_1703_03637_gb300 as hp
    hbm, src = peaks()
    bytes_row = 3 * esz   # fused H v + Lanczos pass 1: read C once, read P, write P
    hv_avg_ms = t["hv_avg_ms"]
    achieved = D * bytes_row / (hv_avg_ms / 1e3) / 1e9
    traffic = MEASURED_TRAFFIC.get((args.workload, args.prec))
    note = "no ncu capture of this kernel version"
    cols = ((tune or {}).get(args.prec) or {}).get("split_hi_cols")
    if traffic and args.workload == "heisenberg_6x6_sz0" and cols not in (None, 0, 4):
        traffic, note = None, f"captured at 4 pass-H columns per lane; this run uses {cols}"
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic[0] if traffic else None,
            "traffic_source": traffic[1] if traffic else note,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6.8 TB/s",
            "kernel": hv_group_kernels(spec, hp_model_stub(spec), prec), "kernel_avg_ms": round(hv_avg_ms, 4),
            "algorithmic_bytes_per_launch": D * bytes_row}
    if t.get("one_cluster"):
        roof["kernel"] = ("k_lz_cl: the whole recurrence in one 16-CTA cluster, both vectors in distributed "
                          "shared memory (on chip); kernel_avg_ms is the run's device time per step")
    if prec == hp.FP64 and spec.kind == wl.SPIN and spec.basis == wl.BASIS_SZ:
        ops = SEC_FP64_OPS_PER_ROW * D
        roof["fp64_pipe"] = {"ops_per_row": SEC_FP64_OPS_PER_ROW, "achieved_tops": round(ops / (hv_avg_ms / 1e3) / 1e12, 4),
                             "peak_tops": FP64_PEAK_TOPS, "frac": round(ops / (hv_avg_ms / 1e3) / 1e12 / FP64_PEAK_TOPS, 4),
                             "peak_source": "fp64 FMA throughput probe on this pool's GB300 (DFMA 0.50 T thread-op/s; "
                                            "int64->fp64 conversions 0.60 T/s)"}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == hp.FP64 else "f32+f64acc", "data": "synthetic",
        "config": {"workload": args.workload, "dim": D, "lanczos_steps_per_bench_step": steps,
                   "workload_lanczos_steps": wl.workload(args.workload)["steps"], "model": spec.name,
                   "sector": {0: "full", 1: f"S^z: n_up={spec.n_a}", 2: f"N_up={spec.n_a}, N_dn={spec.n_b}"}[spec.basis],
                   "start": "philox gaussian, seed 123432+rank, generated inside each bench step",
                   "l2": l2_note(D * esz), "parallelism": f"replicas{world}"},
        "lanczos_steps_per_s": round(steps / (ms_step / 1e3), 3),
        "e0": t["res"]["eig"][0], "roofline": roof, "e2e": e2e, "gpu_launches": t["launches"], "clocks": t["clocks"],
    }
    if e2e is None and e2e_note:
        out["e2e_note"] = e2e_note
    if mixed is not None:
        out["mixed"] = mixed
    if tune is not None:
        out["autotune"] = tune
    if args.cpu_baseline:
        out["cpu_baseline"] = oracle_baseline(spec)
    return out


def hp_model_stub(spec):
    """The is_complex flag hv_group_name needs, without building a model."""
    class _S:
        is_complex = spec.is_complex
    return _S()


def run_hubbard_sub(args, world, local, rank):
    """The 4x4 Hubbard Lanczos line (200 fp64 steps per run, autotuned two-pass kernels) as a
    sub-object of the default line."""
    import torch
    import paper_1703_03637_gb300 as hp
    W = wl.workload("hubbard_4x4_8u8d")
    spec = W["model"]
    m = hp.Model.from_spec(spec)
    D = m.dim
    tune = m.autotune(hp.FP64)
    t = timed_lanczos(m, W["steps"], hp.FP64, wl.START_SEED, args, world, local, rank)
    m.close()
    torch.cuda.empty_cache()
    hbm, _ = peaks()
    ms_step = t["ms"] / t["n"]
    achieved = D * 24 / (t["hv_avg_ms"] / 1e3) / 1e9
    traffic = MEASURED_TRAFFIC.get(("hubbard_4x4_8u8d", "fp64"))
    return {"value": round(whole_job_rate(D * W["steps"] * t["n"], world, t["ms"] / 1e3), 4), "unit": "Gelem/s",
            "ms_per_step": round(ms_step, 3), "lanczos_steps": W["steps"],
            "lanczos_steps_per_s": round(W["steps"] / (ms_step / 1e3), 2), "e0": t["res"]["eig"][0],
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "traffic": traffic[0] if traffic else None,
                         "kernel": "k_hub_dn + k_hub_up_q (Lanczos pass 1; k_maxexp + k_quant in the first step only)",
                         "kernel_avg_ms": round(t["hv_avg_ms"], 4), "algorithmic_bytes_per_launch": D * 24},
            "autotune": tune, "gpu_launches": t["launches"], "clocks": t["clocks"]}


def run_tpq(args, world, rank, local):
    """mTPQ on the 64-start Kitaev cluster: one benchmark step is one hphi_tpq_run of `iters`
    multiplications by (l - H/N_s) for all starts (a bounded slice of the 1000-step run: every
    multiplication costs the same)."""
    import torch
    import paper_1703_03637_gb300 as hp

    torch.cuda.set_device(local)
    W = wl.workload(args.workload)
    spec, K, nv = W["model"], (args.lanczos_steps or 20), W["n_starts"]
    prec = hp.FP64 if args.prec == "fp64" else hp.FP32
    m = hp.Model.from_spec(spec)
    D = m.dim
    esz = (8 if prec == hp.FP64 else 4) * (2 if m.is_complex else 1)
    seed = wl.START_SEED + 1000 * rank
    for _ in range(args.warmup):
        m.tpq(nv, K, l=W["l"], prec=prec, seed=seed, profile=True)
    stream = torch.cuda.current_stream()
    clk = Clocks(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hv_ms, hv_n, launches, res = 0.0, 0, 0, None
    e0.record(stream)
    for _ in range(args.steps):
        res = m.tpq(nv, K, l=W["l"], prec=prec, seed=seed, profile=True)
        hv_ms += res["hv_ms"]
        hv_n += res["hv_launches"]
        launches += res["launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop() if clk else None
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    units = D * nv * K  # row x start elements multiplied per benchmark step
    value = whole_job_rate(units * args.steps, world, ms / 1e3)

    # end to end: the fp64 start block from pinned host memory, records back to the host
    if D * nv > (1 << 28):  # drawn on the device chunk by chunk and copied out
        psi_host = pinned_gaussian(D * nv, seed, m.is_complex).view(D, nv)
    else:
        psi_host = torch.from_numpy(wl.gaussian_vector(seed, D, nv, complex_=m.is_complex)).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(1):
        psi_dev = psi_host.to("cuda", non_blocking=True)
        m.tpq(nv, K, l=W["l"], prec=prec, psi0=psi_dev)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": whole_job_rate(units, world, e2e_s), "unit": "Gelem/s",
           "h2d_bytes_per_step": int(psi_host.numel() * psi_host.element_size()),
           "d2h_bytes_per_step": int(3 * 8 * K * nv)}
    del psi_host
    if rank != 0:
        return None
    hbm, src = peaks()
    bytes_elem = 2 * esz  # fused H v + TPQ update: gather-read X once, write X_{k+1}
    hv_avg_ms = hv_ms / max(hv_n, 1)
    achieved = D * nv * bytes_elem / (hv_avg_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": None, "peak_source": src,
            "kernel": hv_group_name(spec, m, prec, nv, "mTPQ step"), "kernel_avg_ms": round(hv_avg_ms, 4),
            "algorithmic_bytes_per_launch": D * nv * bytes_elem}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ("c128" if prec == hp.FP64 else "c64+f64acc") if m.is_complex else
        ("f64" if prec == hp.FP64 else "f32+f64acc"), "data": "synthetic",
        "config": {"workload": args.workload, "dim": D, "n_starts": nv, "tpq_steps_per_run": K, "l": W["l"],
                   "model": spec.name, "start": "philox gaussian, seed 123432+1000*rank",
                   "l2": l2_note(D * nv * esz), "parallelism": f"replicas{world}"},
        "tpq_steps_per_s": round(K * args.steps / (ms / 1e3), 3),
        "u_last_mean": float(np.mean(res["u"][-1])), "roofline": roof, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks,
    }
    if args.cpu_baseline:
        if D * 16 <= 16e9:
            rps, n, dt, cores = oracle_rows_per_s(spec)
            sample = (f"oracle H v on {n} contiguous rows, one start ({dt:.1f} s, OpenMP over {cores} host "
                      f"threads); an mTPQ step is one such H v per row and start")
        else:
            rps, n, dt, cores = oracle_sampled_rows_per_s(spec)
            sample = (f"oracle H v on {n} randomly sampled rows, input elements regenerated from the Philox "
                      f"definition of the start vector ({dt:.1f} s, OpenMP over {cores} host threads); an "
                      f"mTPQ step is one such H v per row and start")
        out["cpu_baseline"] = {"value": round(rps / 1e9, 6), "unit": "Gelem/s", "cores": cores, "kind": "oracle",
                               "sample": sample}
    return out


def run_sectors(args, world, rank, local):
    """Lanczos in every S^z sector of the 28-site J1-J2 ring, all sectors as parallel branches
    of one CUDA graph; one benchmark step is one hphi_lanczos_run_sectors call."""
    import torch
    import paper_1703_03637_gb300 as hp

    torch.cuda.set_device(local)
    W = wl.workload(args.workload)
    spec, steps, sectors = W["model"], (args.lanczos_steps or W["steps"]), W["sectors"]
    prec = hp.FP64 if args.prec == "fp64" else hp.FP32
    refine = prec == hp.FP32
    m = hp.Model.from_spec(spec)
    seed = wl.START_SEED + rank
    # untimed: the split-row shape of every sector of at least 2^20 rows
    tune = m.autotune(prec) if args.autotune else None
    for _ in range(args.warmup):
        m.lanczos_sectors(sectors, steps, prec=prec, seed=seed, refine=refine)
    stream = torch.cuda.current_stream()
    clk = Clocks(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches, rs = 0, None
    e0.record(stream)
    for _ in range(args.steps):
        rs = m.lanczos_sectors(sectors, steps, prec=prec, seed=seed, refine=refine)
        launches += sum(r["launches"] for r in rs)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop() if clk else None
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    # rows x steps actually taken (tiny sectors stop at breakdown)
    dims = [math.comb(spec.n_sites, n) for n in sectors]
    units = sum(d * r["steps"] for d, r in zip(dims, rs))
    value = whole_job_rate(units * args.steps, world, ms / 1e3)
    if rank != 0:
        return None
    e = [(r["e_refined"] if refine else r["eig"][0]) for r in rs]
    # the sector runs are parallel branches of one graph, so no single kernel can be timed:
    # the achieved rate is the whole call's (a lower bound for the fused H v kernels)
    hbm, src = peaks()
    esz = 8 if prec == hp.FP64 else 4
    alg = 3 * esz * units  # fused H v + Lanczos pass 1 traffic of all sectors and steps
    achieved = alg * args.steps / (ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": None, "peak_source": src,
            "kernel": "whole sector graph (split-row or one-CTA Lanczos per sector + pass 2 + solvers); lower bound",
            "algorithmic_bytes_per_launch": alg}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == hp.FP64 else "f32+f64acc+f64 refine", "data": "synthetic",
        "config": {"workload": args.workload, "dim_total": sum(dims), "sectors": len(sectors), "lanczos_steps": steps,
                   "model": spec.name, "start": "philox gaussian, seed 123432+rank",
                   "l2": l2_note(max(dims) * (8 if prec == hp.FP64 else 4)), "parallelism": f"replicas{world}"},
        "e0_min": min(e), "roofline": roof, "gpu_launches": launches, "clocks": clocks, "autotune": tune,
    }
    if args.cpu_baseline:
        sub = spec.with_basis(wl.BASIS_SZ, spec.n_sites // 2)
        rps, n, dt, cores = oracle_rows_per_s(sub)
        out["cpu_baseline"] = {"value": round(rps / 1e9, 6), "unit": "Gelem/s", "cores": cores, "kind": "oracle",
                               "sample": f"oracle H v on {n} contiguous rows of the S^z=0 sector ({dt:.1f} s, OpenMP "
                                         f"over {cores} host threads)"}
    return out


def run_reference(args, world, rank):
    """The CPU oracle, as it stands, on the host cores: each step is a bounded sample of the same
    workload's H v -- a slice of rows when the oracle can hold the input vector in host memory,
    else randomly sampled rows whose input elements it regenerates from their Philox index."""
    if rank != 0:
        return None
    import oracle
    W = wl.workload(args.workload)
    spec = W["model"]
    D = oracle.dim(spec)
    cores = os.cpu_count() or 1
    if D * 16 <= 16e9:
        rng = np.random.default_rng(0)
        v = np.empty(D, dtype=np.complex128)
        v.real = rng.standard_normal(D)
        v.imag = 0.0
        n = min(300_000, D)
        for _ in range(args.warmup):
            oracle.apply_H_slice(spec, v, 0, n // 10)
        t0 = time.perf_counter()
        for k in range(args.steps):
            oracle.apply_H_slice(spec, v, (k * n) % max(D - n, 1), n)
        dt = time.perf_counter() - t0
        sample = f"oracle H v on {n} contiguous rows per step of the {args.workload} basis"
    else:
        rng = np.random.default_rng(0)
        n = 200_000
        for _ in range(args.warmup):
            oracle.apply_H_rows_philox(spec, np.sort(rng.integers(0, D, size=n // 10)).astype(np.uint64), 777, False)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.apply_H_rows_philox(spec, np.sort(rng.integers(0, D, size=n)).astype(np.uint64), 777, False)
        dt = time.perf_counter() - t0
        sample = (f"oracle H v on {n} randomly sampled rows per step of the {args.workload} basis, input elements "
                  f"regenerated from the Philox definition of the start vector")
    val = n * args.steps / dt / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": "Gelem/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "dim": D, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(val, 6), "unit": "Gelem/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(val, 6), "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heisenberg_6x6_sz0", choices=wl.WORKLOADS)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--lanczos-steps", "--iters", dest="lanczos_steps", type=int, default=0,
                    help="Lanczos steps (or mTPQ multiplications) per benchmark step; 0: the workload's "
                         "(mTPQ: 20 of the 1000)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false", help="skip the fp32 + fp64-refinement run")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", help="use the built-in launch shape")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false", help="skip the pinned-host-start-vector run")
    ap.add_argument("--no-sub", dest="sub", action="store_false", help="skip the 4x4 Hubbard sub-line")
    ap.add_argument("--split", default="", help="L,K: fixed split-row shape of the S^z-sector kernels (no autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks exit without work
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        out = run_reference(args, world, rank)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
        return
    world, rank, local = dist_setup(args.gpus)
    if "n_starts" in wl.workload(args.workload):
        out = run_tpq(args, world, rank, local)
    elif args.workload == "j1j2_ring28_all_sectors":
        out = run_sectors(args, world, rank, local)
    else:
        out = run_ours(args, world, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
