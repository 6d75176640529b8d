"""Throughput of the CPRA hot path on GB300: angle-iterations per second.

One step = one whole reconstruction of the N = 512, Np = 360 workload (object
256^3 voxels, 6 ellipsoids, 1e6 photons per pattern): intensity preparation,
the seeded start, 220 global iterations (200 HIO + 20 ER, carousel coupling
every 10), and the 3D assembly (spectra, gridding, inverse 3D FFT).
value = Np * 220 / step time, inputs already in HBM.  e2e = the same metric
through the C ABI with pinned host buffers: every step's intensity upload and
the download of its complex volume are inside the timed region (the download
overlaps the next step's work; the region ends when the last one has landed).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs its own reconstruction (independent problems,
no collective) and rank 0 prints one JSON line.
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

METRIC = "CPRA angle-iterations/s at N=512,Np=360 vs plain GPU; p50/p99 reconstruct latency"
N, NP, T_HIO, T_ER = 512, 360, 200, 20
ITERS = T_HIO + T_ER
PROFILE_NOTE = ("--np/--iters shrink the workload for profiler captures only; the bench "
                "number is the default N=512, Np=360, 220-iteration reconstruction")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_rate(units_per_rank, ms_local, dist=None, device="cpu"):
    """Whole-job throughput of replicas: every rank processed units_per_rank
    units; the job took as long as its slowest rank.  Returns (units/s over
    all ranks, the max-over-ranks milliseconds)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms = float(t.item())
    return world * units_per_rank / (ms * 1e-3), ms


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0])]
        mx = [num(r[1]) for r in self.rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if "Active" in r[3 + i]
                          and not r[3 + i].startswith("Not")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def bench_config(world: int) -> dict:
    """The workload both arms name (the reference arm times a bounded sample
    of it, described in its cpu_baseline and ms_per_step_note)."""
    return {"workload": f"CPRA N={N} Np={NP}: {T_HIO} HIO + {T_ER} ER iterations, "
                        "coupling alpha=(0.2,0.6,0.2) every 10, 512^3 assembly",
            "N": N, "Np": NP, "iterations": ITERS,
            "l2": "inputs larger than L2 (state 0.75 GB, intensities 0.38 GB)",
            "parallelism": f"replicas x{world}"}


def make_inputs(device, n_angles=NP):
    import synth
    return synth.make_case("metric", device=device, Np=n_angles)


# The method's algorithmic bytes per angle-iteration (what one pass over an
# angle must move, whatever the design): read and write the real FP32
# iterate, read the Hermitian-symmetrised amplitude on the half plane
# (N (N/2 + 1) floats) and the support bitmask.
def method_bytes_per_angle_iteration(n: int) -> int:
    return 4 * n * n + 4 * n * n + 4 * n * (n // 2 + 1) + n * n // 8


# Measured DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum)
# of the iteration kernels, bytes per angle-iteration, with the capture's
# date and a fingerprint of the kernel sources it was taken on.  The bench
# reports it only while the sources still have that fingerprint.
NCU_ITERATION_TRAFFIC = {
    # k_colpass_w<512> 423.15 MB + k_rowpass_w<512> 699.45 MB for 180 angles
    # (one launch each, --set full, which starts every replay with a flushed
    # L2, so what a pass inherits in L2 from the previous one is not seen);
    # the coupling prime (one launch in ten iterations, 5 % of the time) was
    # not captured and is not included
    (("k_colpass", "k_rowpass", "k_prime"), 512): ((423.146496e6 + 699.453952e6) / 180,
                                                   "2026-12-04", "9e401db110ddc5d1"),
}  # {(kernel classes that ran, N): (bytes per angle-iteration, capture date, fingerprint)}
# the kernels' sources and the host code that orders their launches and
# tiles (the order decides what the L2 still holds between passes)
KERNEL_SOURCES = ("fast_kernels.cuh", "fftw.cuh", "fftw_pair.cuh", "fft.cuh", "cpra_internal.h",
                  "k_fast.cu", "k_fused.cu", "taps.cuh", "api.cu")


def kernel_fingerprint() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        path = os.path.join(ROOT, "paper_2402_05283_gb300", "csrc", f)
        if os.path.exists(path):
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def roofline_figures(plan, cp, peaks, Np_total, iters_timed):
    """The method's roofline: one all-angle iteration is the unit.

    achieved = the method's algorithmic bytes of one all-angle iteration
    (Np x method_bytes_per_angle_iteration) / the mean device time of one
    iteration, the summed CUDA-event time of the iteration kernels (row and
    column passes, coupling primes, fused launches, shrink-wrap) over the
    timed region divided by the iterations run there.  The per-kernel
    figures beside it credit each kernel with the bytes its own design moves
    (effective bandwidth of that kernel, not the method's fraction)."""
    stats = {k: plan.kernel_stats(k) for k in range(cp.KERNEL_KINDS)}
    total = sum(v[0] for v in stats.values()) or 1.0
    names = {cp.KERNEL_COLPASS: "k_colpass", cp.KERNEL_ROWPASS: "k_rowpass",
             cp.KERNEL_FUSED: "k_fused", cp.KERNEL_PRIME: "k_prime",
             cp.KERNEL_SHRINKWRAP: "k_sw", cp.KERNEL_ASSEMBLE: "assembly",
             cp.KERNEL_PREPARE: "k_prepare"}
    iteration_kinds = [cp.KERNEL_COLPASS, cp.KERNEL_ROWPASS, cp.KERNEL_PRIME, cp.KERNEL_FUSED,
                       cp.KERNEL_SHRINKWRAP]
    iter_ms = sum(stats[k][0] for k in iteration_kinds)
    if iter_ms <= 0 or iters_timed <= 0:
        return None, stats
    NN = N * N
    unit_bytes = Np_total * method_bytes_per_angle_iteration(N)
    ms_per_iter = iter_ms / iters_timed
    achieved = unit_bytes / (ms_per_iter * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    ran = [names[k] for k in iteration_kinds if stats[k][1]]
    key = (tuple(ran), N)
    fp = kernel_fingerprint()
    traffic, traffic_note = None, "no ncu capture of these kernel sources (fingerprint %s)" % fp
    if key in NCU_ITERATION_TRAFFIC and NCU_ITERATION_TRAFFIC[key][2] == fp:
        per_ai, date, _ = NCU_ITERATION_TRAFFIC[key]
        traffic = int(per_ai * Np_total)
        traffic_note = f"ncu DRAM bytes of the iteration kernels, captured {date}, per iteration"
    # each kernel's own design bytes per angle of one launch (effective bandwidth)
    design = {
        cp.KERNEL_COLPASS: 4 * NN + 4 * NN + 2 * NN + 4 * N,        # Hp in/out, A_sym
        cp.KERNEL_ROWPASS: 4 * NN * 4 + NN // 8,                     # Hp in/out, g in/out, S
        cp.KERNEL_PRIME: 3 * 4 * NN + 4 * NN + 4 * NN,               # 3 taps, g out, Hp out
    }
    per_kernel = {}
    for k in iteration_kinds:
        ms, launches = stats[k]
        if not launches:
            continue
        entry = {"ms_per_launch": round(ms / launches, 4), "launches": launches,
                 "share_of_kernel_time": round(ms / total, 3)}
        if k in design:
            gbs = design[k] * Np_total / (ms / launches * 1e-3) / 1e9
            entry.update({"design_bytes_per_launch": design[k] * Np_total,
                          "effective_gbs": round(gbs, 1), "effective_frac": round(gbs / peak, 4)})
        per_kernel[names[k]] = entry
    # the FP32 context: radix-2 flop count of the R2C + C2R pair plus the
    # pixel work, against 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
    flops = 10.0 * NN * math.log2(N) + 20.0 * NN
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    alu_tf = Np_total * flops / (ms_per_iter * 1e-3) / 1e12
    return {"bound": "hbm", "kernel": "one all-angle iteration: " + " + ".join(ran),
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_note": traffic_note,
            "bytes_per_iteration": int(unit_bytes),
            "bytes_per_angle_iteration": method_bytes_per_angle_iteration(N),
            "ms_per_iteration": round(ms_per_iter, 5),
            "per_kernel": per_kernel,
            "alu_context": {"flops_per_angle_iteration": int(flops), "achieved_tflops": round(alu_tf, 2),
                            "fp32_peak_tflops": round(alu_peak, 1), "frac": round(alu_tf / alu_peak, 4),
                            "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (unit counts and "
                                           "maximum SM clock)"},
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"
                           if not peaks.get("_fallback") else "fallback 6800 GB/s"}, stats


def sample_inputs(n_angles: int = 8):
    """The first angles of the workload's patterns, on the host."""
    import torch
    import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    d = synth.make_case("metric", device=dev)
    I = d["I"][:n_angles]
    I = I.cpu().numpy() if hasattr(I, "cpu") else np.asarray(I)
    return I, d["support"]


def _oracle_worker(job):
    """One host process of the CPU baseline: the oracle as it stands (Jacobi
    steps with numpy.fft transforms, its pinned FFT mode) on a slice of the
    workload's angles, stepping until `seconds` have passed."""
    I, S, seconds = job
    import oracle as O
    na = I.shape[0]
    run = O.OracleRun.start(O.OracleConfig(N=I.shape[-1], Np=na, n_ei=10, seed=0, fft=True), I, S)
    t0 = time.perf_counter()
    it = 0
    while True:
        run.step()
        it += 1
        if time.perf_counter() - t0 > seconds:
            break
    return na * it, time.perf_counter() - t0


def cpu_baseline(I, S, seconds: float = 10.0, pool=None):
    """The FP64 oracle on the host cores: a bounded sample of the workload.

    One process per core (spawned: the pool never inherits a CUDA context),
    each running the oracle on its own slice of angles (Jacobi angles are
    independent within an iteration), so the host is used the way the
    oracle's angle loop allows.  value = all processes' angle-iterations over
    the longest process time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    na = I.shape[0]
    per = max(1, na // cores)
    jobs = [(I[i:i + per], S, seconds) for i in range(0, per * min(cores, na // per), per)]
    own = pool is None
    if own:
        pool = oracle_pool(len(jobs))
    try:
        res = pool.map(_oracle_worker, jobs)
    finally:
        if own:
            pool.close()
            pool.join()
    units = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return {"value": round(units / dt, 3), "unit": "angle-iterations/s", "cores": len(jobs),
            "kind": "oracle",
            "sample": f"FP64 oracle (numpy.fft mode) on {per * len(jobs)} angles of the N={N} "
                      f"workload, {len(jobs)} processes of {per} angles, {units} angle-iterations "
                      f"in {dt:.1f} s"}


# ---------------------------------------------------------------- systems forms
_SERVE_POOL = {}

def form_batch(cp, torch, seed=3):
    """cfg 3: 16 reconstructions of uneven N and Np, 300 iterations each.
    Three ways: one at a time (plain plans, AUTO engines, no graph); one
    batch with one launch per kernel and size group (autotuned engines, CUDA
    graph); one batch in persistent work-queue mode (warp engine, one
    persistent launch per size group between coupling steps, CUDA graph).
    Batched results must equal the same engine run alone bit for bit."""
    import synth
    rng = np.random.default_rng(seed)
    Ns = rng.choice([128, 192, 256, 384], size=16)
    Nps = rng.choice([90, 180, 360], size=16)
    iters = 300
    cases = {}
    for i in range(16):
        key = (int(Ns[i]), int(Nps[i]))
        if key not in cases:
            d = synth.make_case("cfg1", device="cuda", N=key[0], Np=key[1], request=i)
            cases[key] = (d["I"].contiguous(), d["thetas"])

    def plans(engine):
        out = []
        for i in range(16):
            I, th = cases[(int(Ns[i]), int(Nps[i]))]
            p = cp.Plan(cp.make_config(int(Ns[i]), int(Nps[i]), seed=i, hio_iters=280, er_iters=20,
                                       engine=engine))
            p.load_intensities(I, 0, th)
            out.append(p)
        return out

    def one_at_a_time(ps):
        for p in ps:
            p.iterate(1)
            p.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p in ps:
            p.iterate(iters)
            p.sync()
        return time.perf_counter() - t0

    def batched(ps, persistent):
        b = cp.Batch(ps, use_graph=True)
        if persistent:
            b.set_persistent(1)
        b.iterate(30)  # capture the 30-iteration graph
        for p in ps:
            p.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(iters // 30):
            b.iterate(30)
        torch.cuda.synchronize()
        return b, time.perf_counter() - t0

    work = int(sum(int(n) for n in Nps)) * iters
    alone = plans(cp.ENGINE_AUTO)
    t_alone = one_at_a_time(alone)
    tuned = {int(n): cp.cpra_autotune(int(n))[0] for n in set(Ns.tolist())}
    mixed = plans(cp.ENGINE_TUNED)
    b, t_batch = batched(mixed, False)
    # plans whose tuned engine is the one AUTO picks must agree bit for bit
    auto = {n: (cp.ENGINE_FUSED if n in (64, 128, 256) else cp.ENGINE_WARP) for n in tuned}
    pairs = [(a, m) for a, m in zip(alone, mixed) if tuned[a.N] == auto[a.N]]
    same = all(np.array_equal(a.result(cp.RESULT_STATE), m.result(cp.RESULT_STATE)) for a, m in pairs)
    b.close()
    for p in alone + mixed:
        p.close()
    warp_alone = plans(cp.ENGINE_WARP)
    t_warp_alone = one_at_a_time(warp_alone)
    pers = plans(cp.ENGINE_WARP)
    bp, t_pers = batched(pers, True)
    same_p = all(np.array_equal(a.result(cp.RESULT_STATE), m.result(cp.RESULT_STATE))
                 for a, m in zip(warp_alone, pers))
    launches_p = bp.launches(30)
    bp.close()
    for p in warp_alone + pers:
        p.close()
    return {"workload": "16 reconstructions, N in {128,192,256,384}, Np in {90,180,360}, "
                        "280 HIO + 20 ER", "angle_iterations": work,
            "one_at_a_time": {"value": round(work / t_alone, 1), "seconds": round(t_alone, 3),
                              "engines": "AUTO (fused at 128/256, warp at 192/384)"},
            "batched_graph": {"value": round(work / t_batch, 1), "seconds": round(t_batch, 3),
                              "speedup_vs_one_at_a_time": round(t_alone / t_batch, 3),
                              "tuned_engines": tuned, "bit_identical": bool(same),
                              "compared": len(pairs)},
            "persistent_graph": {"value": round(work / t_pers, 1), "seconds": round(t_pers, 3),
                                 "speedup_vs_one_at_a_time": round(t_alone / t_pers, 3),
                                 "speedup_vs_warp_one_at_a_time": round(t_warp_alone / t_pers, 3),
                                 "launches_per_30_iterations": int(launches_p),
                                 "bit_identical_to_warp_alone": bool(same_p)},
            "warp_one_at_a_time": {"value": round(work / t_warp_alone, 1),
                                   "seconds": round(t_warp_alone, 3)}}


def form_multi_guess(cp, torch, N_=256, Np_=144, n_r=32, n_l=8, iters=220, seed=6):
    """Step C: n_r reconstructions of one pattern set from n_r random starts
    (RAAR beta 0.9 then ER, the paper's rule for its cell data), iterated as
    one batch, then merged (the n_l of lowest error kept, mass centres moved,
    twins chosen, averaged) and assembled; the PRTF of the kept guesses.
    N = 256 with Np = 144 is one of the paper's performance sizes."""
    import synth
    d = synth.make_case("cfg1", device="cuda", N=N_, Np=Np_, request=seed)
    I, th = d["I"].contiguous(), d["thetas"]
    hio = iters - 20
    plans = []
    for i in range(n_r):
        p = cp.Plan(cp.make_config(N_, Np_, seed=100 + i, hio_iters=hio, er_iters=20,
                                   update=cp.UPDATE_RAAR))
        p.load_intensities(I, 0, th)
        plans.append(p)
    dst = cp.Plan(cp.make_config(N_, Np_))
    dst.load_intensities(I, 0, th)
    b = cp.Batch(plans, use_graph=True)
    b.iterate(10)  # capture
    prtf = torch.zeros((Np_, N_ // 2), device="cuda")
    cp.cpra_merge(plans[:2], 1, 0, dst, prtf)  # first use: scratch and gridding lists
    for p in plans:
        p.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters // 10):
        b.iterate(10)
    torch.cuda.synchronize()
    t_iter = time.perf_counter() - t0
    t0 = time.perf_counter()
    sel, inv = cp.cpra_merge(plans, n_l, 0, dst, prtf)
    torch.cuda.synchronize()
    t_merge = time.perf_counter() - t0
    ring = prtf.mean(0).cpu().numpy()
    below = np.nonzero(ring < 0.5)[0]
    errs = [float(p.result(cp.RESULT_ERRORS)[-1].mean()) for p in plans]
    b.close()
    for p in plans + [dst]:
        p.close()
    work = n_r * Np_ * iters
    return {"workload": f"N={N_}, Np={Np_}: {n_r} random starts x ({hio} RAAR + 20 ER), "
                        f"batched with a CUDA graph; merge of the best {n_l}",
            "angle_iterations": work, "value": round(work / t_iter, 1), "unit": "angle-iterations/s",
            "iterate_s": round(t_iter, 3), "merge_and_assemble_ms": round(t_merge * 1e3, 2),
            "selected": sel, "inverted": [int(v) for v in inv],
            "final_fourier_error_best_worst": [round(min(errs), 5), round(max(errs), 5)],
            "prtf_mean_ring_0_to_8": [round(float(v), 4) for v in ring[:8]],
            "prtf_first_ring_below_0.5": int(below[0]) if below.size else None}


def form_refine(cp, torch, plan, iters=50, shrink_every=5):
    """Step D refinement on the bench plan's assembled N = 512 volume: the
    paper's 50 tomographic iterations with the 3D support shrunk every 5.
    Bytes of the five-pass design per iteration: x rows read rho and write
    the spectrum, y and z lines read and write it twice, the z pass reads
    the data on the measured cells, x rows read it and write rho:
    (4 + 1/8 + 8 + 16 + 16 + 8 f + 16 + 12) N^3, f = measured fraction."""
    Nn = plan.N
    plan.assemble_3d()
    plan.refine_3d(2)  # allocation and set-up outside the timed region
    plan.assemble_3d()
    torch.cuda.synchronize()
    plan.set_profiling(True)
    t0 = time.perf_counter()
    errs = plan.refine_3d(iters, shrink_every=shrink_every, sigma=2.0, tau=0.1)
    wall = time.perf_counter() - t0
    ms, launches = plan.kernel_stats(cp.KERNEL_REFINE)
    plan.set_profiling(False)
    n3 = float(Nn) ** 3
    per_iter = (4 + 1 / 8 + 8 + 16 + 16 + 16 + 12) * n3
    return {"workload": f"N={Nn}^3 refinement of the bench reconstruction, {iters} iterations, "
                        f"3D shrink-wrap every {shrink_every} (sigma 2, tau 0.1)",
            "device_ms": round(ms, 2), "ms_per_iteration": round(ms / iters, 3),
            "wall_s": round(wall, 3), "launches": launches,
            "design_bytes_per_iteration_excl_data": int(per_iter),
            "achieved_gbs_excl_data": round(per_iter * iters / (ms * 1e-3) / 1e9, 1),
            "error_first_last": [round(float(errs[0]), 5), round(float(errs[-1]), 5)]}


def form_config2(cp, torch, iters=500, every=20):
    """cfg 2 as written: N = 256, Np = 180, a 128^3 object of 40 ellipsoids
    with Gaussian-correlated texture (sigma 2 voxels) at 1e7 photons, 500 HIO
    iterations with shrink-wrap every 20 (sigma 2 px, tau 0.1), then the
    256^3 assembly and inverse 3D FFT.  The same run without shrink-wrap
    gives the shrink-wrap overhead."""
    import synth
    t_gen = time.perf_counter()
    d = synth.make_case("cfg2", device="cuda")
    t_gen = time.perf_counter() - t_gen
    N_, Np_ = d["N"], d["Np"]
    I, th = d["I"].contiguous(), d["thetas"]
    out = {"workload": f"N={N_}, Np={Np_}: 40-ellipsoid textured 128^3 object, 1e7 photons, "
                       f"{iters} HIO, shrink-wrap every {every}; {N_}^3 assembly",
           "input_seconds": round(t_gen, 2)}
    for name, sw in (("shrinkwrap", every), ("no_shrinkwrap", 0)):
        plan = cp.Plan(cp.make_config(N_, Np_, hio_iters=iters, er_iters=0, shrinkwrap_every=sw))
        plan.load_intensities(I, 0, th)
        plan.iterate(2)
        plan.assemble_3d()  # first use allocates the assembly buffers and lists
        plan.reset()
        plan.load_support(None)
        torch.cuda.synchronize()
        plan.set_profiling(True)
        t0 = time.perf_counter()
        plan.iterate(iters)
        plan.assemble_3d()
        plan.sync()
        dt = time.perf_counter() - t0
        sw_ms, sw_n = plan.kernel_stats(cp.KERNEL_SHRINKWRAP)
        asm_ms, _ = plan.kernel_stats(cp.KERNEL_ASSEMBLE)
        plan.set_profiling(False)
        err = plan.result(cp.RESULT_ERRORS)
        sup = plan.result(cp.RESULT_SUPPORT)
        out[name] = {"value": round(Np_ * iters / dt, 1), "unit": "angle-iterations/s",
                     "seconds_with_assembly": round(dt, 4), "shrinkwrap_ms": round(sw_ms, 3),
                     "shrinkwrap_launch_groups": sw_n, "assembly_ms": round(asm_ms, 3),
                     "final_fourier_error_mean": round(float(err[-1].mean()), 5),
                     "support_fraction_mean": round(float(sup.mean()), 4)}
        plan.close()
    a_, b_ = out["shrinkwrap"], out["no_shrinkwrap"]
    out["shrinkwrap_overhead"] = round(a_["seconds_with_assembly"] / b_["seconds_with_assembly"] - 1.0, 4)
    return out


def form_serving(cp, torch, n_req=16, compress=10.0, seed=4, max_active=0, early_start=False):
    """cfg 4 with time compressed by `compress`: Poisson arrivals at 4/s,
    each request streams its Np patterns at 10 patterns/s (both x compress),
    N in {256, 512}, Np in {180, 360}, 220 iterations; continuous batching
    (max_active 0) or one request at a time (max_active 1)."""
    import synth
    rng = np.random.default_rng(seed)
    combos = [(256, 180), (256, 360), (512, 180), (512, 360)]
    pool = _SERVE_POOL
    for N_, Np_ in combos:
        if (N_, Np_) not in pool:
            d = synth.make_case("cfg1", device="cuda", N=N_, Np=Np_, request=N_ + Np_)
            pool[(N_, Np_)] = (d["I"].cpu().numpy(), d["thetas"])
    arrivals = np.cumsum(rng.exponential(1.0 / (4.0 * compress), size=n_req))
    picks = [combos[i] for i in rng.integers(0, 4, size=n_req)]
    rate = 10.0 * compress  # patterns per second
    chunk = 10
    srv = cp.Server(hbm_reserve_bytes=8 << 30, max_active=max_active, iters_per_round=10,
                    early_start=early_start)
    sched = []  # (time, kind, request index, first)
    for r in range(n_req):
        sched.append((arrivals[r], 0, r, 0))
        Np_ = picks[r][1]
        for f in range(0, Np_, chunk):
            sched.append((arrivals[r] + (f + chunk) / rate, 1, r, f))
    sched.sort()
    ids = [None] * n_req
    t0 = time.perf_counter()
    for t_ev, kind, r, f in sched:
        dt = t_ev - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        N_, Np_ = picks[r]
        if kind == 0:
            ids[r] = srv.submit(cp.make_config(N_, Np_, seed=r, hio_iters=200, er_iters=20))
        else:
            I, th = pool[(N_, Np_)]
            k = min(chunk, Np_ - f)
            srv.push(ids[r], I[f:f + k], f, th[f:f + k])
    for rid in ids:
        srv.wait(rid, 600.0)
    wall = time.perf_counter() - t0
    first, final, first_sub, final_sub, ferr = [], [], [], [], []
    for rid in ids:
        info = srv.info(rid)
        ferr.append(float(srv.result(rid, cp.RESULT_ERRORS)[-1].mean()))
        first.append(info["t_first_estimate"] - info["t_last_pattern"])
        final.append(info["t_final"] - info["t_last_pattern"])
        first_sub.append(info["t_first_estimate"] - info["t_submit"])
        final_sub.append(info["t_final"] - info["t_submit"])
    st = srv.stats()
    srv.stop()
    q = lambda a: [round(float(x), 4) for x in np.percentile(a, [50, 99])]  # noqa: E731
    return {"requests": n_req, "time_compression": compress, "max_active": max_active,
            "p50_p99_s_first_estimate_after_last_pattern": q(first),
            "p50_p99_s_final_after_last_pattern": q(final),
            "p50_p99_s_first_estimate_after_submit": q(first_sub),
            "p50_p99_s_final_after_submit": q(final_sub),
            "angle_iterations": int(st["angle_iterations"]),
            "value": round(st["angle_iterations"] / wall, 1), "wall_s": round(wall, 3),
            "max_batch": int(st["max_batch"]), "rounds": int(st["rounds"]),
            "early_start": bool(early_start),
            "mean_final_fourier_error": round(float(np.mean(ferr)), 5)}


def form_p0(torch, I_dev, S_box, iters=20, beta=0.9, n_ei=10):
    """The comparison path P0: the same iteration (HIO on the support with
    positivity, Eq. 4 coupling alpha = (0.2, 0.6, 0.2) every n_ei) written as
    cuFFT transforms (torch.fft) plus separate elementwise kernels on a
    complex FP32 spectrum, on the workload of the plain path.  Timed only;
    never on the product path."""
    Np_, N_, _ = I_dev.shape
    A = torch.fft.ifftshift(torch.sqrt(torch.clamp(I_dev, min=0.0)), dim=(-2, -1))
    S = S_box.bool().expand(Np_, N_, N_) if S_box.dim() == 2 else S_box.bool()
    g = torch.rand((Np_, N_, N_), device=I_dev.device) * S

    def step(t, g):
        if t % n_ei == 0:
            g = 0.2 * torch.roll(g, 1, 0) + 0.6 * g + 0.2 * torch.roll(g, -1, 0)
        G = torch.fft.fft2(g)
        mag = torch.abs(G)
        Gp = torch.where(mag > 0, A * G / torch.clamp(mag, min=1e-30), A.to(G.dtype))
        gp = torch.fft.ifft2(Gp).real
        v = S & (gp >= 0)
        return torch.where(v, gp, g - beta * gp)

    for t in range(3):
        g = step(t, g)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(iters):
        g = step(t, g)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": round(Np_ * iters / (ms * 1e-3), 1), "unit": "angle-iterations/s",
            "what": "cuFFT (torch.fft) + separate elementwise kernels, complex64 spectrum, "
                    f"N={N_}, Np={Np_}, {iters} HIO iterations with coupling every {n_ei}"}


def _er_fp64(torch, I_rows, S, x0, iters):
    """FP64 reference of `iters` ER iterations on a stack of patterns, plain
    torch on the GPU: modulus projection onto sqrt(I) (phase 1 where G = 0),
    then the support-positivity projection.  It serves the error figures of
    the 16-bit forms here; the tests check the library against the oracle."""
    A = torch.fft.ifftshift(torch.sqrt(torch.clamp(I_rows.double(), min=0.0)), dim=(-2, -1))
    Sb = torch.as_tensor(S, device=I_rows.device).bool()
    g = x0.double()
    for _ in range(iters):
        G = torch.fft.fft2(g)
        mag = G.abs()
        ph = torch.where(mag > 0, G / torch.where(mag > 0, mag, torch.ones_like(mag)), torch.ones_like(G))
        gp = torch.fft.ifft2(A * ph).real
        g = torch.where(Sb & (gp >= 0), gp, torch.zeros_like(gp))
    return g


def form_config5(cp, torch, iters_acc=20, iters_speed=50, sample=(0, 361)):
    """cfg 5 as written: N = 1024, Np = 720 noiseless patterns of a 512^3
    object of 200 ellipsoids (rasterised and projected on the GPU), run in
    FP32 and with the BF16 / FP16 tensor-core DFT stages: speed over
    iters_speed HIO iterations, error of sampled angles against an FP64
    reference after iters_acc ER iterations from one seeded state (no
    coupling), and the 1024^3 assembly with its inverse 3D FFT."""
    import synth
    N_, Np_ = 1024, 720
    t_gen = time.perf_counter()
    d = synth.make_case("cfg5", device="cuda", raster_on_device=True)
    I_dev = d["I"].contiguous()
    thetas = d["thetas"]
    del d
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    rng = np.random.default_rng(12)
    S = np.zeros((N_, N_), bool)
    S[N_ // 4:3 * N_ // 4, N_ // 4:3 * N_ // 4] = True
    g0 = (rng.random((Np_, N_, N_), dtype=np.float32) * S).astype(np.float32)
    ref = {n: _er_fp64(torch, I_dev[n:n + 1], S, torch.from_numpy(g0[n:n + 1]).cuda(), iters_acc)[0]
           for n in sample}
    out = {"workload": f"N={N_}, Np={Np_}: 200-ellipsoid 512^3 object, noiseless, {Np_} projections",
           "input_seconds": round(t_gen, 1)}
    for name, prec in (("fp32", cp.FP32), ("bf16", cp.BF16_TC), ("fp16", cp.FP16_TC)):
        cfg = cp.make_config(N_, Np_, precision=prec, hio_iters=0, er_iters=iters_acc, n_ei=1 << 20)
        plan = cp.Plan(cfg)
        plan.load_intensities(I_dev, 0, thetas)
        plan.load_support(torch.from_numpy(S.astype(np.uint8)).cuda())
        plan.load_state(g0, 1)  # t = 1: no coupling step inside the run
        plan.iterate(iters_acc)
        g = plan.result(cp.RESULT_STATE)
        errs = [float(np.linalg.norm(g[n] - ref[n].cpu().numpy()) / np.linalg.norm(ref[n].cpu().numpy()))
                for n in sample]
        plan.close()
        plan = cp.Plan(cp.make_config(N_, Np_, precision=prec, hio_iters=iters_speed, er_iters=0))
        plan.load_intensities(I_dev, 0, thetas)
        plan.iterate(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.iterate(iters_speed)
        plan.sync()
        dt = time.perf_counter() - t0
        entry = {"value": round(Np_ * iters_speed / dt, 1), "unit": "angle-iterations/s",
                 "rel_l2_vs_fp64_after_%d_er" % iters_acc: [float("%.3e" % e) for e in errs]}
        if prec == cp.FP32:
            plan.assemble_3d()  # first use: buffers and gridding lists
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.assemble_3d()
            plan.sync()
            entry["assembly_1024cubed_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        plan.close()
        out[name] = entry
    return out


def form_precision(cp, torch, I_dev, thetas, S_box, n_angles=NP, N_=N, sample=(0, 1), iters=5):
    """Throughput of the FP32 / BF16 / FP16 forms on the bench workload and
    their iterate error against an FP64 reference (_er_fp64) after `iters`
    ER iterations from a seeded state, on sampled angles (neighbours coupled
    at t = 0)."""
    rng = np.random.default_rng(11)
    S = np.zeros((N_, N_), bool)
    S[N_ // 4:3 * N_ // 4, N_ // 4:3 * N_ // 4] = True
    g0 = (rng.random((n_angles, N_, N_), dtype=np.float32) * S).astype(np.float32)
    out = {}
    ref = {}
    for n in sample:
        idx = [(n - 1) % n_angles, n, (n + 1) % n_angles]
        x = 0.2 * g0[idx[0]].astype(np.float64) + 0.6 * g0[idx[1]] + 0.2 * g0[idx[2]]
        ref[n] = _er_fp64(torch, I_dev[n:n + 1], S, torch.from_numpy(x[None]).cuda(), iters)[0].cpu().numpy()
    for name, prec in (("fp32", cp.FP32), ("bf16", cp.BF16_TC), ("fp16", cp.FP16_TC)):
        plan = cp.Plan(cp.make_config(N_, n_angles, precision=prec, hio_iters=0, er_iters=iters))
        plan.load_intensities(I_dev, 0, thetas)
        plan.load_support(S_box)
        plan.load_state(g0, 0)
        plan.iterate(iters)
        g = plan.result(cp.RESULT_STATE)
        errs = [float(np.linalg.norm(g[n] - ref[n]) / np.linalg.norm(ref[n])) for n in sample]
        plan.load_state(g0, 0)
        plan.iterate(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.iterate(20)
        plan.sync()
        dt = time.perf_counter() - t0
        plan.close()
        out[name] = {"value": round(n_angles * 20 / dt, 1), "unit": "angle-iterations/s",
                     "rel_l2_vs_fp64_after_%d_er" % iters: [float("%.3e" % e) for e in errs]}
    return out


def oracle_pool(n: int):
    """Host processes for the oracle, spawned (never forked from a process
    that may hold a CUDA context)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (there is no
    reference implementation of the paper to install).  Every step is a
    bounded sample of the bench workload; ms_per_step is extrapolated from
    the sampled rate to a whole reconstruction."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    I, S = sample_inputs(max(cores, 8))
    pool = oracle_pool(min(cores, len(I)))
    per_step = []
    cb = None
    t_run = time.perf_counter()
    try:
        for i in range(args.warmup + args.steps):
            c = cpu_baseline(I, S, seconds=6.0 if i >= args.warmup else 1.0, pool=pool)
            if i >= args.warmup:
                per_step.append(c)
                cb = c
    finally:
        pool.close()
        pool.join()
    vals = [c["value"] for c in per_step]
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "angle-iterations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(NP * ITERS / v * 1e3, 1),
            "ms_per_step_note": "extrapolated: one reconstruction (Np x 220 angle-iterations) at "
                                "the sampled rate; each timed step is a 6 s sample",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(1),
            "wall_s": round(time.perf_counter() - t_run, 1),
            "cpu_baseline": {**cb, "value": v},
            "e2e": {"value": v, "unit": "angle-iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import paper_2402_05283_gb300 as cp
    from paper_2402_05283_gb300 import build as b

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    cp.lib()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {"hbm_gbs": 6800.0, "_fallback": True}

    NPa, IT = args.np, args.iters
    d = make_inputs(f"cuda:{local}", NPa)
    I_dev = d["I"].contiguous()
    thetas = d["thetas"]
    S_box = torch.from_numpy(d["support"]).cuda()
    stream = torch.cuda.current_stream()
    hio = min(T_HIO, IT)
    engine = {"auto": cp.ENGINE_AUTO, "warp": cp.ENGINE_WARP, "fused": cp.ENGINE_FUSED,
              "two_pass": cp.ENGINE_TWO_PASS}[args.engine]
    prec = {"fp32": cp.FP32, "bf16": cp.BF16_TC, "fp16": cp.FP16_TC}[args.precision]
    cfg = cp.make_config(N, NPa, hio_iters=hio, er_iters=IT - hio, seed=rank, engine=engine,
                         precision=prec)
    plan = cp.Plan(cfg, stream=stream.cuda_stream)
    vol = torch.empty((N, N, N, 2), dtype=torch.float32, device=f"cuda:{local}")

    def step():
        plan.load_intensities(I_dev, 0, thetas)
        plan.load_support(S_box)
        plan.reset()
        plan.iterate(IT)
        plan.assemble_3d(vol)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.form:
        # one form alone after the warm-up reconstructions (profiler captures)
        if rank == 0:
            print(json.dumps({"forms": {f: run_form(f, cp, torch, plan, I_dev, thetas, S_box)
                                        for f in args.form}}), flush=True)
        plan.close()
        return
    if dist:
        dist.barrier()
    launches0 = cp.cpra_launch_count()
    plan.set_profiling(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    launches = cp.cpra_launch_count() - launches0
    step_ms = [a.elapsed_time(b_) for a, b_ in evs]
    total_ms = sum(step_ms)
    roof, kstats = roofline_figures(plan, cp, peaks, NPa, IT * args.steps)
    plan.set_profiling(False)
    value, total_ms = job_rate(NPa * IT * args.steps, total_ms, dist, device=f"cuda:{local}")
    if args.no_extras:
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": value, "N": N, "Np": NPa,
                              "iterations": IT, "kernel_ms": {k: v[0] for k, v in kstats.items()}}))
        plan.close()
        return

    # end to end through the C ABI with pinned host buffers: every step uploads
    # its intensities and support and downloads its whole volume inside the
    # timed region.  The download is queued without waiting
    # (cpra_assemble_3d_async: a device-to-device copy into the plan's staging
    # buffer, then the transfer on the plan's second stream), so it overlaps
    # the next step's upload and iterations; two host buffers alternate, and
    # the timed region ends when the last download has landed.
    I_host = I_dev.cpu().pin_memory()
    S_host = S_box.cpu().pin_memory()
    vol_host = [torch.empty((N, N, N, 2), dtype=torch.float32).pin_memory() for _ in range(2)]
    e2e_steps = max(1, min(args.steps, 5))

    def step_host(k):
        plan.load_intensities(I_host, 0, thetas)
        plan.load_support(S_host)
        plan.reset()
        plan.iterate(IT)
        plan.assemble_3d_async(vol_host[k % 2])

    for k in range(2):  # the host link is slow on its first transfers after an idle spell
        step_host(k)
    plan.download_wait()
    torch.cuda.synchronize()
    te = time.perf_counter()
    for k in range(e2e_steps):
        step_host(k)
    plan.download_wait()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - te) / e2e_steps
    e2e_value, _ = job_rate(NPa * IT, e2e_s * 1e3, dist, device=f"cuda:{local}")

    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        forms = {f: run_form(f, cp, torch, plan, I_dev, thetas, S_box) for f in FORMS}
    if rank == 0:
        cores = len(os.sched_getaffinity(0))
        cb = cpu_baseline(I_dev[:max(cores, 8)].cpu().numpy(), d["support"]) if world == 1 else None
        qs = np.percentile(step_ms, [50, 99])
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "angle-iterations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}[args.precision], "data": "synthetic",
            "config": bench_config(world),
            "p50_ms": round(float(qs[0]), 3), "p99_ms": round(float(qs[1]), 3),
            "wall_s": round(wall, 3),
            "roofline": roof,
            "kernel_ms": {k: round(v[0] / args.steps, 3) for k, v in kstats.items() if v[1]},
            "cpu_baseline": cb,
            "e2e": {"value": round(e2e_value, 1), "unit": "angle-iterations/s",
                    "h2d_bytes_per_step": int(I_host.numel() * 4 + S_host.numel() * S_host.element_size()),
                    "d2h_bytes_per_step": int(vol_host[0].numel() * 4)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


FORMS = ("refine_3d", "p0_cufft_pointwise", "precision", "config5", "batching", "multi_guess_merge",
         "config2", "serving_config4", "serving_continuous", "serving_one_at_a_time",
         "serving_early_start")


def run_form(name, cp, torch, plan, I_dev, thetas, S_box):
    """One of the measurements beside the bench number (FORMS)."""
    if name == "refine_3d":
        return form_refine(cp, torch, plan)
    if name == "p0_cufft_pointwise":
        return form_p0(torch, I_dev, S_box)
    if name == "precision":
        return form_precision(cp, torch, I_dev, thetas, S_box)
    if name == "config5":
        return form_config5(cp, torch)
    if name == "batching":
        return form_batch(cp, torch)
    if name == "multi_guess_merge":
        return form_multi_guess(cp, torch)
    if name == "config2":
        return form_config2(cp, torch)
    if name == "serving_config4":
        return form_serving(cp, torch, compress=1.0, early_start=True)
    if name == "serving_continuous":
        return form_serving(cp, torch, max_active=0)
    if name == "serving_one_at_a_time":
        return form_serving(cp, torch, max_active=1)
    if name == "serving_early_start":
        return form_serving(cp, torch, max_active=0, early_start=True)
    raise ValueError(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--np", type=int, default=NP, help=PROFILE_NOTE)
    ap.add_argument("--iters", type=int, default=ITERS, help=PROFILE_NOTE)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e and CPU-baseline legs (profiler captures)")
    ap.add_argument("--engine", default="auto", choices=["auto", "warp", "fused", "two_pass"],
                    help="iteration engine of the plain path")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="arithmetic of the DFT stages (the bench number is the FP32 default; "
                         "bf16/fp16 run them on the tensor cores)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batching / serving / precision measurements")
    ap.add_argument("--form", action="append", choices=FORMS,
                    help="run only this measurement after the warm-up reconstructions (repeatable)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
