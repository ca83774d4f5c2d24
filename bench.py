#!/usr/bin/env python
"""Benchmark: constrained-realization sampling (Eq. mapmakingeq of arXiv
2306.15511, Sect. 2.2.1) at N_side = 1024, l_max = 2048.

Workload: 8 T+E+B realizations sharing C_l, beam and N^-1 (hits-weighted
noise, |b| < 20 deg mask + 200 holes, 10' beam).  One "step" is one
cg_sample call with a fixed iteration budget: RHS assembly (FP64-accurate
transforms), the diagonal preconditioner of Sect. 4 (the library's
default; --precond azim / lowl select the stronger ones), then
--iters-per-step batched mixed-precision
PCG iterations (FP32 operator applications) with FP64-accurate residual
replacements (reliable updates), the last one at the end of the step.
Inputs are synthetic (seeded Philox), resident in HBM and larger than L2.
The timed steps run the library's default path (the PCG iteration replayed
as a CUDA graph); one more step, run with per-kernel-class CUDA events
after the timed region, gives the kernel shares and the rooflines.

value = batched FP32 PCG iterations per second over the whole job (an
iteration applies the FP32 operator to all 8 realizations; the
FP64-accurate residual replacements are not counted), summed over ranks.
Ranks run independent replicas (weak scaling, no data-path collective);
`--gpus N` spawns N local ranks itself unless it runs under torchrun.

Extras (at N = 1 only, like the CPU baseline): the full solve to a true
FP64-accurate relative residual of 1e-6
with every preconditioner (the azimuthal blocks: App. A's per-m blocks of T
and E from the ring-averaged N^-1, exact up to l = 1024; the two-level low
block; the diagonal), fastest first in the line's `time_to_solution`;
the same steps with native FP64 residual replacements; the plain FP64 PCG
per-iteration time; both forms solved to 1e-6 on the masked temperature
workload (N_side 256, l_max 512), whose iteration ratio turns the FP64 form's
per-iteration time at the benchmark size into its time to 1e-6 (a stated
model, checked by that measured pair); SHT pairs/s; the mixed-geometry
chains; measured FMA peaks for the arithmetic rooflines.

--impl reference times the FP64 CPU oracle (test infrastructure) on bounded
ring samples of the same workload, and once on the full grid to check the
extrapolation.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "CG iters/sec & SHT pairs/sec @Nside=1024,lmax=2048; mixed vs FP64 @1e-6 resid"
UNIT = "CG iterations/s"
NSIDE, LMAX, NB = 1024, 2048, 8   # the benchmark workload; --nside/--lmax/--batch shrink it for profiling
CLASS_NAMES = ["leg_synth_fp32", "leg_analysis_fp32", "ring_fft_fp32", "leg_synth_fp64",
               "leg_analysis_fp64", "ring_fft_fp64", "vector", "precond_diag"]
# CUDA sources of each kernel class (a traffic figure measured by ncu is
# reported only while these files are unchanged since the capture)
CLASS_SOURCES = {
    "leg_synth_fp32": ["legendre_tc.cu", "legendre_kernels.cuh", "legendre32.cu"],
    "leg_analysis_fp32": ["legendre_tc.cu", "legendre_kernels.cuh", "legendre32.cu"],
    "ring_fft_fp32": ["ringfft.cu"],
    "leg_synth_fp64": ["legendre_df.cu", "df.cuh", "legendre_kernels.cuh", "legendre64.cu"],
    "leg_analysis_fp64": ["legendre_df.cu", "df.cuh", "legendre_g64.cu", "legendre64.cu"],
    "ring_fft_fp64": ["ringfft.cu"],
}


# ----------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def sources_hash(names) -> str:
    h = hashlib.sha256()
    for n in sorted(names):
        with open(os.path.join(ROOT, "paper_2306_15511_gb300", "csrc", n), "rb") as f:
            h.update(n.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def traffic_record(cls: str, launch_units: float):
    """DRAM bytes per launch of a kernel class from the committed ncu record
    (profiles/traffic.json: bytes per unit of work, the sources' hash at the
    capture), scaled to this launch's units; None once the sources changed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or cls not in CLASS_SOURCES:
        return None
    with open(path) as f:
        rec = json.load(f).get(cls)
    if not rec or rec.get("sources_sha") != sources_hash(CLASS_SOURCES[cls]):
        return None
    return rec["dram_bytes_per_unit"] * launch_units


def contraction_flops(nalm, npairs, nmaps_t, nmaps_p):
    """Algorithmic flops of the Legendre contraction alone (what the tensor
    cores do in the tensor-core kernels): per (l, m, ring pair) 4 per
    temperature map and 16 per (Q, U) pair."""
    return float(nalm) * float(npairs) * (4 * nmaps_t + 16 * nmaps_p)


def legendre_flops(nalm, npairs, nmaps_t, nmaps_p):
    """Algorithmic flops of one Legendre pass (one direction): per (l, m,
    ring pair) 3 shared recurrence flops + 4 per temperature map, and for
    spin 2 8 shared + 16 per (Q, U) pair."""
    pr = float(nalm) * float(npairs)
    f = 0.0
    if nmaps_t:
        f += pr * (3 + 4 * nmaps_t)
    if nmaps_p:
        f += pr * (8 + 16 * nmaps_p)
    return f


def ring_fft_flops(nside: int) -> float:
    """Algorithmic flops of one direction of the ring transforms of one map
    on a HEALPix grid: one complex DFT of length n per north / south ring pair
    (the pair's two real rings packed into one complex sequence), counted as
    5 n log2 n whatever algorithm computes it (Bluestein's overhead for
    non-power-of-two rings is not counted).  Polar pairs i = 1 .. N-1 have
    n = 4 i; the N + 1 equatorial pairs (the equator ring alone) n = 4 N."""
    f = 0.0
    for i in range(1, nside):
        n = 4 * i
        f += 5.0 * n * np.log2(n)
    n = 4 * nside
    f += (nside + 1) * 5.0 * n * np.log2(n)
    return f


def fma_peaks():
    """Measured FMA throughput (TFLOP/s) of this GPU, FP32 and FP64, and its SM count."""
    from paper_2306_15511_gb300.api import fma_peak
    sms, fp32 = fma_peak("fp32")
    _, fp64 = fma_peak("fp64")
    return {"sm_count": sms, "fp32_tflops": fp32, "fp64_tflops": fp64,
            "how": "8 independent FMA chains per thread, every SM filled, CUDA events, 2 flops per FMA"}


class Clocks:
    """nvidia-smi sampler (every 200 ms) running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def rank_summary(rep, ms_local: float, iters_local: float, steps: int):
    """Whole-job timing over replicas: the slowest rank's time per step and
    the sum of all ranks' iterations; value = iterations / time."""
    ms = rep.max(ms_local)
    total = rep.sum(iters_local)
    return ms, total, total / (ms * steps / 1000.0)


# ------------------------------------------------------------------ inputs
def make_inputs(plan, device, rank=0):
    """T+E+B workload (8 realizations, N_side 1024, l_max 2048) drawn on the
    device; d = Y B a + n with the library's own FP64 synthesis.  Ranks > 0
    draw fresh white noise w1 and w2 (independent chains)."""
    import torch
    from inputs import configs as C
    from inputs import philox as px
    from paper_2306_15511_gb300.replicas import w1_key, w2_key
    probs = C.teb_realizations(NB, NSIDE, LMAX, device=device)
    if rank:
        nalm = C.nalm(LMAX)
        for b, p in enumerate(probs):
            k1, k2 = w1_key(rank, b), w2_key(rank, b)
            p.w1 = torch.stack([C.white_alm(LMAX, k1, px.STREAM_W1, k * 2 * nalm, device)
                                for k in range(3)])
            p.w2 = torch.stack([px.normal_torch(k2, px.STREAM_W2, plan.npix, k * plan.npix, device)
                                for k in range(3)])
    p0 = probs[0]
    ls = torch.as_tensor(C.alm_lm(LMAX)[0], device=device)
    bl = torch.as_tensor(p0.bl, device=device)[ls]
    a = torch.stack([p.signal_alm for p in probs]) * bl          # [nb, 3, nalm]
    T = plan.alm2map(a[:, 0].contiguous())
    QU = plan.alm2map(a[:, 1:].contiguous(), spin=2)
    d = torch.cat([T[:, None], QU], dim=1) + torch.stack([p.noise_map for p in probs])
    w1 = torch.stack([p.w1 for p in probs]).contiguous()
    w2 = torch.stack([p.w2 for p in probs]).contiguous()
    ninv = torch.as_tensor(p0.ninv, device=device).contiguous()
    torch.cuda.synchronize()
    return {"cl": p0.cl, "bl": p0.bl, "ninv": ninv, "d": d.contiguous(), "w1": w1, "w2": w2,
            "fsky": p0.extra["fsky"]}


# ----------------------------------------------------------- CPU baseline
_ORACLE = {}


def _oracle_full():
    """Full-grid inputs of the T+E+B workload (N_side 1024, l_max 2048) for
    the FP64 CPU oracle: geometry, C_l, b_l, N^-1 and one alm vector."""
    if "full" in _ORACLE:
        return _ORACLE["full"]
    from inputs import configs as C
    from inputs import philox as px
    from oracle import sht as osht
    g = osht.healpix(NSIDE)
    tt = C.cl_damped(LMAX)
    ee = 0.05 * tt
    cl4 = np.stack([tt, ee, 1e-3 * ee, 0.3 * np.sqrt(tt * ee)])
    bl = C.gauss_beam(LMAX, 10.0 * C.ARCMIN)
    z, phi = C.pixel_centres(NSIDE)
    hits = C.hits_proxy(z, phi)
    masked = C.latitude_cut(z, 20.0) | C.point_source_holes(z, phi, 200, 1.0, 4)
    ninv = np.stack([np.where(masked, 0.0, hits / 30.0 ** 2), np.where(masked, 0.0, hits / 42.0 ** 2)])
    x = np.stack([C.white_alm(LMAX, 9, px.STREAM_W1, k * 2 * C.nalm(LMAX)) for k in range(3)])
    _ORACLE["full"] = (g, cl4, bl, ninv, x)
    return _ORACLE["full"]


def _oracle_problem(nsub_stride=32):
    """The oracle's T+E+B operator restricted to every nsub_stride-th ring."""
    if nsub_stride in _ORACLE:
        return _ORACLE[nsub_stride]
    from oracle import solver as osol
    g, cl4, bl, ninv, x = _oracle_full()
    rings = np.arange(0, g.nring, nsub_stride)
    ninv_sub = np.stack([np.concatenate([ninv[c][g.ofs[r]:g.ofs[r] + g.nphi[r]] for r in rings])
                         for c in range(2)])
    prob = osol.Problem(g.subset(rings), LMAX, cl4, bl, ninv_sub)
    _ORACLE[nsub_stride] = (prob, x, g.nring, rings.size)
    return _ORACLE[nsub_stride]


def oracle_threads(n: int = 0) -> int:
    """Set (n > 0) and return the oracle's worker threads."""
    from oracle import _lib
    return int(_lib.lib().orc_set_threads(int(n)))


def oracle_sample(strides=(32, 16)):
    """Time one T+E+B operator application of the FP64 oracle on every
    s-th ring of the N_side 1024 grid for each stride s, fit
    t = a + b x (rings) through those samples (a: the ring-independent
    harmonic work, b: the cost per ring) and extrapolate to all rings and a
    batched CG iteration of 8 realizations."""
    pts = []
    for st in strides:
        prob, x, nring, nsub = _oracle_problem(st)
        t0 = time.perf_counter()
        prob.matvec(x)
        pts.append((nsub, time.perf_counter() - t0))
    (n1, t1), (n2, t2) = min(pts), max(pts)
    b = (t2 - t1) / (n2 - n1) if n2 > n1 else t2 / n2
    a = t2 - b * n2
    if a < 0.0 or b < 0.0:          # timing noise: fall back to scaling the denser sample
        a, b = 0.0, t2 / n2
    per_real = a + b * nring
    desc = ", ".join(f"{t:.2f} s on {n} rings" for n, t in sorted(pts))
    return {"value": 1.0 / (per_real * NB), "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
            "per_realization_s": per_real,
            "sample": (f"one FP64 T+E+B operator application of 1 realization on ring subsets of "
                       f"the {nring}-ring grid (every {'th / '.join(str(s_) for s_ in strides)}th "
                       f"ring): {desc}; fitted a + b x rings (a = {a:.2f} s, b = {1e3 * b:.2f} ms) "
                       f"and extrapolated to {nring} rings, then x{NB} realizations")}


def oracle_full_grid():
    """One T+E+B operator application of the FP64 oracle on the whole grid
    (1 realization), timed: the check of the ring-sample extrapolation."""
    from oracle import solver as osol
    g, cl4, bl, ninv, x = _oracle_full()
    prob = osol.Problem(g, LMAX, cl4, bl, ninv)
    t0 = time.perf_counter()
    prob.matvec(x)
    return time.perf_counter() - t0


def oracle_extras():
    """The oracle's other figures (FP64, host cores): SHT pairs/s on the
    masked temperature grid (N_side 256, l_max 512), CG iterations/s on the
    full-sky workload (solved to its 1e-8) and on the masked one (5
    iterations), and the benchmark operator on one core."""
    from inputs import configs as C
    from oracle import sht as osht
    from oracle import solver as osol
    out = {"cores": oracle_threads()}
    p = C.masked_temperature(256, 512)
    g = osht.healpix(256)
    t0 = time.perf_counter()
    osht.alm2map_adjoint(g, 512, osht.alm2map(g, 512, p.signal_alm[0]))
    out["sht_pairs_per_s_nside256_lmax512"] = 1.0 / (time.perf_counter() - t0)
    prob = osol.Problem(g, 512, p.cl, p.bl, p.ninv)
    b = prob.rhs(p.noise_map, p.w1, p.w2)
    t0 = time.perf_counter()
    _, it, _ = osol.pcg(prob, b, 1e-6, maxiter=5)
    out["cg_iters_per_s_nside256_lmax512"] = it / (time.perf_counter() - t0)
    q = C.fullsky_temperature()
    g0 = osht.healpix(q.nside)
    prob0 = osol.Problem(g0, q.lmax, q.cl, q.bl, q.ninv)
    b0 = prob0.rhs(q.noise_map, q.w1, q.w2)
    t0 = time.perf_counter()
    _, it0, hist = osol.pcg(prob0, b0, q.tol, maxiter=1000)
    el = time.perf_counter() - t0
    out["fullsky_nside32_lmax64"] = {"iterations_to_1e-8": it0, "s": el, "cg_iters_per_s": it0 / el}
    nthr = oracle_threads()
    try:
        oracle_threads(1)
        s1 = oracle_sample(strides=(128, 64))
        out["single_core"] = {"value": s1["value"], "unit": UNIT, "sample": s1["sample"]}
    finally:
        oracle_threads(nthr)
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    full_s = oracle_full_grid()
    for _ in range(min(args.warmup, 1)):
        oracle_sample()
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample())
    el = time.perf_counter() - t0
    v = float(np.median([x["value"] for x in vals]))
    pred = float(np.median([x["per_realization_s"] for x in vals]))
    extras = oracle_extras() if not getattr(args, "no_extras", False) else {}
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"T+E+B constrained realizations, HEALPix N_side={NSIDE}, "
                                   f"l_max={LMAX}, batch {NB}, tol 1e-6",
                       "global_batch": NB, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "fit_check": {"full_grid_operator_s": full_s, "fit_predicted_s": pred,
                          "rel_err": (pred - full_s) / full_s,
                          "full_grid_value": 1.0 / (full_s * NB)},
            "extras": extras, "wall_s": el}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
def _event_time(fn, reps=1):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        r = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps, r


def _apply_sizes(args):
    global NSIDE, LMAX, NB
    NSIDE, LMAX, NB = args.nside, args.lmax, args.batch


def gpu_rank(args):
    """One rank of the GPU arm (rank 0 prints the JSON line)."""
    import torch
    from paper_2306_15511_gb300 import Plan
    from paper_2306_15511_gb300.replicas import Replicas

    _apply_sizes(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rep = Replicas("nccl", dev)
    rank, world = rep.rank, rep.world

    plan = Plan(nside=NSIDE, lmax=LMAX, max_batch=NB, spin2=True)
    inp = make_inputs(plan, dev, rank=rank)
    kw = dict(tol=1e-6, mode=args.mode, maxiter=args.iters_per_step,
              reliable_delta=args.reliable_delta, check_every=args.check_every,
              allow_not_converged=True, fp64_arith=args.fp64_arith, precond=args.precond,
              lowl_lmax=args.lowl_lmax, block_lmax=args.block_lmax)
    out = torch.empty(NB, 3, plan.nalm, dtype=torch.complex128, device=dev)

    def step(profile=False, **over):
        k = dict(kw)
        k.update(over)
        return plan.cg_sample(inp["cl"], inp["bl"], inp["ninv"], inp["d"], inp["w1"], inp["w2"],
                              out=out, profile=profile, **k)[1]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rep.barrier()
    clocks = Clocks(local)
    clocks.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    stats = [step() for _ in range(args.steps)]
    e1.record(st)
    torch.cuda.synchronize()
    ck = clocks.stop()
    rep.barrier()
    ms_local = e0.elapsed_time(e1) / args.steps
    iters_local = float(sum(s["iterations"] for s in stats))
    ms, iters_all, value = rank_summary(rep, ms_local, iters_local, args.steps)
    launches = int(sum(s["launches"] for s in stats))

    # ---------------------------------------------------------- e2e (host)
    e2e = None
    if not args.no_e2e:
        hd = inp["d"].cpu().pin_memory()
        hw1 = inp["w1"].cpu().pin_memory()
        hw2 = inp["w2"].cpu().pin_memory()
        hn = inp["ninv"].cpu().pin_memory()
        hout = torch.empty(NB, 3, plan.nalm, dtype=torch.complex128).pin_memory()
        ke = max(1, min(args.steps, args.e2e_steps))
        torch.cuda.synchronize()
        rep.barrier()
        t0 = time.perf_counter()
        e2e_stats = [plan.cg_sample(inp["cl"], inp["bl"], hn, hd, hw1, hw2, out=hout, **kw)[1]
                     for _ in range(ke)]
        torch.cuda.synchronize()
        el = rep.max(time.perf_counter() - t0)
        it_e = rep.sum(float(sum(s["iterations"] for s in e2e_stats)))
        h2d = hd.numel() * 8 + hw2.numel() * 8 + hw1.numel() * 16 + hn.numel() * 8
        e2e = {"value": it_e / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(hout.numel() * 16), "steps": ke}

    if rank != 0:
        rep.close()
        return 0

    # ------------------------------------------ profiled step (kernel shares)
    sp = step(profile=True)
    kms = np.asarray(sp["kernel_ms"], dtype=np.float64)
    kcnt = np.asarray(sp["kernel_launches"], dtype=np.int64)
    inner, outer = sp["iterations"], sp["fp64_matvecs"]
    peaks_alu = fma_peaks()

    # the extras and the CPU baseline describe one GPU: measured at N = 1 only
    extras = {}
    if not args.no_extras and world == 1:
        extras = measure_extras(plan, inp, dev, kw, step, full_solve=not args.no_full_solve)

    # ------------------------------------------------------------ roofline
    # One entry per kernel class with the resource that bounds it and the
    # class's algorithmic work over its CUDA-event time in the profiled step
    # (per-launch averages: the work of one launch over its mean duration);
    # "roofline" is the class with the largest share.
    #  - tensor-core Legendre kernels (mode mixed_tc): the contraction's
    #    flops against the measured sustained bf16 tensor rate (three bf16
    #    products per FP32-accurate multiply-add are issued on top);
    #  - CUDA-core FP32 Legendre kernels (mode mixed): all flops against the
    #    measured FP32 FMA rate;
    #  - FP64-accurate Legendre kernels: in double-FP32 (the mixed modes'
    #    default) against the measured FP32 FMA rate / 6 (a double-FP32 flop
    #    costs about six FP32 operations), in native FP64 against the
    #    measured FP64 FMA rate;
    #  - FP32 ring stage: HBM, the bytes of the Fourier coefficients read and
    #    written plus the N^-1 map;
    #  - FP64 ring stage: the measured FP64 FMA rate, with 5 n log2 n flops
    #    per ring-pair transform and direction.
    peaks, src = measured_peaks()
    fp32_peak, fp64_peak = peaks_alu["fp32_tflops"], peaks_alu["fp64_tflops"]
    bf16_sus = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    nalm, npairs = plan.nalm, 2 * NSIDE
    nring, npix = 4 * NSIDE - 1, 12 * NSIDE * NSIDE
    per_pass = legendre_flops(nalm, npairs, NB, NB)           # T and Q/U launches of one pass
    per_pass_c = contraction_flops(nalm, npairs, NB, NB)
    df = args.fp64_arith == "df64" or (args.fp64_arith == "default" and args.mode != "fp64")
    coef32 = 2.0 * 3 * NB * nring * (LMAX + 1) * 8           # read + write, T, Q, U of NB maps
    fft1 = ring_fft_flops(NSIDE) * 3 * NB                     # one direction, all maps
    # work of the whole profiled step per class, and the units of one launch
    work = {0: per_pass_c * inner if args.mode == "mixed_tc" else per_pass * inner,
            1: per_pass_c * inner if args.mode == "mixed_tc" else per_pass * inner,
            2: (coef32 + 2 * npix * 4) * inner,
            3: per_pass * outer, 4: per_pass * (outer + 1),
            5: fft1 * (2 * outer + 1)}
    coef_units = 3 * NB * nring * (LMAX + 1)                 # Fourier coefficients of one pass
    roofs = {}
    for c in range(len(CLASS_NAMES)):
        if kms[c] <= 0 or c not in work:
            continue
        t = kms[c] / 1000.0
        name = CLASS_NAMES[c]
        if c in (0, 1):
            if args.mode == "mixed_tc":
                r = {"bound": "tensor", "achieved": work[c] / t / 1e12, "peak": bf16_sus, "unit": "TFLOP/s",
                     "peak_source": f"{src} bf16 (sustained)"}
            else:
                r = {"bound": "alu", "achieved": work[c] / t / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                     "peak_source": "measured FP32 FMA rate (probe)"}
        elif c in (3, 4):
            if df:
                r = {"bound": "alu", "achieved": work[c] / t / 1e12, "peak": fp32_peak / 6.0,
                     "unit": "TFLOP/s", "peak_source": "measured FP32 FMA rate (probe) / 6 (double-FP32)"}
            else:
                r = {"bound": "alu", "achieved": work[c] / t / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "peak_source": "measured FP64 FMA rate (probe)"}
        elif c == 2:
            r = {"bound": "hbm", "achieved": work[c] / t / 1e9, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                 "peak_source": f"{src} copy bandwidth"}
        else:
            r = {"bound": "alu", "achieved": work[c] / t / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                 "peak_source": "measured FP64 FMA rate (probe); 5 n log2 n flops per ring-pair DFT"}
        r["frac"] = r["achieved"] / r["peak"] if r["peak"] else None
        r["ms_per_launch"] = float(kms[c]) / max(1, int(kcnt[c]))
        r["launches"] = int(kcnt[c])
        # DRAM traffic of one pass (all launches of one operator direction) from
        # the committed ncu record, scaled by the Fourier coefficients per pass
        tr = traffic_record(name, coef_units) if c in (0, 1, 2) else None
        r["traffic"] = tr
        r["traffic_per"] = "pass" if tr is not None else None
        if c == 2:
            r["algorithmic_bytes_per_pass"] = coef32 + 2 * npix * 4
        r["kernel"] = name
        roofs[name] = r
    dom = CLASS_NAMES[int(np.argmax(kms))]
    roof = roofs.get(dom) or {"bound": "hbm", "achieved": None, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                              "frac": None, "traffic": None, "kernel": dom}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = oracle_sample(strides=(16, 4))
            cpu.pop("per_realization_s", None)
        except Exception as e:  # the oracle is test infrastructure; report why it is missing
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {e}"}

    total_kms = float(np.sum(kms))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32" if args.mode == "mixed" else "f32/bf16x3" if args.mode == "mixed_tc" else "f64") +
                 ("+df64" if df else "+f64") + (" (f64 ring FFTs)" if args.mode != "fp64" else ""),
        "data": "synthetic",
        "config": {"workload": f"T+E+B constrained realizations, HEALPix N_side={NSIDE}, "
                               f"l_max={LMAX}, batch {NB} per GPU, mixed FP32 PCG + FP64-accurate "
                               f"residual replacement" + (" (double-FP32 Legendre sums)" if df else "") +
                               f", tol 1e-6, {args.iters_per_step} FP32 "
                               f"iterations per step" +
                               (", Legendre sums on the tensor cores (bf16 hi/lo split)"
                                if args.mode == "mixed_tc" else ""),
                   "mode": args.mode, "fp64_arith": args.fp64_arith, "iters_per_step": args.iters_per_step,
                   "precond": args.precond + (f" (l_c {args.lowl_lmax or 32})" if args.precond == "lowl" else
                                              f" (l_b {args.block_lmax or min(LMAX, 1024)})"
                                              if args.precond == "azim" else ""),
                   "global_batch": NB * world, "fsky": inp["fsky"], "parallelism": f"replicas x{world}",
                   "timed_path": "default (PCG iteration replayed as a CUDA graph)",
                   "value_counts": "FP32 PCG iterations (FP64-accurate residual replacements not counted)",
                   "l2": "inputs larger than L2 (d, w2: 2.4 GB each)"},
        "e2e": e2e, "gpu_launches": launches, "clocks": ck, "roofline": roof, "rooflines": roofs,
        "time_to_solution": _time_to_solution(extras),
        "alu_peaks": peaks_alu,
        "cpu_baseline": cpu,
        "step": {"fp32_iterations": iters_local / len(stats),
                 "fp64_residual_replacements": float(np.mean([s["fp64_matvecs"] for s in stats])),
                 "rel_residual_after_step": max(s["rel_residual"] for s in stats),
                 "ms_rhs": float(np.mean([s["ms_rhs"] for s in stats]))},
        "profiled_step": {"note": "one step with per-class CUDA events (eager launches), after the timed steps",
                          "ms_total": sp["ms_total"], "iterations": inner, "fp64_matvecs": outer},
        "kernel_share": {CLASS_NAMES[i]: round(float(kms[i]) / total_kms, 4)
                         for i in range(len(CLASS_NAMES)) if total_kms > 0},
        "kernel_ms_per_step": {CLASS_NAMES[i]: float(kms[i]) for i in range(8)},
        "kernel_launches_per_step": {CLASS_NAMES[i]: int(kcnt[i]) for i in range(8)},
        "extras": extras,
    }
    print(json.dumps(line), flush=True)
    rep.close()
    return 0


def _time_to_solution(extras):
    """The full solves to 1e-6 of the extras, fastest first."""
    out = []
    for key, v in extras.items():
        if key.startswith("mixed_full_solve") and isinstance(v, dict):
            out.append({"precond": v["precond"], "s": v["time_to_1e-6_s"], "fp32_iterations": v["iterations"],
                        "converged": v["converged"], "rel_residual": v["rel_residual"]})
    return sorted(out, key=lambda d: d["s"]) or None


def run_gpu(args):
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        from paper_2306_15511_gb300.replicas import launch_local
        launch_local(args.gpus, gpu_rank, (args,))
        return 0
    return gpu_rank(args)


def _sht_rate(plan, dev, spin, nb, prec, reps):
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    ct = torch.complex64 if prec in ("fp32", "tc32") else torch.complex128
    shape = (nb, 2, plan.nalm) if spin == 2 else (nb, plan.nalm)
    a = torch.randn(*shape, dtype=ct, device=dev, generator=g)
    kw = {"tensor_cores": prec == "tc32", "double_float": prec == "df64"}

    def pair():
        return plan.alm2map_adjoint(plan.alm2map(a, spin=spin, **kw), spin=spin, **kw)

    pair()
    t, _ = _event_time(pair, reps)
    return nb / t


def measure_extras(plan, inp, dev, kw, step, full_solve=True):
    import torch
    ex = {}
    if full_solve:
        # to 1e-6 with the bench's preconditioner, then with the other one
        # to 1e-6 with the bench's preconditioner and with the others
        pcs = [kw["precond"]] + [x for x in ("azim", "lowl", "diag") if x != kw["precond"]]
        for pc in pcs:
            key = "mixed_full_solve" if pc == kw["precond"] else f"mixed_full_solve_{pc}"
            kwf = dict(kw)
            kwf["maxiter"] = 6000
            kwf["precond"] = pc
            t, (_, st) = _event_time(lambda: plan.cg_sample(inp["cl"], inp["bl"], inp["ninv"], inp["d"],
                                                            inp["w1"], inp["w2"], **kwf))
            lbl = f" (l_b {kw['block_lmax'] or min(LMAX, 1024)})" if pc == "azim" else ""
            ex[key] = {"precond": pc + lbl, "time_to_1e-6_s": t,
                       "iterations": st["iterations"],
                       "fp64_matvecs": st["fp64_matvecs"], "converged": bool(st["converged"]),
                       "rel_residual": st["rel_residual"], "ms_setup": st["ms_setup"], "ms_rhs": st["ms_rhs"]}
    # the headline steps with native FP64 residual replacements and RHS
    t, sts = _event_time(lambda: [step(fp64_arith="fp64") for _ in range(2)])
    ex["steps_fp64_arith_fp64"] = {"value": sum(s["iterations"] for s in sts) / (2 * t), "unit": UNIT,
                                   "ms_per_step": 1000.0 * t,
                                   "fp64_matvecs_per_step": sts[0]["fp64_matvecs"]}
    # plain FP64 PCG: per-iteration time from two budgets (4 and 8 iterations),
    # so the RHS, the preconditioner and the final residual drop out
    for arith in ("fp64", "df64"):
        plan.cg_sample(inp["cl"], inp["bl"], inp["ninv"], inp["d"], inp["w1"], inp["w2"], tol=1e-6,
                       mode="fp64", maxiter=1, allow_not_converged=True, fp64_arith=arith)   # tuning
        runs = {}
        for nit in (4, 8):
            t, (_, st) = _event_time(lambda: plan.cg_sample(
                inp["cl"], inp["bl"], inp["ninv"], inp["d"], inp["w1"], inp["w2"], tol=1e-6,
                mode="fp64", maxiter=nit, check_every=4, allow_not_converged=True, fp64_arith=arith))
            runs[nit] = (t, st)
        per_it = (runs[8][0] - runs[4][0]) / (runs[8][1]["iterations"] - runs[4][1]["iterations"])
        ex[f"fp64_form_{arith}"] = {"s_per_iteration": per_it, "iters_per_s": 1.0 / per_it,
                                    "fixed_s": runs[4][0] - 4 * per_it,
                                    "how": "two calls with 4 and 8 PCG iterations, difference / 4"}
    if full_solve:
        # both forms solved to 1e-6 at this size with the azimuthal blocks,
        # which the first mixed solve set up and the plan keeps (a chain's
        # later samples): the mixed form again, and the plain FP64 PCG with
        # double-FP32 Legendre sums (FP64-accurate: within 1e-12 of the
        # native FP64 kernels); the native FP64 form's time is its measured
        # per-iteration time times the measured iteration count
        def full(mode, arith, maxiter):
            return _event_time(lambda: plan.cg_sample(
                inp["cl"], inp["bl"], inp["ninv"], inp["d"], inp["w1"], inp["w2"], tol=1e-6, mode=mode,
                maxiter=maxiter, check_every=8, precond="azim", fp64_arith=arith, allow_not_converged=True))
        tm, (_, sm) = full(kw["mode"], kw.get("fp64_arith", "default"), 6000)
        tf, (_, sf) = full("fp64", "df64", 1000)
        f64 = ex["fp64_form_fp64"]
        native = f64["fixed_s"] + sf["iterations"] * f64["s_per_iteration"]
        ex["both_forms_to_1e-6_azim"] = {
            "mixed": {"s": tm, "iterations": sm["iterations"], "fp64_matvecs": sm["fp64_matvecs"],
                      "converged": bool(sm["converged"]), "rel_residual": sm["rel_residual"],
                      "ms_setup": sm["ms_setup"]},
            "fp64_df64": {"s": tf, "iterations": sf["iterations"], "converged": bool(sf["converged"]),
                          "rel_residual": sf["rel_residual"], "ms_setup": sf["ms_setup"]},
            "fp64_native_s": native,
            "speedup_vs_fp64_df64": tf / tm, "speedup_vs_fp64_native": native / tm,
            "note": ("blocks kept from the first solve; native FP64 = its measured fixed cost + the FP64 "
                     "form's measured iteration count x its measured s/iteration")}
        # the azimuthal blocks over fewer multipoles: a cheaper set-up (the
        # factorizations grow as l_b^4), more iterations
        for lb in (512, 256):
            kwf = dict(kw)
            kwf.update(maxiter=6000, precond="azim", block_lmax=lb)
            t, (_, st) = _event_time(lambda: plan.cg_sample(inp["cl"], inp["bl"], inp["ninv"], inp["d"],
                                                            inp["w1"], inp["w2"], **kwf))
            ex[f"mixed_full_solve_azim_lb{lb}"] = {
                "precond": f"azim (l_b {lb})", "time_to_1e-6_s": t, "iterations": st["iterations"],
                "fp64_matvecs": st["fp64_matvecs"], "converged": bool(st["converged"]),
                "rel_residual": st["rel_residual"], "ms_setup": st["ms_setup"], "ms_rhs": st["ms_rhs"]}
    ex["masked_nside256"] = measure_masked_pair(dev, kw["precond"])
    if "mixed_full_solve" in ex:
        fs = ex["mixed_full_solve"]
        ratio = ex["masked_nside256"]["iteration_ratio_fp64_over_mixed"]
        f64 = ex["fp64_form_fp64"]
        it_model = fs["iterations"] * ratio
        ex["fp64_form_time_to_1e-6_model"] = {
            "s": f64["fixed_s"] + it_model * f64["s_per_iteration"],
            "iterations_model": it_model,
            "model": ("measured fixed cost + measured s/iteration x (the mixed solve's FP32 iterations at "
                      "this size x the FP64 / mixed iteration ratio measured to 1e-6 on the masked "
                      "N_side 256 workload, both with the bench's preconditioner)")}
        ex["mixed_speedup_time_to_1e-6"] = ex["fp64_form_time_to_1e-6_model"]["s"] / fs["time_to_1e-6_s"]
    sht = {}
    for spin in (0, 2):
        for nb in (1, NB):
            for prec, reps in (("fp32", 3), ("tc32", 3), ("fp64", 1), ("df64", 1)):
                sht[f"spin{spin}_batch{nb}_{prec}"] = _sht_rate(plan, dev, spin, nb, prec, reps)
    ex["sht_pairs_per_s"] = sht
    ex["sht_pairs_per_s_note"] = ("one alm2map + one alm2map_adjoint per map (spin 2: per (E, B) -> "
                                  "(Q, U) map pair), N_side 1024, l_max 2048, CUDA events")
    ex["chains"] = measure_chains(dev)
    torch.cuda.synchronize()
    return ex


def measure_masked_pair(dev, precond="diag"):
    """Both forms solved to 1e-6 on the masked temperature workload
    (N_side 256, l_max 512): iterations and time to 1e-6 of the plain FP64
    PCG (native FP64) and of the mixed solver (tensor cores), with the given
    preconditioner and, for comparison, the other one."""
    import torch
    from inputs import configs as C
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(256, 512)
    plan = Plan(nside=256, lmax=512)
    ls = torch.as_tensor(C.alm_lm(512)[0], device=dev)
    a = torch.as_tensor(p.signal_alm[0], device=dev) * torch.as_tensor(p.bl, device=dev)[ls]
    d = (plan.alm2map(a[None].contiguous()) + torch.as_tensor(p.noise_map, device=dev))[:, None].contiguous()
    args = (p.cl, p.bl, torch.as_tensor(p.ninv, device=dev), d,
            torch.as_tensor(p.w1[None], device=dev).contiguous(), torch.as_tensor(p.w2[None], device=dev).contiguous())
    out = {"precond": precond}
    other = "azim" if precond != "azim" else "diag"
    for pc, sfx in ((precond, ""), (other, f"_{other}")):
        for mode in ("mixed_tc", "fp64"):
            plan.cg_sample(*args, tol=1e-6, mode=mode, maxiter=2, allow_not_converged=True, precond=pc)   # tuning
            t, (_, st) = _event_time(lambda: plan.cg_sample(*args, tol=1e-6, mode=mode, maxiter=8000,
                                                            check_every=8, precond=pc))
            out[mode + sfx] = {"time_to_1e-6_s": t, "iterations": st["iterations"],
                               "fp64_matvecs": st["fp64_matvecs"], "converged": bool(st["converged"]),
                               "rel_residual": st["rel_residual"], "ms_setup": st["ms_setup"]}
    out["iteration_ratio_fp64_over_mixed"] = out["fp64"]["iterations"] / max(1, out["mixed_tc"]["iterations"])
    out["speedup_time_to_1e-6"] = out["fp64"]["time_to_1e-6_s"] / out["mixed_tc"]["time_to_1e-6_s"]
    plan.close()
    return out


def measure_chains(dev, nchains=64):
    """Mixed-geometry chains: 64 independent chains with N_side in {64, 128, 256},
    l_max in {2 N_side, 3 N_side - 1} and their own signal amplitudes (six
    geometries), all solved to 1e-6 in one chains call, three ways: the groups
    concurrently on their plans' streams (tensor-core or CUDA-core FP32
    Legendre sums), and grouped (SHTG_GROUPED: every stage of the FP32
    iteration one launch over all six geometries); each with the azimuthal
    block and with the diagonal preconditioner."""
    import torch
    from inputs import configs as C
    from paper_2306_15511_gb300 import Plan, chains_sample
    groups = {}
    for ch in C.mixed_geometry_chains(nchains):
        groups.setdefault((ch.nside, ch.lmax), []).append(ch)
    req = []
    for (ns, L), chs in sorted(groups.items()):
        plan = Plan(nside=ns, lmax=L, max_batch=len(chs))
        ls = torch.as_tensor(C.alm_lm(L)[0], device=dev)
        bl = torch.as_tensor(chs[0].bl, device=dev)
        a = torch.stack([torch.as_tensor(ch.signal_alm[0], device=dev) for ch in chs]) * bl[ls]
        n = torch.stack([torch.as_tensor(ch.noise_map[0], device=dev) for ch in chs])
        d = (plan.alm2map(a.contiguous()) + n)[:, None].contiguous()
        req.append({"plan": plan, "cl": C.cl_flat(L), "bl": chs[0].bl,
                    "ninv": torch.as_tensor(chs[0].ninv, device=dev).contiguous(), "d": d,
                    "w1": torch.stack([torch.as_tensor(ch.w1, device=dev) for ch in chs]).contiguous(),
                    "w2": torch.stack([torch.as_tensor(ch.w2, device=dev) for ch in chs]).contiguous(),
                    "cl_scale": [ch.extra["amp"] for ch in chs]})
    runs = {}
    for precond in ("azim", "diag"):
        for name, kw in (("concurrent_tc", {"mode": "mixed_tc"}), ("concurrent", {"mode": "mixed"}),
                         ("grouped", {"mode": "mixed", "grouped": True})):
            chains_sample(req, tol=1e-6, maxiter=4000, precond=precond, **kw)   # tuning, warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = chains_sample(req, tol=1e-6, maxiter=4000, precond=precond, **kw)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            runs[f"{name}_{precond}"] = {
                "time_to_1e-6_s": el, "chains_per_s": nchains / el,
                "iterations": [st["iterations"] for _, st in res],
                "launches": int(sum(st["launches"] for _, st in res)),
                "converged": all(st["converged"] == 1 for _, st in res)}
    best = min(runs, key=lambda k: runs[k]["time_to_1e-6_s"])
    return {"chains": nchains, "groups": len(req),
            "geometries": [f"N_side {ns} l_max {L} x{len(chs)}" for (ns, L), chs in sorted(groups.items())],
            "fastest": best, "time_to_1e-6_s": runs[best]["time_to_1e-6_s"],
            "chains_per_s": runs[best]["chains_per_s"], "runs": runs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="shtg", choices=["shtg", "reference"])
    ap.add_argument("--iters-per-step", type=int, default=160)
    ap.add_argument("--mode", default="mixed_tc", choices=["mixed", "mixed_tc"],
                    help="inner FP32 operator: CUDA-core or tensor-core Legendre sums")
    ap.add_argument("--fp64-arith", default="default", choices=["default", "fp64", "df64"],
                    help="arithmetic of the FP64-accurate steps (default: double-FP32 in the mixed modes)")
    ap.add_argument("--nside", type=int, default=NSIDE, help="profiling only: smaller grid")
    ap.add_argument("--lmax", type=int, default=LMAX, help="profiling only: smaller l_max")
    ap.add_argument("--batch", type=int, default=NB, help="profiling only: fewer realizations")
    ap.add_argument("--no-full-solve", action="store_true")
    ap.add_argument("--precond", default="diag", choices=["none", "diag", "lowl", "azim"],
                    help="diagonal preconditioner of Sect. 4, two-level (exact inverse on l <= l_c), or "
                         "azimuthal blocks (App. A's per-m blocks from ring-averaged N^-1, l <= l_b)")
    ap.add_argument("--lowl-lmax", type=int, default=0, help="l_c of the two-level preconditioner (0: 32)")
    ap.add_argument("--block-lmax", type=int, default=0, help="l_b of the azimuthal blocks (0: 1024)")
    ap.add_argument("--reliable-delta", type=float, default=1e-2)
    ap.add_argument("--check-every", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    _apply_sizes(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
