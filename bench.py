#!/usr/bin/env python
"""Benchmark of the staggered phase-field fracture load step on GB300.

Workload (one GPU): eight 512x512 periodic plane-strain grids sharing one
synthetic Young's modulus field (E = exp(0.3 z)/mean, z Gaussian with
correlation length 32 px), ell = 4 px, nu = 0.2, G_c = 1, CG tolerance 1e-8,
one simulation per model variant {AT1, AT2} x {isotropic, strain-spectral} x
{crack-set, whole-domain irreversibility}, advanced together by the batched
mixed-precision path (FP32 fields, FP64 reductions).  A step is one
near-equilibrium load step (Algorithm 4) of all eight simulations.  The
simulations start from eps_bar_yy = 0.95 eps_M so that every timed step runs
the mechanics and phase-field solvers.

Metric: pixel-CG-iterations per second (pixels x (mechanics CG + BCCG
iterations), summed over simulations and GPUs) per unit wall time of the timed
load steps.  Also reported: load steps per second, p50/p99 step latency, the
plain per-simulation FP64 GPU path on the same grid, the live roofline of the
dominant kernel class, an end-to-end number through host buffers and the FP64
NumPy oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
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

N = 512
LC = 32.0
ELL = 4.0
NU = 0.2
TOL = 1e-8
PRELOAD = 0.95
VARIANTS = [(f, s, i) for f in ("AT1", "AT2") for s in ("ISOTROPIC", "SPECTRAL") for i in ("CRACK_SET", "DAMAGE")]
WORKLOAD = "grid512_lc32_ell4_8variants_batched_mixed"
GROUP_SIZE = 1
FP64_RUN = False      # --precision fp64: the same batched workload with FP64 fields (not the headline)
# Mechanics share of the iterations of the timed region (mechanics CG / (mechanics CG + BCCG)),
# as the GPU path measures it on this workload (the "iteration_mix" key of every run reports
# the current figure); the reference arm weights the oracle's per-iteration costs by it.
WORKLOAD_MECH_FRACTION = 0.53
# Loosest sub-solver tolerance at which the FP64 path still meets the 1e-5 relative-L2 bar
# against the FP64 oracle on the 64x64 workload's checkpoints (mechanics error <= 3.9e-6,
# phase field <= 3.2e-7 at 1e-6; 4.1e-5 on the mechanics at 1e-5): the FP64 path's setting
# for the equal-accuracy comparison.
EQUAL_ACCURACY_TOL = 1e-6
MIXED_MECH_TOL_FLOOR = 1e-6   # the library's floor on the FP32 mechanics tolerance


def workload_config(world=1):
    """The config dict both arms print (the workload and its effective stopping rules)."""
    return {"workload": WORKLOAD.replace("_mixed", "_fp64") if FP64_RUN else WORKLOAD, "grid": N,
            "simulations_per_gpu": len(VARIANTS),
            "variants": ["/".join(v) for v in VARIANTS], "ell_px": ELL, "lc_px": LC, "nu": NU,
            "tol": TOL,
            "effective_tolerances": {
                "mechanics": f"Newton residual <= max(tol, {MIXED_MECH_TOL_FLOOR:g}) ||C0:eps_bar|| in FP32 "
                             f"(the FP32 floor); inner CG to max(that, 1e-4 ||R||) for the spectral split",
                "phase_field": f"BCCG ||r|| <= tol ||r0|| on explicit residuals, or in FP32 the rounding-level stop "
                               f"(64 iterations without a new smallest explicit residual, or a confirming "
                               f"evaluation that improves less than 2x)"},
            "start": f"eps_bar_yy = {PRELOAD} eps_M",
            "precision": "FP64 fields and reductions" if FP64_RUN else "FP32 fields, FP64 reductions",
            "launch_groups": (f"{len(VARIANTS) // GROUP_SIZE} concurrent streams of {GROUP_SIZE} simulation(s)"
                              if GROUP_SIZE else "one launch group on one stream"),
            "l2": "inputs larger than L2: device working set "
                  f"{len(VARIANTS) * 23.6:.0f} MB > {L2_BYTES / 1e6:.0f} MB",
            "parallelism": f"replicas x{world}"}
L2_BYTES = 129e6
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0    # HBM3e nominal bandwidth of the part (context beside the measured peak)


def eps_m():
    from paper_2203_16467_gb300.inputs import eps_M
    return eps_M(1.0, NU, 1.0, ELL)


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
KERNEL_SOURCES = ("common.cuh", "fft.cuh", "ops.cuh", "kernels.cuh", "k_rowfwd.cu", "k_rowinv.cu", "k_col.cu",
                  "k_elem.cu", "launch.h")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_16467_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes (read + write) per launch of the kernel class from the committed ncu capture
    (one launch with every simulation active), scaled to the average launch of this run by the
    algorithmic bytes it moves; None when there is no capture or the kernel sources changed
    since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except Exception:
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k or d.get("source_hash") != kernel_source_hash() or not alg_bytes_per_launch:
        return None
    return k["dram_bytes_per_launch"] * alg_bytes_per_launch / k["algorithmic_bytes_per_launch"]


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                return float(v["value"] if isinstance(v, dict) else v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------- oracle sample (CPU)
def cpu_sample(n_mech, n_bccg):
    """Time the FP64 oracle on the workload's grid: n_mech mechanics CG iterations and
    n_bccg BCCG iterations (AT1, strain-spectral, crack set) from the preloaded state.
    Returns seconds per iteration of each."""
    from oracle import constitutive as cm
    from oracle import fourier, mechanics, phasefield
    from oracle.params import AT1, CRACK_SET, SPECTRAL, Params
    from paper_2203_16467_gb300.inputs import modulus_field
    E = modulus_field(N, N, LC, 0)
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=CRACK_SET, ell=ELL, nu=NU)
    lam, mu = cm.lame(E, NU)
    eb = np.array([[0.0, 0.0], [0.0, 1.2 * eps_m()]])
    eps = np.broadcast_to(eb, (N, N, 2, 2)).copy()
    phi = np.zeros((N, N))
    ts = time.perf_counter()
    tang = cm.Tangent(eps, phi, lam, mu, SPECTRAL)
    R = fourier.project(cm.stress(eps, phi, lam, mu, SPECTRAL)) + 1e-3 * fourier.project(
        np.random.default_rng(0).standard_normal((N, N, 2, 2)))
    t0 = time.perf_counter()
    mechanics.cg(lambda p: fourier.project(tang(p)), -R, 0.0, n_mech)
    t1 = time.perf_counter()
    psi = cm.psi_plus(eps, lam, mu, SPECTRAL)
    b = phasefield.minus_F_phi(phi, psi, par)
    vcon = phasefield.phi_con(phi, par) - phi
    t1b = time.perf_counter()
    phasefield.bccg(lambda x: phasefield.J_apply(x, psi, par), b, vcon, 0.0, 0.0, n_bccg)
    t2 = time.perf_counter()
    return (t1 - t0) / n_mech, (t2 - t1b) / n_bccg, t2 - ts


def run_cpu_sample_subprocess(n_mech, n_bccg):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench.cpu_sample({n_mech}, {n_bccg})))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_cpu_sample_all_cores(n_mech, n_bccg, procs=None):
    """The same oracle sample in one single-threaded process per host core, all started at one
    time after their imports (independent simulations, as the GPU path batches them).  Returns
    the mean per-iteration seconds of mechanics CG and BCCG under that contention, the process
    count and the wall time of the slowest process."""
    procs = procs or os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    t_start = time.time() + 8.0 + 0.05 * procs   # after every process has imported the oracle
    code = (f"import sys, json, time; sys.path.insert(0, {ROOT!r}); import bench, oracle.mechanics; "
            f"time.sleep(max(0.0, {t_start!r} - time.time())); "
            f"r = bench.cpu_sample({n_mech}, {n_bccg}); print(json.dumps([time.time(), r]))")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(procs)]
    ends, tms, tbs = [], [], []
    for p in ps:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        t_end, (tm, tb, _) = json.loads(out.strip().splitlines()[-1])
        ends.append(t_end)
        tms.append(tm)
        tbs.append(tb)
    return statistics.mean(tms), statistics.mean(tbs), procs, max(ends) - t_start


# ------------------------------------------------------------------------- reference arm (oracle)
def run_reference(args, rank):
    if rank != 0:
        return None
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    n_mech, n_bccg = 2, 16
    mech_t, bccg_t, steps = [], [], []
    for s in range(args.warmup + args.steps):
        tm, tb, tot = cpu_sample(n_mech, n_bccg)
        if s >= args.warmup:
            steps.append(tot)
            mech_t.append(tm)
            bccg_t.append(tb)
    f = WORKLOAD_MECH_FRACTION
    t_iter = f * statistics.mean(mech_t) + (1.0 - f) * statistics.mean(bccg_t)
    value = N * N / t_iter
    line = {"impl": "reference", "metric": "pixel_cg_iters_per_s", "value": value, "unit": "pixel-CG-iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(steps) / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.gpus),
            "reference": "FP64 NumPy oracle (the paper publishes no code)",
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "pixel-CG-iters/s", "cores": 1,
                             "sample": f"per step: {n_mech} mechanics CG + {n_bccg} BCCG iterations of the oracle "
                                       f"on one {N}x{N} AT1 strain-spectral grid (set-up excluded); value = pixels / "
                                       f"per-iteration time at the workload's iteration mix ({f:.2f} mechanics CG, "
                                       f"{1 - f:.2f} BCCG); {statistics.mean(mech_t):.3f} s and "
                                       f"{statistics.mean(bccg_t):.4f} s per iteration"},
            "e2e": {"value": value, "unit": "pixel-CG-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# ------------------------------------------------------------------------- our arm
def aggregate(elapsed, work, world, device="cpu"):
    """Replicas only: the slowest rank's time and the work summed over ranks.
    Returns (max elapsed, [summed work...]); world == 1 returns the inputs."""
    if world <= 1:
        return float(elapsed), [float(w) for w in work]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)] + [float(w) for w in work], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax.item()), [float(x) for x in t[1:].tolist()]


def bytes_per_px(es, nx, iso=False):
    """Algorithmic bytes per pixel of each kernel class (family, op) for one problem launch
    (iso: isotropic contact model, whose tangent does not read the strain)."""
    s_pc = 2 * es * (nx // 2 + 1) / nx   # half-spectrum bytes per pixel per component
    return {
        (0, 1): (14 - 3 * iso) * es + 3 * s_pc,   # direction + tangent + row FFT: read p,r,eps*,phi,E; write p,S
        (2, 1): 6 * s_pc,                      # column pass Gamma: read + write S (3 comps)
        (1, 1): 15 * es + 3 * s_pc,            # row inverse + CG update + r.r: read S,th,r,p; write th,r
        (0, 3): 3 * es + 1 + s_pc,             # BCCG direction: read r,p,flag; write p,S
        (2, 9): 2 * s_pc,                      # column pass Laplacian of p + Parseval sum -> alpha
        (1, 9): 9 * es + 1 + s_pc,             # J p + iterate: read S,p,a,v,vcon,R,r; write v,R,r',flag
        (0, 4): es + s_pc,                     # explicit J v only: read v; write S
        (2, 6): 2 * s_pc,                      # explicit J v only: column pass Laplacian of v
        (1, 5): 7 * es + s_pc + 2,             # explicit residual only: read S,r,v,a,b,p,flag; write R,r,flag
        # the four-pass BCCG iteration (kernel variant): the direction pass (0, 3) as above, then
        (2, 4): 2 * s_pc,                      # column pass Laplacian of p
        (1, 4): 4 * es + s_pc,                 # J p, p.Jp, r.p: read S,p,a,r; write Jp
        (3, 11): 9 * es + 1,                   # iterate: read v,p,v_con,R,Jp,r; write v,R,r',flag
    }


KERNEL_NAMES = {(0, 1): "row_fwd_cg", (2, 1): "col_gamma_cg", (1, 1): "row_inv_cg", (0, 3): "row_fwd_bccg_dir",
                (2, 9): "col_lap_bccg_dir", (1, 9): "row_inv_bccg_iter",
                (0, 4): "row_fwd_bccg_v", (2, 6): "col_lap_bccg_v", (1, 5): "row_inv_bccg_explicit",
                (2, 4): "col_lap_bccg_dir_4pass", (1, 4): "row_inv_bccg_Jp_4pass", (3, 11): "elem_bccg_iter_4pass"}
BCCG3 = ((2, 9), (1, 9))            # the default three-pass iteration's own classes
BCCG4 = ((2, 4), (1, 4), (3, 11))   # the four-pass iteration's own classes


def kernel_bytes(reps_per_problem, isos, es, nx, ny, bccg4=False):
    """Algorithmic bytes of each kernel class summed over the problems' working launches."""
    out = {k: 0.0 for k in KERNEL_NAMES}
    for reps, iso in zip(reps_per_problem, isos):
        a = active_launches([reps], bccg4)
        b = bytes_per_px(es, nx, iso)
        for k in out:
            out[k] += a[k] * b[k] * nx * ny
    return out


def active_launches(reps_per_problem, bccg4=False):
    """Problem-launches of each kernel class that do work, from the per-step iteration counts
    (the explicit-residual chain works only in iterations that evaluate J v explicitly; bccg4:
    the BCCG iterations ran as four passes)."""
    cnt = {k: 0 for k in KERNEL_NAMES}
    for reps in reps_per_problem:
        for r in reps:
            cg, nw, pf, full = r["mech_cg_iters"], r["newton_iters"], r["bccg_iters"], r["bccg_full_iters"]
            cnt[(0, 1)] += cg
            cnt[(2, 1)] += cg
            cnt[(1, 1)] += cg
            for k in ((0, 3),) + (BCCG4 if bccg4 else BCCG3):
                cnt[k] += pf
            for k in ((0, 4), (2, 6), (1, 5)):
                cnt[k] += full
    return cnt


def make_problems(pff, stream, seed, precision, variants):
    from paper_2203_16467_gb300.inputs import modulus_field
    E = modulus_field(N, N, LC, seed)
    em = eps_m()
    probs = []
    for v in variants:
        p = pff.Problem(N, N, precision, stream=stream, E=E, model=v,
                        params=dict(nu=NU, ell=ELL, mech_tol=TOL, pf_tol=TOL, d_eps_bar=(0.0, em / 20, 0.0)))
        p.set_strain(None, (0.0, PRELOAD * em, 0.0))
        probs.append(p)
    return probs, E


def run_ours(args, rank, world, dev):
    import torch
    from paper_2203_16467_gb300 import pff
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()          # non-default stream: the library replays CUDA graphs on it
    torch.cuda.set_stream(stream)
    sp = stream.cuda_stream
    # kernel-variant autotuning on a throwaway batch of the same eight simulations from the same
    # start, launched as the timed region launches them (the choice stays set for the run)
    shape = None
    prec, es = (pff.FP64, 8) if FP64_RUN else (pff.MIXED, 4)
    if not args.no_tune and not FP64_RUN:
        tprobs, _ = make_problems(pff, sp, rank, pff.MIXED, VARIANTS)
        tb = pff.create_batch(len(tprobs), sum(pff.problem_bytes(N, N, pff.MIXED) for _ in tprobs), sp)
        pff.batch_set_group_size(tb, GROUP_SIZE)
        for p in tprobs:
            assert pff.batch_admit(tb, p.h) is not None
        chosen, scores, _ = pff.batch_autotune_kernels(tb, len(tprobs), steps_each=4)
        pff.destroy_batch(tb)
        for p in tprobs:
            p.close()
        names = [f"col1={c & 1},col3={(c >> 1) & 1},bccg={(c >> 2) & 1}" for c in range(8)]
        shape = {"chosen": {"column_pass_1_component_columns_per_block": 4 if chosen[0] == 0 else 2,
                            "column_pass_3_components_columns_per_block": 4 if chosen[1] == 0 else 2,
                            "bccg_passes_per_iteration": 3 if chosen[2] == 0 else 4},
                 "scores_pixel_iters_per_s": dict(zip(names, scores)),
                 "how": "pff_batch_autotune_kernels: 4 rounds (alternate rounds in reverse order), in each "
                        "every one of the 8 variant combinations runs 2 load steps (1 timed) of a separate batch "
                        "of the eight simulations from the benchmark start, same launch mode"}
    probs, E = make_problems(pff, sp, rank, prec, VARIANTS)
    nprob = len(probs)
    budget = sum(pff.problem_bytes(N, N, prec) for _ in probs)
    b = pff.create_batch(nprob, budget, sp)
    # each simulation on its own stream and host thread: the variants converge at
    # different iteration counts, and independent progress beats lock-step launches
    pff.batch_set_group_size(b, GROUP_SIZE)
    for p in probs:
        assert pff.batch_admit(b, p.h) is not None
    if args.warmup:
        pff.batch_step(b, nprob, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    l0 = pff.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    reps = [[] for _ in range(nprob)]
    for s in range(args.steps):
        out = pff.batch_step(b, nprob, 1)
        for i in range(nprob):
            reps[i].extend(out[i])
        evs[s + 1].record(stream)
    torch.cuda.synchronize()
    launches = pff.kernel_launches() - l0
    clk = clocks.stop()
    step_ms = [evs[s].elapsed_time(evs[s + 1]) for s in range(args.steps)]
    # fields after warm-up + timed steps, for the equal-accuracy comparison with the FP64 path
    phi_mixed = [p.get_fields(pff.FIELD_PHI) for p in probs] if rank == 0 and not args.no_baselines else None
    # kernel-class durations: CUDA events around every launch, on the batch stream,
    # over further load steps of the same run (event brackets need direct launches)
    ki = max(1, min(args.steps, 3))
    pff.batch_set_group_size(b, 0)        # one stream: the event brackets of different kernels do not overlap
    pff.timing_reset()
    pff.timing_enable(True)
    reps_k = [[] for _ in range(nprob)]
    out = pff.batch_step(b, nprob, ki)
    for i in range(nprob):
        reps_k[i].extend(out[i])
    pff.timing_enable(False)
    pff.batch_set_group_size(b, GROUP_SIZE)
    elapsed = sum(step_ms) / 1e3
    mech = sum(r["mech_cg_iters"] for rr in reps for r in rr)
    bccg = sum(r["bccg_iters"] for rr in reps for r in rr)
    nsteps_done = sum(len(rr) for rr in reps)
    # kernel-class timing (live, CUDA events on the batch stream)
    bccg4 = pff.get_kernel_variant(pff.VARIANT_BCCG_PASSES, N, 1) == 1
    kt = {k: pff.timing_read(*k) for k in KERNEL_NAMES}
    kb = kernel_bytes(reps_k, [v[1] == "ISOTROPIC" for v in VARIANTS], es, N, N, bccg4)
    kernels = {}
    for k, name in KERNEL_NAMES.items():
        ms, nl = kt[k]
        byts = kb[k]
        kernels[name] = {"ms": round(ms, 3), "launches": nl, "share": None,
                         "achieved_GBs": (byts / (ms / 1e3) / 1e9) if ms > 0 else None,
                         "alg_bytes_per_launch": byts / nl if nl else None}
    tot_ms = sum(v["ms"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = round(v["ms"] / tot_ms, 4) if tot_ms > 0 else None
    dom = max(kernels, key=lambda n: kernels[n]["ms"])
    # the whole path in the timed launch mode: algorithmic bytes of every kernel class over the
    # timed region (iteration counts of its own reports) per unit of its wall time
    timed_bytes = sum(kernel_bytes(reps, [v[1] == "ISOTROPIC" for v in VARIANTS], es, N, N, bccg4).values())
    # distributed aggregation: max time, summed work (no data-path collective)
    elapsed_max, (mech_all, bccg_all, steps_all) = aggregate(elapsed, [mech, bccg, nsteps_done], world,
                                                             f"cuda:{dev}")
    value = (mech_all + bccg_all) * N * N / elapsed_max
    line = None
    extra = {}
    if rank == 0 and not args.no_baselines and not FP64_RUN:
        dom_key = {name: k for k, name in KERNEL_NAMES.items()}[dom]
        extra = baselines(args, pff, torch, stream, sp, probs, b, E, mech, bccg, elapsed, phi_mixed, dom_key)
    for p in probs:
        pass
    pff.destroy_batch(b)
    if rank == 0:
        peak, peak_kind = hbm_peak()
        ach = kernels[dom]["achieved_GBs"]
        ws = sum(pff.problem_bytes(N, N, prec) for _ in probs)
        line = {
            "metric": "pixel_cg_iters_per_s", "value": value, "unit": "pixel-CG-iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if FP64_RUN else "f32",
            "data": "synthetic",
            "config": workload_config(world),
            "kernel_autotune": shape,
            "iteration_mix": {"mechanics_cg": mech, "bccg": bccg,
                              "mechanics_fraction": mech / (mech + bccg) if mech + bccg else None},
            "load_steps_per_s": steps_all / elapsed_max,
            "mech_pixel_cg_iters_per_s": mech_all * N * N / elapsed_max,
            "bccg_pixel_iters_per_s": bccg_all * N * N / elapsed_max,
            "bccg_clamp_fraction": (sum(r["bccg_clamp_iters"] for rr in reps for r in rr) / bccg) if bccg else None,
            "bccg_explicit_fraction": (sum(r["bccg_full_iters"] for rr in reps for r in rr) / bccg) if bccg else None,
            "step_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": (ach / peak) if ach else None, "peak_kind": peak_kind,
                         "frac_of_nominal": (ach / NOMINAL_HBM_GBS) if ach else None,
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "traffic": (None if FP64_RUN else   # the committed capture is of the FP32 kernels
                                     measured_traffic(dom, kernels.get(dom, {}).get("alg_bytes_per_launch"))),
                         "traffic_unit": "bytes per launch (ncu DRAM read + write, scaled to this run's average launch)",
                         "timed_region": {"achieved": timed_bytes / elapsed / 1e9, "frac": timed_bytes / elapsed / 1e9 / peak,
                                          "unit": "GB/s", "what": "algorithmic bytes of all kernel classes over the "
                                                                  "timed load steps / their wall time (headline launch "
                                                                  "mode: concurrent streams, CUDA graphs)"}},
            "kernels": kernels,
            "kernel_timing": f"CUDA events around each launch, over {ki} further load steps of the run with all "
                             f"eight simulations in one launch group on one stream (direct launches queued behind "
                             f"a short delay kernel; the timed region replays CUDA graphs on per-simulation streams)",
            "clocks": clk,
        }
        line.update(extra)
    return line


def plain_fp64(args, pff, torch, stream, sp, tol, phi_mixed):
    """The plain per-simulation FP64 GPU path on the benchmark's eight variants: one simulation at a
    time, unbatched, from the same start with the same warm-up and timed step counts as the mixed
    region; CUDA events on the stream around each simulation's timed steps.  Returns throughput and
    each variant's final phase field's relative L2 difference from the mixed path's."""
    f_iters, f_steps, f_time, diffs, finals = 0, 0, 0.0, [], []
    for j, v in enumerate(VARIANTS):
        [p64], _ = make_problems(pff, sp, 0, pff.FP64, [v])
        p64.set_params(mech_tol=tol, pf_tol=tol)
        if args.warmup:
            p64.step_load(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = p64.step_load(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        f_time += e0.elapsed_time(e1) / 1e3
        f_iters += sum(r["mech_cg_iters"] + r["bccg_iters"] for r in reps)
        f_steps += len(reps)
        phi = p64.get_fields(pff.FIELD_PHI)
        finals.append(phi)
        if phi_mixed is not None:
            ref = max(np.linalg.norm(phi), 1e-30)
            diffs.append(float(np.linalg.norm(phi_mixed[j] - phi) / ref))
        p64.close()
    return {"pixel_cg_iters_per_s": f_iters * N * N / f_time, "load_steps_per_s": f_steps / f_time,
            "mech_tol": tol, "pf_tol": tol, "steps_timed": f_steps,
            "phi_rel_l2_vs_mixed_max": max(diffs) if diffs else None}, finals


def baselines(args, pff, torch, stream, sp, probs, b, E, mech, bccg, elapsed, phi_mixed=None, dom_key=(0, 1)):
    out = {}
    ours_steps = len(probs) * args.steps / elapsed
    ours_iters = (mech + bccg) * N * N / elapsed
    # plain per-simulation FP64 GPU path, all eight variants, same start / warm-up / steps:
    # at the loosest tolerance that meets the 1e-5 bar (the equal-accuracy comparison) and at
    # the workload's nominal 1e-8
    eq, fin_eq = plain_fp64(args, pff, torch, stream, sp, EQUAL_ACCURACY_TOL, phi_mixed)
    nom, fin_nom = plain_fp64(args, pff, torch, stream, sp, TOL, phi_mixed)
    eq["phi_rel_l2_vs_fp64_tol1e-8_max"] = max(float(np.linalg.norm(a - c) / max(np.linalg.norm(c), 1e-30))
                                               for a, c in zip(fin_eq, fin_nom))
    out["plain_fp64_gpu"] = {
        "equal_accuracy": eq, "nominal_tol": nom,
        "sample": f"the eight variants one at a time, unbatched, from eps_bar_yy = {PRELOAD} eps_M, {args.warmup} "
                  f"warm-up and {args.steps} timed load steps each (the mixed region's counts); equal accuracy: "
                  f"sub-solver tolerances {EQUAL_ACCURACY_TOL:g}, the loosest at which the FP64 path meets the 1e-5 "
                  f"relative-L2 bar against the oracle on the 64x64 workload's checkpoints, as the mixed path does"}
    out["vs_plain_fp64_gpu"] = {"load_steps_per_s": ours_steps / eq["load_steps_per_s"],
                                "pixel_cg_iters_per_s": ours_iters / eq["pixel_cg_iters_per_s"],
                                "basis": "equal accuracy (FP64 at tolerance 1e-6)",
                                "load_steps_per_s_vs_nominal_tol": ours_steps / nom["load_steps_per_s"]}
    # the FFT kernels alone against cuFFT (timed comparator only)
    try:
        out["cufft_comparison"] = cufft_compare(pff, torch, stream)
    except Exception as e:
        out["cufft_comparison"] = {"error": str(e)[:200]}
    # the dominant kernel class at 1, 2, 4 and 8 identical simulations per launch
    try:
        out["dominant_kernel_scaling"] = kernel_scaling(pff, torch, sp, key=dom_key)
    except Exception as e:
        out["dominant_kernel_scaling"] = {"error": str(e)[:200]}
    # the two BCCG iteration structures (three / four operator passes), same start, same launches
    try:
        out["bccg_passes_compare"] = bccg_passes_compare(pff, torch, sp)
    except Exception as e:
        out["bccg_passes_compare"] = {"error": str(e)[:200]}
    # the opt-in Fourier-Helmholtz preconditioned BCCG against Algorithm 1, both from the
    # same start of the same eight variants, batched the way the timed region is
    try:
        out["preconditioned_bccg"] = precond_compare(pff, torch, sp)
    except Exception as e:
        out["preconditioned_bccg"] = {"error": str(e)[:200]}
    # end to end through the public API with host buffers
    ke = max(1, min(args.steps, 5))
    # pinned host buffers (page-locked, as a serving front end would hold them): the modulus
    # field each simulation uploads and the phase field each one reads back, every step
    pin_t = [torch.empty(N * N, dtype=torch.float64, pin_memory=True) for _ in range(len(probs) + 1)]
    E_pin = pin_t[0].numpy()
    E_pin[:] = np.asarray(E, dtype=np.float64).ravel()
    phi_pin = [t.numpy() for t in pin_t[1:]]
    # the simulations' transfers run from one host thread each, as a front end serving them would
    # issue them (handles are independent; ctypes releases the GIL during each call)
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max_workers=len(probs))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_e = 0
    for s in range(ke):
        list(pool.map(lambda p: p.set_modulus_field(E_pin), probs))
        out_s = pff.batch_step(b, len(probs), 1)
        it_e += sum(r["mech_cg_iters"] + r["bccg_iters"] for rr in out_s for r in rr)
        list(pool.map(lambda a: a[0].get_fields(pff.FIELD_PHI, out=a[1]), zip(probs, phi_pin)))
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    pool.shutdown()
    out["e2e"] = {"value": it_e * N * N / te, "unit": "pixel-CG-iters/s",
                  "h2d_bytes_per_step": len(probs) * N * N * 8, "d2h_bytes_per_step": len(probs) * N * N * 8,
                  "steps": ke, "host_buffers": "pinned (torch pin_memory), FP64; one host thread per simulation",
                  "path": "pff_set_modulus_field (host E) + pff_batch_step + pff_get_fields(PHI)"}
    # the other workloads: 64x64 whole run, one 2048x2048 grid, a batch of 64 256x256 grids
    for key, fn in (("grid64_whole_run", grid64_whole_run), ("grid2048", grid2048),
                    ("batch64_grid256", batch64_grid256)):
        try:
            out[key] = fn(pff, torch, stream, sp)
        except Exception as e:
            out[key] = {"error": str(e)[:300]}
    # continuous-batching serving: seeded Poisson arrivals of whole simulations
    try:
        out["serving"] = serving_run(pff, sp)
    except Exception as e:
        out["serving"] = {"error": str(e)[:200]}
    # FP64 oracle on the host cores, same iteration mix as the timed region
    try:
        tm, tb, tot = run_cpu_sample_subprocess(8, 80)
        cpu_time = mech * tm + bccg * tb
        out["cpu_baseline"] = {"value": (mech + bccg) * N * N / cpu_time, "unit": "pixel-CG-iters/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"oracle timed for 8 mechanics CG + 80 BCCG iterations on one {N}x{N} grid "
                                         f"({tot:.1f} s; {tm:.3f} s and {tb:.4f} s per iteration), weighted by the "
                                         f"timed region's mix of {mech} mechanics CG and {bccg} BCCG iterations"}
    except Exception as e:  # the baseline is reported, never required
        out["cpu_baseline"] = {"value": None, "unit": "pixel-CG-iters/s", "cores": 1, "kind": "oracle",
                               "sample": f"failed: {e}"}
    try:
        tm_p, tb_p, procs, wall = run_cpu_sample_all_cores(4, 40)
        out["cpu_baseline"]["all_cores"] = {
            "value": procs * (mech + bccg) * N * N / (mech * tm_p + bccg * tb_p), "unit": "pixel-CG-iters/s",
            "cores": procs,
            "sample": f"{procs} single-threaded oracle processes, each 4 mechanics CG + 40 BCCG iterations on its "
                      f"own {N}x{N} grid, started together ({wall:.1f} s wall; {tm_p:.3f} s and {tb_p:.4f} s per "
                      f"iteration under that contention), weighted by the timed region's iteration mix"}
    except Exception as e:
        out["cpu_baseline"]["all_cores"] = {"value": None, "sample": f"failed: {str(e)[:200]}"}
    return out


def kernel_table(pff, reps_per_problem, nx, ny, iso=False):
    """Per kernel class: time (CUDA events around each launch), launches, algorithmic GB/s."""
    bccg4 = pff.get_kernel_variant(pff.VARIANT_BCCG_PASSES, nx, 1) == 1
    kb = kernel_bytes(reps_per_problem, [iso] * len(reps_per_problem), 4, nx, ny, bccg4)
    out = {}
    for k, name in KERNEL_NAMES.items():
        ms, nl = pff.timing_read(*k)
        byts = kb[k]
        out[name] = {"ms": round(ms, 3), "launches": nl,
                     "achieved_GBs": (byts / (ms / 1e3) / 1e9) if ms > 0 else None}
    return out


def roofline_of(kernels):
    peak, kind = hbm_peak()
    dom = max(kernels, key=lambda n: kernels[n]["ms"])
    ach = kernels[dom]["achieved_GBs"]
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if ach else None, "peak_kind": kind}


def grid64_whole_run(pff, torch, stream, sp, oracle_steps=12):
    """The 64x64 workload (AT1, strain-spectral, crack set, ell = 2 px, correlation length 8 px,
    seed 0, Delta eps_bar_yy = eps_M/20, tolerances 1e-8) run to C-bar < C_broken on the GPU in
    FP64 and in mixed precision (CUDA events around the whole run), the crack set compared with
    the stored oracle run, and the FP64 oracle timed on the host for a bounded sample of load
    steps (the first steps and the steps after the stored mid-run checkpoint), its whole-run
    time estimated from the GPU run's iteration count at the sampled rate."""
    from oracle import evolution as ev
    from oracle.params import AT1, CRACK_SET, SPECTRAL, Params
    from paper_2203_16467_gb300.inputs import eps_M, modulus_field
    n, lc, ell = 64, 8.0, 2.0
    em = eps_M(1.0, NU, 1.0, ell)
    E = modulus_field(n, n, lc, 0)
    gold = np.load(os.path.join(ROOT, "tests", "golden", "grid64_run.npz"))
    res = {"workload": "grid64_lc8_ell2_AT1_spectral_crackset_whole_run", "tol": 1e-8}
    for name, prec in (("fp64", pff.FP64), ("mixed", pff.MIXED)):
        p = pff.Problem(n, n, prec, stream=sp, E=E, model=("AT1", "SPECTRAL", "CRACK_SET"),
                        params=dict(nu=NU, ell=ell, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 20, 0.0)))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = p.step_load(5000)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        phi = p.get_fields(pff.FIELD_PHI)
        p.close()
        it = sum(r["mech_cg_iters"] + r["bccg_iters"] for r in reps)
        a, g = phi > 0.95, gold["phi_final"] > 0.95
        res[name] = {"load_steps": len(reps), "seconds": t, "load_steps_per_s": len(reps) / t,
                     "pixel_cg_iters_per_s": it * n * n / t, "iterations": it, "broken": bool(reps[-1]["broken"]),
                     "cracked_px": int(a.sum()), "iou_vs_oracle_run": float((a & g).sum() / max(1, (a | g).sum()))}
    # oracle sample on one host core
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=CRACK_SET, ell=ell, nu=NU,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 20)), mech_tol=1e-8, pf_tol=1e-8)
    t_or, it_or = 0.0, 0
    starts = [ev.State.initial(E)]
    mid = ev.State.initial(E)
    mid.phi, mid.eps_star, mid.eps_bar = gold["phi_700"].copy(), gold["eps_star_700"].copy(), gold["eps_bar_700"].copy()
    mid.flag = bool(gold["flag_700"])
    starts.append(mid)
    for st in starts:
        t0 = time.perf_counter()
        for _ in range(oracle_steps):
            r = ev.load_step(st, par)
            it_or += r["mech_cg"] + r["bccg"]
        t_or += time.perf_counter() - t0
    rate = it_or * n * n / t_or
    res["oracle"] = {"cores": 1, "pixel_cg_iters_per_s": rate,
                     "whole_run_seconds_estimated": res["fp64"]["iterations"] * n * n / rate,
                     "sample": f"{oracle_steps} load steps from the start and {oracle_steps} from the stored step-700 "
                               f"state ({t_or:.1f} s, {it_or} iterations); the whole-run time is the FP64 GPU run's "
                               f"iteration count at this rate (extrapolated)"}
    res["speedup_vs_oracle_whole_run"] = {k: res["oracle"]["whole_run_seconds_estimated"] / res[k]["seconds"]
                                          for k in ("fp64", "mixed")}
    return res


def grid2048(pff, torch, stream, sp, warm=2, steps=8):
    """One 2048x2048 grid, correlation length 64 px, ell = 2 px, AT2 strain-spectral, crack set,
    mixed precision, from 0.97 eps_M: load steps timed with CUDA events, then one more load step
    with per-kernel event timing for the roofline of its dominant kernel class."""
    from paper_2203_16467_gb300.inputs import eps_M, modulus_field
    n, lc, ell = 2048, 64.0, 2.0
    em = eps_M(1.0, NU, 1.0, ell)
    E = modulus_field(n, n, lc, 0)
    p = pff.Problem(n, n, pff.MIXED, stream=sp, E=E, model=("AT2", "SPECTRAL", "CRACK_SET"),
                    params=dict(nu=NU, ell=ell, mech_tol=TOL, pf_tol=TOL, d_eps_bar=(0.0, em / 20, 0.0)))
    p.set_strain(None, (0.0, 0.97 * em, 0.0))
    p.step_load(warm)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = p.step_load(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    it = sum(r["mech_cg_iters"] + r["bccg_iters"] for r in reps)
    pff.timing_reset()
    pff.timing_enable(True)
    rk = p.step_load(1)
    pff.timing_enable(False)
    kern = kernel_table(pff, [rk], n, n)
    p.close()
    return {"workload": "grid2048_lc64_ell2_AT2_spectral_crackset_mixed", "load_steps": len(reps),
            "ms_per_load_step": 1e3 * t / len(reps), "load_steps_per_s": len(reps) / t,
            "pixel_cg_iters_per_s": it * n * n / t, "mech_cg_iters": sum(r["mech_cg_iters"] for r in reps),
            "bccg_iters": sum(r["bccg_iters"] for r in reps), "roofline": roofline_of(kern), "kernels": kern,
            "sample": f"{warm} warm-up and {steps} timed load steps from eps_bar_yy = 0.97 eps_M (labelled sample of "
                      f"the 300-step run); kernel classes timed over one further load step"}


def batch64_grid256(pff, torch, stream, sp, warm=2, steps=8):
    """64 independent 256x256 microstructures (seeds 0..63, correlation length 16 px, ell = 2 px,
    AT1 strain-spectral, crack set, mixed precision) advanced together from 0.95 eps_M, launch
    grouping chosen by pff_batch_autotune; load steps timed with CUDA events; kernel classes timed
    over one further load step in one launch group."""
    from paper_2203_16467_gb300.inputs import eps_M, modulus_field
    n, lc, ell, ns = 256, 16.0, 2.0, 64
    em = eps_M(1.0, NU, 1.0, ell)
    probs = []
    for seed in range(ns):
        p = pff.Problem(n, n, pff.MIXED, stream=sp, E=modulus_field(n, n, lc, seed),
                        model=("AT1", "SPECTRAL", "CRACK_SET"),
                        params=dict(nu=NU, ell=ell, mech_tol=TOL, pf_tol=TOL, d_eps_bar=(0.0, em / 20, 0.0)))
        p.set_strain(None, (0.0, PRELOAD * em, 0.0))
        probs.append(p)
    b = pff.create_batch(ns, sum(pff.problem_bytes(n, n, pff.MIXED) for _ in probs), sp)
    for p in probs:
        assert pff.batch_admit(b, p.h) is not None
    chosen = pff.batch_autotune(b, ns, group_sizes=(1, 8, 64), steps_each=1)[0]
    pff.batch_step(b, ns, warm)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = pff.batch_step(b, ns, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    rr = [r for o in out for r in o]
    it = sum(r["mech_cg_iters"] + r["bccg_iters"] for r in rr)
    pff.batch_set_group_size(b, 0)
    pff.timing_reset()
    pff.timing_enable(True)
    ok = pff.batch_step(b, ns, 1)
    pff.timing_enable(False)
    kern = kernel_table(pff, ok, n, n)
    pff.destroy_batch(b)
    for p in probs:
        p.close()
    return {"workload": "batch64_grid256_lc16_ell2_AT1_spectral_crackset_mixed", "simulations": ns,
            "group_size": chosen, "load_steps": len(rr), "ms_per_batch_step": 1e3 * t / steps,
            "load_steps_per_s": len(rr) / t, "pixel_cg_iters_per_s": it * n * n / t,
            "roofline": roofline_of(kern), "kernels": kern,
            "sample": f"autotune over group sizes (1, 8, 64), {warm} warm-up and {steps} timed batch steps from "
                      f"eps_bar_yy = {PRELOAD} eps_M; kernel classes timed over one further step in one launch group"}


def cufft_compare(pff, torch, stream, n=N, reps=200, warm=20):
    """Laplacian of one n x n field through a real 2-D FFT round trip: this library's three
    kernels (allocation-free C-ABI entries, FP32 and FP64) against torch.fft (cuFFT) with the
    same multiplier -|2 pi q|^2, device-resident, CUDA events around reps calls on one stream."""
    import ctypes
    res = {"transform": f"real 2-D FFT, multiplier -|2 pi q|^2, inverse; {n}x{n}, one field",
           "cufft": "torch.fft.rfft2 -> multiply -> torch.fft.irfft2 (cuFFT)", "reps": reps}
    g = torch.Generator(device="cuda").manual_seed(7)
    ky = torch.fft.fftfreq(n, d=1.0, device="cuda", dtype=torch.float64) * 2 * np.pi
    kx = torch.fft.rfftfreq(n, d=1.0, device="cuda", dtype=torch.float64) * 2 * np.pi
    mult64 = -(ky[:, None] ** 2 + kx[None, :] ** 2)
    msg = ctypes.c_char_p()
    for name, dt, fn in (("f32", torch.float32, pff.lib.pff_apply_laplacian_noalloc_f32),
                         ("f64", torch.float64, pff.lib.pff_apply_laplacian_noalloc)):
        x = torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64).to(dt)
        y = torch.empty_like(x)
        mult = mult64.to(dt)
        sp = ctypes.c_void_p(stream.cuda_stream)

        def ours():
            rc = fn(n, n, 1.0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), sp, ctypes.byref(msg))
            if rc:
                raise RuntimeError(f"noalloc rc {rc}: {msg.value}")

        def theirs():
            return torch.fft.irfft2(torch.fft.rfft2(x) * mult, s=(n, n))

        times = {}
        with torch.cuda.stream(stream):
            for tag, f in (("ours", ours), ("cufft", theirs)):
                for _ in range(warm):
                    f()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    f()
                e1.record(stream)
                torch.cuda.synchronize()
                times[tag] = 1e3 * e0.elapsed_time(e1) / reps
            ours()
            ref = theirs()
        torch.cuda.synchronize()
        err = float((y.double() - ref.double()).abs().max() / ref.double().abs().max())
        res[name] = {"ours_us": times["ours"], "cufft_us": times["cufft"], "speedup": times["cufft"] / times["ours"],
                     "max_rel_diff": err}
    return res


def kernel_scaling(pff, torch, sp, key=(0, 1), variant=("AT1", "SPECTRAL", "CRACK_SET")):
    """Average launch duration (CUDA events) and algorithmic GB/s of the kernel classes when
    every launch carries k identical simulations (all active in every launch), k = 1..8:
    separates the fixed cost of a launch from the bandwidth of its work.  `rows` are those of
    class key; `classes` holds the same figures for every class of the iteration."""
    peak, _ = hbm_peak()
    bccg4 = pff.get_kernel_variant(pff.VARIANT_BCCG_PASSES, N, 1) == 1
    bpp = bytes_per_px(4, N, variant[1] == "ISOTROPIC")
    per = {k: [] for k in KERNEL_NAMES}
    for k in (1, 2, 4, 8):
        probs, _ = make_problems(pff, sp, 0, pff.MIXED, [variant] * k)
        b = pff.create_batch(k, sum(pff.problem_bytes(N, N, pff.MIXED) for _ in probs), sp)
        pff.batch_set_group_size(b, 0)
        for p in probs:
            assert pff.batch_admit(b, p.h) is not None
        pff.batch_step(b, k, 2)
        torch.cuda.synchronize()
        pff.timing_reset()
        pff.timing_enable(True)
        out = pff.batch_step(b, k, 1)
        pff.timing_enable(False)
        act_all = active_launches(out, bccg4)   # problem-launches that did work
        for kk in KERNEL_NAMES:
            ms, nl = pff.timing_read(*kk)
            if not nl:
                continue
            act = act_all[kk]
            gbs = act * bpp[kk] * N * N / (ms * 1e-3) / 1e9 if ms > 0 else None
            per[kk].append({"simulations_per_launch": k, "launches": nl, "working_launches": act // k,
                            "us_per_launch": 1e3 * ms / nl, "achieved_GBs": gbs, "frac": gbs / peak if gbs else None})
        pff.destroy_batch(b)
        for p in probs:
            p.close()
    return {"kernel": KERNEL_NAMES[key], "variant": "/".join(variant), "rows": per[key],
            "classes": {KERNEL_NAMES[kk]: {str(r["simulations_per_launch"]): round(r["frac"], 3) if r["frac"] else None
                                           for r in v} for kk, v in per.items() if v},
            "note": "one load step after two warm-up steps; the identical simulations work in the same "
                    "launches; the skipped launches at the end of each 12-iteration chunk count against "
                    "the time, as in the roofline figure; classes: fraction of the measured peak per class "
                    "and simulations per launch"}


def bccg_passes_compare(pff, torch, sp, warm=3, steps=8):
    """The eight variants from the benchmark start under each BCCG iteration structure (three
    passes with alpha from the column pass, or four with alpha from p.Jp), batched as the timed
    region is, CUDA events on the stream around the timed batch steps."""
    res = {}
    keep = pff.get_kernel_variant(pff.VARIANT_BCCG_PASSES, 0, 1)
    try:
        for v in (0, 1):
            pff.set_kernel_variant(pff.VARIANT_BCCG_PASSES, 0, 1, v)
            probs, _ = make_problems(pff, sp, 0, pff.MIXED, VARIANTS)
            b = pff.create_batch(len(probs), sum(pff.problem_bytes(N, N, pff.MIXED) for _ in probs), sp)
            pff.batch_set_group_size(b, GROUP_SIZE)
            for p in probs:
                assert pff.batch_admit(b, p.h) is not None
            pff.batch_step(b, len(probs), warm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = pff.batch_step(b, len(probs), steps)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            rr = [r for o in out for r in o]
            it = sum(r["mech_cg_iters"] + r["bccg_iters"] for r in rr)
            res["three_passes" if v == 0 else "four_passes"] = {
                "ms_per_batch_step": 1e3 * dt / steps, "pixel_cg_iters_per_s": it * N * N / dt,
                "bccg_iters": sum(r["bccg_iters"] for r in rr), "mech_cg_iters": sum(r["mech_cg_iters"] for r in rr)}
            pff.destroy_batch(b)
            for p in probs:
                p.close()
    finally:
        pff.set_kernel_variant(pff.VARIANT_BCCG_PASSES, 0, 1, keep)
    res["speedup_three_over_four"] = (res["four_passes"]["ms_per_batch_step"] / res["three_passes"]["ms_per_batch_step"])
    res["sample"] = (f"the eight variants from eps_bar_yy = {PRELOAD} eps_M, {warm} warm-up and {steps} timed batch "
                     f"steps each, host wall clock around synchronised batch steps")
    return res


def precond_compare(pff, torch, sp, warm=2, steps=6):
    res = {}
    for pre in (0, 1):
        probs, _ = make_problems(pff, sp, 0, pff.MIXED, VARIANTS)
        for p in probs:
            p.set_params(pf_precondition=pre)
        b = pff.create_batch(len(probs), sum(pff.problem_bytes(N, N, pff.MIXED) for _ in probs), sp)
        pff.batch_set_group_size(b, GROUP_SIZE)
        for p in probs:
            assert pff.batch_admit(b, p.h) is not None
        pff.batch_step(b, len(probs), warm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = pff.batch_step(b, len(probs), steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rr = [r for o in out for r in o]
        res[pre] = {"load_steps_per_s": len(rr) / dt, "bccg_iters": sum(r["bccg_iters"] for r in rr),
                    "mech_cg_iters": sum(r["mech_cg_iters"] for r in rr)}
        pff.destroy_batch(b)
        for p in probs:
            p.close()
    return {"algorithm1": res[0], "preconditioned": res[1],
            "load_steps_speedup": res[1]["load_steps_per_s"] / res[0]["load_steps_per_s"],
            "sample": f"the eight variants from the benchmark start, {warm} warm-up and {steps} timed load steps "
                      f"each, host wall clock around synchronised batch steps"}


def serving_run(pff, stream, n_requests=100, rate=40.0, max_steps=10):
    """Poisson arrivals of simulations with grid sizes uniform over {128^2, 256^2, 512^2,
    1024^2} and variants uniform over {AT1, AT2} x {isotropic, spectral}, E recipe of the
    64^2 workload (correlation length 8 px, ell = 2 px), mixed precision, preloaded to
    0.97 eps_M, each run for max_steps load steps (or until broken); admission by HBM budget;
    one lane (batch, stream, worker thread) per grid size."""
    from paper_2203_16467_gb300 import serving
    reqs = serving.poisson_requests(n_requests, rate, seed=1234, max_steps=max_steps, preload=0.97, lc=8.0, ell=2.0)
    server = serving.Server(hbm_budget=16 << 30, max_slots=64)
    for r in reqs:
        server.submit(r)
    st = server.run()
    server.close()
    ms = (lambda d: {k: (1e3 * v if v is not None else None) for k, v in d.items()})
    return {"requests": n_requests, "arrival_rate_per_s": rate, "steps_per_request": max_steps,
            "load_steps_per_s": st["load_steps_per_s"], "step_latency_ms": ms(st["step_latency_s"]),
            "start_latency_ms": ms(st["start_latency_s"]), "simulation_latency_s": st["sim_latency_s"],
            "per_size": {k: {"requests": v["requests"], "step_latency_ms": ms(v["step_latency_s"]),
                             "start_latency_ms": ms(v["start_latency_s"]),
                             "simulation_latency_s": v["sim_latency_s"]} for k, v in st["per_size"].items()},
            "completed": st["completed"], "peak_active": st["peak_active"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-baselines", action="store_true", help="skip the FP64 / e2e / CPU extras")
    ap.add_argument("--no-tune", action="store_true", help="keep the default kernel variants (no autotuning)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed",
                    help="fields in FP32 with FP64 reductions (the headline), or the same workload all in FP64")
    ap.add_argument("--group-size", type=int, default=None,
                    help="simulations per launch group (default 1: one stream per simulation; 0: all in one group)")
    args = ap.parse_args()
    global GROUP_SIZE, FP64_RUN
    if args.group_size is not None:
        GROUP_SIZE = args.group_size
    FP64_RUN = args.precision == "fp64"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
        if line:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local)
    if line:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
