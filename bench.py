#!/usr/bin/env python3
"""OC iterations per second of the SIMP + OC hot path on a 480x160x80 cantilever.

One step = one OC iteration of the whole path (SIMP moduli, preconditioner
set-up, equilibrium solve to ||f - K u|| <= 1e-8 ||f||, element energies and
sensitivities, rmin filter, OC bisection update) on the synthetic cantilever
480x160x80 (load at the centre of the x = nelx face, volfrac 0.2, rmin 2.5).

The chosen form: BF16 tensor-core operator with FP32 inner CG and FP64
defect correction, preconditioned by the learned multigrid V-cycle (its
parameters learned first on a 96x32x16 cantilever of the same family).
Beside it, on the same three designs of the timed window (its start, middle
and end, each with the displacement the run had there): plain FP64
Jacobi-PCG, the learned-FCG form (FP64 flexible CG with the learned
multigrid) and the Jacobi-preconditioned defect correction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--precond lmg|jacobi]
  python bench.py --impl reference ...    (the CPU FP64 oracle, bounded sample)

Prints one JSON line (rank 0).  N > 1 (torchrun): independent replicas, one
per GPU, with the max time over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "OC iters/s at 480x160x80, chosen vs plain FP64 Jacobi-PCG at rel.res 1e-8"
UNIT = "OC iters/s"
PREC_NAMES = {0: "fp64", 1: "bf16-dc", 2: "bf16x2-dc", 3: "fp16-dc", 4: "fp16x2-dc"}
# the arithmetic type of the tensor-core operand (the dominant kernel) and the
# whole form in words
DTYPES = {0: "f64", 1: "bf16", 2: "bf16", 3: "f16", 4: "f16"}
ARITHMETIC = {
    0: "f64 Jacobi-PCG, f64 matvec",
    1: "bf16 operand x integer-exact bf16 stiffness, f32 accumulate, f32 inner CG, "
       "f64 residual / dots / u (defect correction)",
    2: "bf16 hi+lo operand, f32 accumulate, f32 inner CG, f64 defect correction",
    3: "scaled f16 operand, f32 accumulate, f32 inner CG, f64 defect correction",
    4: "scaled f16 hi+lo operand, f32 accumulate, f32 inner CG, f64 defect correction"}
# FP64 Jacobi-PCG iterations per OC iteration, used to turn the oracle's
# measured per-iteration cost into OC iterations/s when no GPU run in the
# same process supplies the count (reference arm): the library's FP64 form
# at 480x160x80 needs 5116 iterations from the design after OC iteration 5
# and 6321 from the one after iteration 10; about 5700 over iterations 4-11.
REF_ITERS_PER_OC = 5700
# the learned multigrid parameters are learned on this cantilever of the
# bench's family (centre load, volfrac 0.2, rmin 2.5) after a few OC iterations
TRAIN_GRID = (96, 32, 16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=1,
                    help="0 fp64, 1 bf16, 2 bf16 hi+lo, 3 fp16, 4 fp16 hi+lo (tensor-core forms "
                         "with FP64 defect correction)")
    ap.add_argument("--size", default="480x160x80")
    ap.add_argument("--workload", default="large",
                    choices=["large", "batched64", "paper32", "config1", "config2"],
                    help="large: the 480x160x80 cantilever; batched64: 64 seeded uneven "
                         "cantilevers stepped together (extra measurement)")
    ap.add_argument("--precond", default="lmg", choices=["lmg", "jacobi"],
                    help="lmg: learned multigrid (the chosen form); jacobi: Jacobi-PCG")
    ap.add_argument("--inner-rtol", type=float, default=None,
                    help="residual-replacement factor of the defect-correction forms "
                         "(default 0.01 with the multigrid, 0.3 with Jacobi)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the comparison forms")
    ap.add_argument("--fp64-cuda-cores", action="store_true",
                    help="FP64 K p of the chosen and learned forms on the CUDA cores instead of "
                         "the sliced tensor-core kernel")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--unet", action="store_true",
                    help="also time one OC iteration of the U-Net flexible-CG form (network "
                         "trained first on a 96x32x16 cantilever; several minutes)")
    ap.add_argument("--export", default=None,
                    help="paper32: directory for the usage example's voxel dump and STL")
    ap.add_argument("--cpu-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-its", type=float, default=REF_ITERS_PER_OC, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-reps", type=int, default=20, help=argparse.SUPPRESS)
    a = ap.parse_args()
    if a.inner_rtol is None:
        a.inner_rtol = 0.05 if a.precond == "lmg" else 0.3
    return a


def dims(args):
    a, b, c = (int(v) for v in args.size.split("x"))
    return a, b, c


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg
def cpu_leg(args):
    """Time the oracle's assembled-CSR FP64 Jacobi-PCG and element steps (C,
    OpenMP, all host cores) on a slab of the workload and extrapolate to OC
    iterations/s at the full grid (prints one JSON dict)."""
    import numpy as np
    from oracle import csr, fem
    from synth import problems

    nelx, nely, nelz = dims(args)
    KE = fem.element_stiffness(0.3)
    zs = max(1, nelz // 8)                  # an eighth-depth slab of the grid
    sp = problems.config_large(nelx=nelx, nely=nely, nelz=zs)
    x = sp.initial_density()
    E = fem.simp_modulus(x, sp.penal)
    f = fem.masked_load(sp.load, sp.fixed)
    t0 = time.perf_counter()
    op = csr.Operator(nelx, nely, zs, E, KE, sp.fixed)
    t_asm = (time.perf_counter() - t0) * (nelz / zs)
    # PCG iterations: reps iterations minus one, so the set-up cancels
    reps = max(args.cpu_reps, 2)
    t = []
    for m in (1, reps + 1):
        t0 = time.perf_counter()
        op.pcg(f, rtol=0.0, maxit=m)
        t.append(time.perf_counter() - t0)
    t_it = max(t[1] - t[0], 1e-9) / reps * (nelz / zs)
    op.close()
    u = problems.random_vector(sp.ndof, 1, 1e-3)
    t0 = time.perf_counter()
    c, ce, dc = csr.element_steps(nelx, nely, zs, KE, u, x, sp.penal)
    dcf = csr.sensitivity_filter(nelx, nely, zs, sp.rmin, x, dc)
    csr.oc_update(x, dcf, sp.volfrac, None, sp.move, sp.bisect_tol)
    t_el = (time.perf_counter() - t0) * (nelz / zs)
    t_oc = args.cpu_its * t_it + t_el + t_asm
    cores = csr.threads()
    return {"value": 1.0 / t_oc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle's C part (assembled CSR, FP64 Jacobi-PCG, OpenMP on {cores} threads) "
                       f"on a {nelx}x{nely}x{zs} slab of the {nelx}x{nely}x{nelz} grid: {reps} PCG "
                       f"iterations timed ({t_it:.3f} s each at full size), CSR assembly "
                       f"({t_asm:.2f} s) and energies + filter + OC ({t_el:.2f} s), each scaled by "
                       f"element count; OC iteration = {args.cpu_its:.0f} PCG iterations (the "
                       f"library's FP64 Jacobi-PCG count on the bench designs, "
                       f"{'measured in this run' if args.cpu_its != REF_ITERS_PER_OC else 'its mean over OC iterations 4-11 at this size from earlier runs'}"
                       f") + the rest"),
            "t_pcg_iter_s": t_it, "t_assembly_s": t_asm, "t_elementwise_s": t_el,
            "pcg_iters_per_oc": args.cpu_its, "nproc": os.cpu_count()}


def run_cpu_leg_subprocess(args, its):
    env = dict(os.environ, OMP_NUM_THREADS=str(os.cpu_count() or 1))
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--size", args.size,
           "--cpu-its", str(its), "--cpu-reps", str(args.cpu_reps)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def workload_config(args, world):
    """The `config` object both arms print."""
    return {"workload": f"cantilever {args.size}, centre load on x=nelx face, volfrac 0.2, "
                        f"rmin 2.5, penal 3, OC iterations {args.warmup + 1}-"
                        f"{args.warmup + args.steps} from x0 = volfrac",
            "solver_rtol": 1e-8,
            "l2": "working set (>1 GB) larger than L2; no flush needed",
            "parallelism": f"replicas x{world}"}


def reference_arm(args):
    """The oracle as the reference arm: each step is one bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    r = None
    for i in range(args.warmup + args.steps):
        r = run_cpu_leg_subprocess(args, args.cpu_its)
        if "error" in r:
            print(json.dumps({"impl": "reference", "unavailable": r["error"][-200:]}))
            return
        if i >= args.warmup:
            vals.append(r["value"])
    v = statistics.mean(vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(workload_config(args, 1), form="fp64 oracle (CPU)",
                           sample="bounded (see cpu_baseline)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm
# DRAM bytes (read + write) of one launch of the fused tensor-core kernel at
# 480x160x80 from one ncu capture of the current kernel (profiles/), keyed by
# (precision, preconditioner, grid); reported only for the form and size
# captured (the z-segment length, and so the halo traffic, is tuned per form).
TC_TRAFFIC_BYTES = {(1, "lmg", 480, 160, 80): 241_737_216 + 128_706_816}


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (x itself on one process): the
    job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, ms: float) -> float:
    """Whole-job OC iterations per second: every replica runs `steps`."""
    return world * steps / (ms / 1000.0)


def algorithmic_bytes_tc(nelx, nely, nelz):
    """Per launch of the fused tensor-core matvec + direction kernel:
    read r (or z), p_old (4 B/dof each), the per-node scaling (4 B/node), E
    (4 B/element); write p_new and q (4 B/dof each)."""
    N = (nelx + 1) * (nely + 1) * (nelz + 1)
    nel = nelx * nely * nelz
    n = 3 * N
    return 4 * n * 4 + 4 * N + 4 * nel


def cnn_flops(nelx, nely, nelz):
    """Algorithmic FLOPs of one U-Net application on the node grid padded to
    multiples of 8: 2 * 27 * C_in * C_out per voxel and layer, with the real
    4 input and 3 output channels (the kernels pad them to 16)."""
    pad = lambda n: (n + 1 + 7) // 8 * 8
    v0 = pad(nelx) * pad(nely) * pad(nelz)
    layers = [(4, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 64, 2),
              (64, 64, 3), (64, 64, 3), (128, 64, 2), (64, 64, 2), (96, 32, 1), (32, 32, 1),
              (48, 16, 0), (16, 16, 0), (16, 3, 0)]
    return sum(2 * 27 * ci * co * v0 / 8 ** lev for ci, co, lev in layers)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


TRAIN_AT = (8, 16, 24, 32, 40)    # OC iterations after which snapshots are taken
TRAIN_SNAPS = 2                    # snapshots per design
TRAIN_STEPS = 20


def train_lmg(stream):
    """Learn the multigrid parameters on a 96x32x16 cantilever of the bench's
    family: snapshots of designs along its own OC trajectory (the multigrid
    form runs the trajectory); returns (theta, record)."""
    import torch
    from paper_2504_05604_gb300 import LMG, Context
    from synth import problems
    small = problems.config_large(nelx=TRAIN_GRID[0], nely=TRAIN_GRID[1], nelz=TRAIN_GRID[2])
    t0 = time.perf_counter()
    tctx = Context.from_problem(small, precision=0, precond=LMG, stream=stream.cuda_stream)
    it = 0
    for k, at in enumerate(TRAIN_AT):
        while it < at:
            tctx.step()
            it += 1
        last_call = k == len(TRAIN_AT) - 1
        first, last = tctx.mg_train(nsnap=TRAIN_SNAPS, steps=TRAIN_STEPS if last_call else 0,
                                    lr=0.1, seed=3, append=k > 0)
    theta = tctx.mg_params()
    tctx.close()
    torch.cuda.synchronize()
    return theta, {"grid": "x".join(map(str, TRAIN_GRID)), "snapshots_after_oc_iterations":
                   list(TRAIN_AT), "snapshots": TRAIN_SNAPS * len(TRAIN_AT),
                   "adam_steps": TRAIN_STEPS, "loss_first": first, "loss_last": last,
                   "theta": [round(float(v), 4) for v in theta],
                   "seconds": time.perf_counter() - t0}


def unet_leg(prob, stream, x_start, fp64_iters):
    """One OC iteration of the U-Net flexible-CG form from a design (the
    network trained first, on the GPU, on residual snapshots of a 96x32x16
    cantilever of the same family)."""
    import torch
    from paper_2504_05604_gb300 import CNN_FCG, Context
    from synth import problems
    small = problems.config_large(nelx=96, nely=32, nelz=16)
    tctx = Context.from_problem(small, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    first, last = tctx.cnn_train(nsnap=24, per_design=4, steps=1500, lr=1e-3, seed=7)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    flat = tctx.cnn_params()
    tctx.close()
    lctx = Context.from_problem(prob, precond=CNN_FCG, stream=stream.cuda_stream,
                                fcg_ref_iters=int(fp64_iters))
    lctx.set_cnn_params(flat)
    lctx.set_density(x_start)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = lctx.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lctx.close()
    return {"value": 1000.0 / ms, "unit": UNIT, "cg_iters": r["cg_iters"],
            "fell_back_to_jacobi_pcg": r["outer_iters"] == 2, "relres": r["relres"],
            "status": r["status"], "train_s": train_s, "train_loss_first": first,
            "train_loss_last": last}


def form_on_designs(prob, stream, samples, **form):
    """One OC iteration of a form from each sampled (design, displacement):
    CUDA-event times, iterations and residuals."""
    import torch
    from paper_2504_05604_gb300 import Context
    theta = form.pop("theta", None)
    ctx = Context.from_problem(prob, stream=stream.cuda_stream, **form)
    if theta is not None:
        ctx.set_mg_params(theta)
    out = []
    for label, x, u in samples:
        ctx.set_density(x)
        ctx.set_displacement(u)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ctx.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out.append({"design": label, "value": 1000.0 / ms, "ms": ms, "cg_iters": r["cg_iters"],
                    "outer_iters": r["outer_iters"], "relres": r["relres"],
                    "status": r["status"], "compliance": r["compliance"]})
    ctx.close()
    return {"unit": UNIT, "value": len(out) / sum(o["ms"] / 1000.0 for o in out),
            "per_design": out}


def ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2504_05604_gb300 import build as libbuild
    libbuild.build()
    from paper_2504_05604_gb300 import JACOBI, LMG, Context
    from synth import problems

    nelx, nely, nelz = dims(args)
    prob = problems.config_large(nelx=nelx, nely=nely, nelz=nelz)
    stream = torch.cuda.Stream(device=dev)
    lmg = args.precond == "lmg"
    theta, train = (train_lmg(stream) if lmg else (None, None))
    # fp64_tc: the FP64 residual replacements on the tensor cores by exact
    # integer slicing (FP64 accuracy)
    # mg_keep_dir: the inner CG keeps its direction across the residual
    # replacements (restarting only when the true residual fails to halve)
    form = dict(precision=args.precision, precond=LMG if lmg else JACOBI,
                inner_rtol=args.inner_rtol, fp64_tc=0 if args.fp64_cuda_cores else 1,
                mg_keep_dir=1 if lmg else 0)

    def make_ctx():
        c = Context.from_problem(prob, stream=stream.cuda_stream, **form)
        if theta is not None:
            c.set_mg_params(theta)
        return c

    ctx = make_ctx()
    warm = [ctx.step() for _ in range(args.warmup)]

    def barrier():
        if world > 1:
            dist.barrier()

    # the designs the comparison forms start from: the window's start,
    # middle and end, each with the displacement the run had there (every
    # form warm-starts from it); copied on the device, outside the timed parts
    mid = args.steps // 2
    xs = [torch.empty(prob.nel, dtype=torch.float64, device=dev) for _ in range(3)]
    us = [torch.empty(prob.ndof, dtype=torch.float64, device=dev) for _ in range(3)]

    def sample(i):
        with torch.cuda.stream(stream):
            ctx.density(xs[i])
            ctx.displacement(us[i])

    with torch.cuda.stream(stream):
        sample(0)
        ctx.kernel_stats(0, reset=True)
        l0 = ctx.launches
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        clk = ClockSampler(local)
        barrier()
        torch.cuda.synchronize()
        clk.start()
        # an NVTX range marks the timed steps for profilers (ncu --nvtx
        # --nvtx-include "timed/"); it costs nothing without one
        torch.cuda.nvtx.range_push("timed")
        ev[0].record(stream)
        recs = [ctx.step() for _ in range(mid)]
        ev[1].record(stream)
        sample(1)
        ev[2].record(stream)
        recs += [ctx.step() for _ in range(args.steps - mid)]
        ev[3].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clocks = clk.stop()
        barrier()
        ms = ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
        launches = ctx.launches - l0
        tc_ms, tc_n = ctx.kernel_stats(0)
        sample(2)
        torch.cuda.synchronize()
    ms = max_over_ranks(ms, dev)
    value = job_value(world, args.steps, ms)
    status = max(r["status"] for r in recs)
    its = [r["cg_iters"] for r in recs]

    # end to end through the public API with host buffers, on the same OC
    # iterations: a second context repeats the warm-up, then every timed
    # step copies the design host -> device, runs one OC iteration and
    # reads the new design and the iteration record back
    e2e = None
    if not args.no_e2e:
        ctx_e = make_ctx()
        for _ in range(args.warmup):
            ctx_e.step()
        xh = torch.empty(prob.nel, dtype=torch.float64).pin_memory().numpy()
        ctx_e.density(xh)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx_e.set_density(xh)
            ctx_e.step()
            ctx_e.density(xh)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        ctx_e.close()
        te = max_over_ranks(te, dev)
        e2e = {"value": job_value(world, args.steps, 1000.0 * te), "unit": UNIT,
               "h2d_bytes_per_step": 8 * prob.nel,
               "d2h_bytes_per_step": 8 * prob.nel + 112}

    # the other forms, one OC iteration from each of the three designs
    samples = [(f"after OC iteration {args.warmup + k}", xs[i], us[i])
               for i, k in enumerate((0, mid, args.steps))]
    fp64 = learned = jacobi_dc = fp64_sliced = None
    if not args.no_fp64:
        fp64 = form_on_designs(prob, stream, samples, precision=0)
        learned = form_on_designs(prob, stream, samples, precision=0, precond=LMG, theta=theta,
                                  fp64_tc=form["fp64_tc"])
        jacobi_dc = form_on_designs(prob, stream, samples, precision=1, inner_rtol=0.3)
        # plain FP64 Jacobi-PCG with the sliced tensor-core FP64 K p, on the
        # last design only (about half a minute)
        fp64_sliced = form_on_designs(prob, stream, samples[-1:], precision=0, fp64_tc=1)
    unet = None
    if args.unet:
        unet = unet_leg(prob, stream, xs[2].cpu().numpy(),
                        fp64["per_design"][-1]["cg_iters"] if fp64 else 0)

    if rank != 0:
        return
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    tc_avg_ms = tc_ms / tc_n if tc_n else None
    roof = None
    if tc_avg_ms:
        b = algorithmic_bytes_tc(nelx, nely, nelz)
        ach = b / (tc_avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": TC_TRAFFIC_BYTES.get((args.precision, args.precond, nelx, nely, nelz)),
                "kernel": "k_matvec_tc (fused direction + tensor-core K p)",
                "launch_ms": tc_avg_ms, "algorithmic_bytes": b, "samples": tc_n,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}
    cpu = None
    if not args.no_cpu and world == 1:
        # the oracle solves with FP64 Jacobi-PCG: its iteration count is the
        # plain FP64 form's on the same designs
        n64 = (statistics.mean(o["cg_iters"] for o in fp64["per_design"]) if fp64
               else REF_ITERS_PER_OC)
        cpu = run_cpu_leg_subprocess(args, n64)
    name = PREC_NAMES[args.precision] + ("-lmg" if lmg else "")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": dict(workload_config(args, world), form=name, fp64_tc=form["fp64_tc"],
                       arithmetic=ARITHMETIC[args.precision] + (
                           "; preconditioner: learned multigrid V-cycle (FP32, tensor-core "
                           "operator on every level)" if lmg else "; Jacobi preconditioner"),
                       inner_rtol=args.inner_rtol, mg_keep_dir=form["mg_keep_dir"]),
        "gpu_launches": int(launches),
        "status": int(status),
        "cg_iters_per_step": its,
        "phase_ms": {k: statistics.mean(r[k] for r in recs)
                     for k in ("ms_solve", "ms_sens", "ms_filter", "ms_oc")},
        "compliance": [r["compliance"] for r in recs],
        "clocks": clocks,
        "roofline": roof,
        "lmg_training": train,
        "plain_fp64": fp64,
        "learned_fcg": learned,
        "jacobi_dc": jacobi_dc,
        "plain_fp64_sliced_tc": fp64_sliced,
        "unet_fcg": unet,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if fp64:
        line["speedup_vs_plain_fp64_same_designs"] = {
            "chosen_window": value / fp64["value"],
            "learned_fcg": learned["value"] / fp64["value"],
            "jacobi_dc": jacobi_dc["value"] / fp64["value"]}
    print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def batched(args):
    """64 seeded uneven cantilevers (0-3 spherical voids) stepped together,
    one CUDA graph per problem and OC iteration; compared with stepping the
    same problems one after another through single contexts."""
    import torch
    from paper_2504_05604_gb300 import build as libbuild
    libbuild.build()
    from paper_2504_05604_gb300 import Batch, Context
    from synth import problems

    probs = problems.config_batched(64)
    stream = torch.cuda.current_stream()
    lmg = args.precond == "lmg"
    if lmg:
        # the learned multigrid in every problem's graph, with the parameters
        # learned as for the large workload
        from paper_2504_05604_gb300 import LMG
        prec = args.precision
        theta, _ = train_lmg(torch.cuda.Stream())
        b = Batch(probs, precision=prec, precond=LMG, inner_rtol=args.inner_rtol)
        b.set_mg_params(theta)
    else:
        # the two-slice operand: on these small, void-riddled grids the single-
        # slice one stalls the device-side Jacobi defect correction of some problems
        prec = args.precision if args.precision in (2, 4) else 2
        b = Batch(probs, precision=prec, inner_rtol=args.inner_rtol)
    for _ in range(args.warmup):
        b.step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    recs = [b.step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b.close()
    # the same problems one after another through single contexts (host-
    # driven solver, no graphs), the same OC iterations: W untimed, K timed
    t_seq = 0.0
    for pr in probs:
        c = Context.from_problem(pr, precision=prec, inner_rtol=args.inner_rtol,
                                 precond=(2 if lmg else 0))
        if lmg:
            c.set_mg_params(theta)
        for _ in range(args.warmup):
            c.step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c.step()
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
        c.close()
    nel = sum(p.nel for p in probs)
    print(json.dumps({
        "metric": "OC iters/s, 64 seeded uneven cantilevers stepped together",
        "value": 64 * args.steps / (ms / 1000.0), "unit": "problem OC iters/s",
        "elements": nel, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "form": PREC_NAMES[prec] + ("-lmg" if lmg else ""),
        "status": max(r["status"] for rr in recs for r in rr),
        "cg_iters_mean": statistics.mean(r["cg_iters"] for rr in recs for r in rr),
        "sequential_single_contexts": {"value": 64 * args.steps / t_seq,
                                       "unit": "problem OC iters/s",
                                       "note": "the same OC iterations, one problem after "
                                               "another, host wall clock"},
    }))


def paper_benchmark(args):
    """The paper's own benchmark (Section 4.2, Table 1): the 32x16x16
    cantilever, volfrac 0.2, penal 3, rmin 4, 200 OC iterations, timed end to
    end (all 200 iterations, as the paper times its run) in the FP64 form and
    the chosen form; then the usage example (Section 3: the same cantilever
    with a cylindrical obstacle) in the chosen form, with its voxels of
    density above 0.5 and an STL surface written to --export.  The paper's
    laptop-CPU figure is context only."""
    import torch
    from paper_2504_05604_gb300 import build as libbuild
    libbuild.build()
    from paper_2504_05604_gb300 import LMG, Context, export
    from synth import problems
    lmg = args.precond == "lmg"
    theta = train_lmg(torch.cuda.Stream())[0] if lmg else None

    def run(prob, prec, use_lmg):
        kw = dict(precision=prec, inner_rtol=args.inner_rtol if use_lmg else 0.3)
        if use_lmg:
            kw["precond"] = LMG
        ctx = Context.from_problem(prob, **kw)
        if use_lmg:
            ctx.set_mg_params(theta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs = ctx.run(prob.iters)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        x = ctx.density()
        ctx.close()
        return {"value": prob.iters / te, "unit": UNIT, "total_s": te,
                "final_compliance": recs[-1]["compliance"],
                "final_volume": recs[-1]["volume"],
                "cg_iters_mean": statistics.mean(r["cg_iters"] for r in recs),
                "status": max(r["status"] for r in recs)}, x

    prob = problems.config_paper_benchmark()
    out = {}
    out["fp64"], _ = run(prob, 0, False)
    chosen = PREC_NAMES[args.precision] + ("-lmg" if lmg else "")
    out[chosen], _ = run(prob, args.precision, lmg)
    out["fp64-lmg"], _ = run(prob, 0, lmg)
    best = max(out, key=lambda k: out[k]["value"])
    usage = problems.config_paper_usage()
    use_rec, x = run(usage, args.precision, lmg)
    pas = usage.passive
    use_rec["obstacle_elements"] = int((pas == 1).sum())
    use_rec["obstacle_max_density"] = float(x[pas == 1].max())
    if args.export:
        os.makedirs(args.export, exist_ok=True)
        dims = (usage.nelx, usage.nely, usage.nelz)
        export.write_voxels(os.path.join(args.export, "usage_voxels.npy"), x, dims)
        tris = export.isosurface(x, dims)
        export.write_stl(os.path.join(args.export, "usage_design.stl"), tris)
        use_rec["export"] = {"voxels_above_0.5": int((x > 0.5).sum()), "stl_triangles": len(tris),
                             "dir": args.export}
    print(json.dumps({
        "metric": "OC iters/s on the paper's benchmark (32x16x16, 200 iterations, whole run)",
        "value": out[best]["value"], "unit": UNIT, "chosen_form": best,
        "forms": out,
        "usage_example_with_obstacle": use_rec,
        "paper_context": {"value": 200 / 147.3, "unit": UNIT, "total_s": 147.3,
                          "hardware": "Intel Core Ultra 7 155U laptop CPU (Section 4.2, Table 1)",
                          "note": "another machine and a direct solver: context, not a target"},
    }))


def whole_runs(args):
    """Whole runs of the 60x20x4 (50 OC iterations) or the 240x80x40
    void-cylinder (100 OC iterations) cantilever: plain FP64 Jacobi-PCG, the
    chosen form (learned parameters as for the large workload) and Jacobi
    BF16 defect correction, each timed over the whole run."""
    import torch
    from paper_2504_05604_gb300 import build as libbuild
    libbuild.build()
    from paper_2504_05604_gb300 import LMG, Context
    from synth import problems
    prob = problems.config_small() if args.workload == "config1" else problems.config_void_cylinder()
    theta = train_lmg(torch.cuda.Stream())[0]
    forms = {"fp64": dict(precision=0),
             PREC_NAMES[args.precision] + "-lmg": dict(precision=args.precision, precond=LMG,
                                                       inner_rtol=args.inner_rtol, fp64_tc=1,
                                                       mg_keep_dir=1),
             "fp64-lmg (learned FCG)": dict(precision=0, precond=LMG, fp64_tc=1),
             "bf16-dc (Jacobi)": dict(precision=1, inner_rtol=0.3)}
    out = {}
    for name, kw in forms.items():
        ctx = Context.from_problem(prob, **kw)
        if kw.get("precond") == LMG:
            ctx.set_mg_params(theta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs = ctx.run(prob.iters)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        out[name] = {"value": prob.iters / te, "unit": UNIT, "total_s": te,
                     "final_compliance": recs[-1]["compliance"],
                     "final_volume": recs[-1]["volume"],
                     "cg_iters_mean": statistics.mean(r["cg_iters"] for r in recs),
                     "cg_iters_max": max(r["cg_iters"] for r in recs),
                     "status": max(r["status"] for r in recs)}
        ctx.close()
    ref = out["fp64"]["final_compliance"]
    for v in out.values():
        v["final_compliance_vs_fp64"] = v["final_compliance"] / ref - 1.0
    print(json.dumps({"metric": f"OC iters/s, whole run of {prob.name} ({prob.iters} OC iterations)",
                      "unit": UNIT, "forms": out}))


def main():
    args = parse()
    if args.workload == "batched64" and not args.cpu_leg and args.impl == "ours":
        batched(args)
        return
    if args.workload in ("config1", "config2") and not args.cpu_leg and args.impl == "ours":
        whole_runs(args)
        return
    if args.workload == "paper32" and not args.cpu_leg and args.impl == "ours":
        paper_benchmark(args)
        return
    if args.cpu_leg:
        print(json.dumps(cpu_leg(args)))
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    ours(args)


if __name__ == "__main__":
    main()
