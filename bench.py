"""Benchmark: zone-updates/s of the IMEX-SSP2(2,2,2) resistive-GRMHD step on
the 256^3 cylindrical-blast workload (flat space, MC2 + HLLE, sigma = 1e3),
mixed precision (FP32 reconstruction/fluxes, FP64 recovery and accumulation)
as the headline and the FP64 path beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--n 256] [--precision mixed|fp64] [--no-adjoint]
                    [--adjoint-n 128] [--adjoint-steps 60] [--adjoint-every 10]

The "adjoint" object times the gradient of a B^y misfit after 60 steps of
the 128^3 Alfven cube (rmhd_adjoint_forward + rmhd_adjoint_backward); the
"configs" object the Brio-Wu shocktube's latency per step, the 128^3
Alfven cube and the 192^3 curved star (--no-adjoint, --no-configs skip them).

Timing: untimed steps from the initial data (the W warm-up steps, then on
to the middle of the configuration's 100-step run), then K steps through
rmhd_step (one step captured as a CUDA graph and replayed: the product
call), CUDA events on the launching stream with a synchronize on both
sides; `value` is that window (steps 41-60 for K = 20).  The cost of a step
grows as the blast evolves, and a window in the middle of the run costs
about its mean.  The same K steps are then re-run from the same state
through rmhd_step_profiled (events between the kernel groups) for the
per-kernel rooflines, and the configuration's whole 100-step run from the
initial data is timed in ten blocks for both precisions ("run100",
"fp64_run100"), then run again with events between the kernel groups (ms per
step of each group by block of ten steps).

One JSON line on stdout (rank 0).  With N > 1 (torchrun) the grid is split
into z-slabs, one per rank and GPU, with halos exchanged point to point after
every step (paper_2510_18968_b300/slabs.py); value = the grid's
zone-updates / the slowest rank's time (strong scaling).
--impl reference times the FP64 CPU oracle on a bounded z-slab of the same
workload on the host cores.
"""
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

import workloads as W  # noqa: E402

METRIC = "zone-updates/s per IMEX-RK2 step at 256^3 (FP64 vs mixed) + % HBM roofline"
UNIT = "zone-updates/s"

# Measured on this machine's B300 (HBM copy bandwidth written by the driver, FP64
# and FP32 FMA throughput by our own probe): see the design notes.
# Compulsory state bytes per zone-update of a fully fused step (each state
# array read or written once per stage; flat metric): FP64 path, and the
# mixed path with FP32 primitives and FP64 conserved / stiff arrays.
ALG_BYTES_PER_ZONE = {"fp64": 1200, "mixed": 904}
FP64_PEAK_TFLOPS = 1.203   # 148 SM x 2 DFMA/clk x 2 flop x 2.032 GHz


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    except OSError:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max_ms(ms, world, device):
    """The slowest rank's time (every rank gets it): the job ends when the
    last replica does."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_cells, steps, world, max_ms):
    """Whole-job zone-updates/s: every rank advances its own replica of
    n_cells by `steps` steps; the job takes the slowest rank's time."""
    return world * n_cells * steps / (max_ms * 1e-3)


def workload(n, imex=0):
    wl = W.cyl_blast(n=n)
    wl.params["imex"] = imex
    return wl


IMEX_LABELS = {0: "SSP2(2,2,2)", 1: "SSP2(3,3,2)", 2: "SSP3(3,3,2)", 3: "SSP3(4,3,3)"}
# Structure of the general IMEX form per scheme (from its tableaux): the rows
# after the first stage as (nonzero explicit coefficients, nonzero implicit
# off-diagonal coefficients, F of the previous stage formed in the row), the
# weights row as (nonzero wt, nonzero w), and the stages whose F is formed
# (one face-flux pass each).  Table imex: one row (1, 1, True), weights (2, 2).
IMEX_ROWS = {
    0: ([(1, 1, True)], (2, 2), 2),
    1: ([(1, 0, True), (2, 2, True)], (3, 3), 3),
    2: ([(1, 1, True), (2, 1, True)], (3, 3), 3),
    3: ([(0, 1, False), (1, 1, True), (2, 3, True)], (3, 3), 3),
}


# Algorithmic work per zone of each kernel group (counted from the kernel
# source; FMA = 2 flops, division / square root = 1).  Recovery kernels: a
# fixed part per cell (stage set-up, IMEX accumulation, outputs) plus the
# paper iteration's flops times the mean number of iterations per recovery
# measured over the timed steps; the fallbacks count as overhead.
# Flux kernels: per face, HBM bytes of a stencil read once (15 fields in,
# 14 out) and flops of reconstruction + two flux states + HLLE.
# FP64 only: the paper iteration's 1/f' and its change measures and stopping
# decisions run in FP32, and so do the mixed path's stage currents.
PAPER_ITER_FLOPS = {"implicit": 94, "fixed_E": 52}   # one paper iteration
FP64_FIXED = {  # per cell, (mixed path, FP64 path)
    "stage1_recovery": (19, 28),
    "stage2_rhs_recovery": (88, 189),
    "final_rhs_recovery": (44, 136),
}


# the FP64 path forms the flux difference and sources in FP64 (92 flops)
RHS_FP64 = 92


def fp64_flops(name, prec, iters, imex=0):
    """Algorithmic FP64 flops per cell of one launch of a recovery group.
    The general IMEX form (imex > 0) counts, per row, 2 flops per field and
    nonzero coefficient of its combination (the average over the rows that
    one launch of the stage-row kernel runs) on top of the recovery."""
    per = PAPER_ITER_FLOPS["fixed_E" if name == "final_rhs_recovery" else "implicit"]
    if imex == 0 or name == "stage1_recovery":
        fixed = FP64_FIXED[name][0 if prec == "mixed" else 1]
        return fixed + iters * per
    rows, (nw, nwr), _ = IMEX_ROWS[imex]
    rhs = RHS_FP64 if prec == "fp64" else 0
    if name == "stage2_rhs_recovery":
        fixed = sum(28 + 2 * 14 * nf + 2 * 3 * nr + (rhs if formed else 0)
                    for nf, nr, formed in rows) / len(rows)
    else:
        fixed = 16 + 2 * 14 * nw + 2 * 3 * nwr + rhs
    return fixed + iters * per
# face flops: 15 reconstructed fields x 2 sides (MC2 slope ~12 flops, WENO5
# ~65 with its four divisions), two one-side flux states (~180 each: W,
# enthalpy, EM energy, E x B, stress rows, EM rows, the HLLE accumulation)
FLUX_FLOPS_PER_FACE_BY_RECON = {0: 30 * 10 + 360, 1: 30 * 12 + 360, 2: 30 * 65 + 360}
FLUX_FIELDS = 15 + 14

# DRAM bytes per cell of one launch (dram__bytes_read.sum +
# dram__bytes_write.sum from ncu on a 128^3 launch of this workload, scaled
# by the cell count; traffic grows with the cells).  Valid for the kernels
# as they are; re-measure after changing one.
TRAFFIC_PER_CELL = {
    ("stage2_rhs_recovery", "mixed"): (884.850944e6 + 493.886976e6) / 128 ** 3,
    # k_flux_xwalk (x) and k_flux_walk (y, z) with TMA tile loads, mean of
    # the three launches
    ("flux_stage2", "mixed"): ((148.613376e6 + 152.915712e6 + 153.597952e6) +
                               (77.392640e6 + 84.397824e6 + 85.279232e6)) / 3 / 128 ** 3,
    # k_flux_run, mean of the x, y, z launches
    ("flux_stage2", "fp64"): ((989.442560e6 + 372.153600e6 + 303.645184e6) +
                              (514.565888e6 + 203.661056e6 + 202.688768e6)) / 3 / 128 ** 3,
}


def launches_per_step(wl):
    """Kernels one step launches: a recovery kernel and its two deferred
    passes (one thread per record, then one warp per record for those that
    need the rest of the fallback chain) per stage and for the final
    recovery, the ghost fills (primitives, and the
    stage currents when the charge flux uses them) of every stage whose F is
    formed and of the result, one flux kernel per active direction and
    formed F."""
    nd = sum(1 for d in range(3) if wl.params["n"][d] > 1)
    rows, _, nflux = IMEX_ROWS[wl.params.get("imex", 0)]
    stages = len(rows) + 1
    ghosts = nflux * (2 if wl.params["qflux_mode"] == 0 else 1) + 1
    return 3 * (stages + 1) + ghosts + nflux * nd


def e2e_pipelined(R, torch, wl, prec, cons_h, prim_h, jobs_per_handle, handles=2):
    """End to end through the public API as a server would run independent
    one-step jobs: several handles, each on its own CUDA stream and driven
    by its own host thread, so that one job's host -> device upload and
    device -> host read overlap other jobs' steps and copies; handle k
    starts once handle k-1 has finished its first upload.  Every job uploads
    its input from pinned host memory, steps once and reads the primitives
    back; returns zone-updates/s.  The input is the primitives alone
    (rmhd_set_prims, which forms the conserved variables on the device) or,
    with cons_h given, the conserved variables with the primitives as the
    recovery guess (rmhd_set_state, twice the upload)."""
    import threading
    params = dict(wl.params, precision=1 if prec == "mixed" else 0)
    streams = [torch.cuda.Stream() for _ in range(handles)]
    solvers = [R.Solver(params, stream=st) for st in streams]
    outs = [torch.empty((14,) + wl.shape, dtype=torch.float64).pin_memory().numpy()
            for _ in solvers]
    uploaded = [threading.Event() for _ in solvers]

    def job(k):
        s = solvers[k]
        if cons_h is None:
            s.set_prims(prim_h)
        else:
            s.set_state(cons_h, prim_h)
        uploaded[k].set()
        s.step(wl.dt, 1, sync=False)
        s.get_prims(outs[k])

    for k in range(handles):   # warm-up: first job of each handle
        job(k)
    barrier = threading.Barrier(handles + 1)

    def worker(k):
        barrier.wait()
        if k > 0:
            uploaded[k - 1].wait()
        for _ in range(jobs_per_handle):
            job(k)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(handles)]
    for t in threads:
        t.start()
    for e in uploaded:
        e.clear()
    barrier.wait()
    t0 = time.perf_counter()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for s in solvers:
        s.close()
    return wl.ncells * handles * jobs_per_handle / dt


def timed_steps(s, dt, k, torch, blocks=1):
    """k steps through rmhd_step (one captured step replayed as a CUDA graph,
    the product call), CUDA events on the launching stream with a
    synchronize on both sides; returns the total ms and the ms of each of
    `blocks` equal blocks of steps."""
    st = torch.cuda.current_stream()
    per = [k // blocks + (1 if b < k % blocks else 0) for b in range(blocks)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(blocks + 1)]
    torch.cuda.synchronize()
    ev[0].record(st)
    for b, kb in enumerate(per):
        if kb:
            s.step(dt, kb, sync=False)
        ev[b + 1].record(st)
    torch.cuda.synchronize()
    blk = [ev[b].elapsed_time(ev[b + 1]) for b in range(blocks)]
    return sum(blk), blk, per


RUN_STEPS = 100   # the cylindrical-blast configuration's run length


def window_start(args):
    """Steps before the timed window.  The cost of a step grows as the blast
    evolves, so the K timed steps sit in the middle of the configuration's
    100-step run (steps 41-60 for K = 20), where the step costs about the
    run's mean; at least the W warm-up steps precede them."""
    if args.no_run100:      # short profiling runs: the window right after warm-up
        return args.warmup
    return max(args.warmup, (RUN_STEPS - args.steps) // 2)


def run_ours(args, rank, world, local):
    import torch
    import paper_2510_18968_b300 as R

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = workload(args.n, args.imex)
    N = wl.ncells
    prim0 = np.ascontiguousarray(wl.prim)
    out = {}
    for prec in (["mixed", "fp64"] if args.precision == "both" else [args.precision]):
        s = R.Solver(dict(wl.params, precision=1 if prec == "mixed" else 0))
        s.set_prims(prim0)
        # untimed steps up to the window: the W warm-up steps (and the graph
        # capture), then on to the window's start in the middle of the run
        s.step(wl.dt, window_start(args))
        torch.cuda.synchronize()
        # state at the start of the timed window (for the per-kernel leg)
        cons_w, prim_w = s.get_cons(), s.get_prims()
        if world > 1:
            torch.distributed.barrier()
        sampler = ClockSampler(local)
        st0 = s.stats()
        with sampler:
            ms_local, _, _ = timed_steps(s, wl.dt, args.steps, torch)
        st1 = s.stats()
        iters = ((st1["c2p_iterations"] - st0["c2p_iterations"]) /
                 max(1, st1["c2p_calls"] - st0["c2p_calls"]))
        ms = reduce_max_ms(ms_local, world, "cuda")
        stats = {k: st1[k] - st0[k] for k in st1}
        # per-kernel leg: the same K steps again from the same state, with
        # CUDA events between the kernel groups (rmhd_step_profiled)
        s.set_state(cons_w, prim_w)
        groups = s.step_profiled(wl.dt, args.steps)
        # the configuration's whole run: RUN_STEPS steps from the initial
        # data through rmhd_step, timed in ten blocks (the cost per step
        # grows as the blast evolves)
        s.set_prims(prim0)
        str0 = s.stats()
        nrun = 10 if args.no_run100 else RUN_STEPS
        ms_run, blk, per = timed_steps(s, wl.dt, nrun, torch, blocks=10)
        str1 = s.stats()
        run = {"steps": nrun, "ms": ms_run,
               "ms_per_step_by_block": [b / k for b, k in zip(blk, per)],
               "paper_iterations_per_recovery":
                   (str1["c2p_iterations"] - str0["c2p_iterations"]) /
                   max(1, str1["c2p_calls"] - str0["c2p_calls"]),
               "fallbacks_per_recovery":
                   (str1["c2p_fallbacks"] - str0["c2p_fallbacks"]) /
                   max(1, str1["c2p_calls"] - str0["c2p_calls"]),
               "atmosphere_resets": (str1["c2p_failures"] - str0["c2p_failures"]) +
                                    (str1["atmo_floor_resets"] - str0["atmo_floor_resets"])}
        # the same run again with events between the kernel groups
        # (rmhd_step_profiled): ms per step of each group, by block of ten steps
        s.set_prims(prim0)
        by_block = []
        for b in range(10):
            sb0 = s.stats()
            g = s.step_profiled(wl.dt, nrun // 10)
            sb1 = s.stats()
            calls = max(1, sb1["c2p_calls"] - sb0["c2p_calls"])
            row = {k: v / (nrun // 10) for k, v in g.items()}
            row["iterations_per_recovery"] = (sb1["c2p_iterations"] - sb0["c2p_iterations"]) / calls
            row["fallbacks_per_recovery"] = (sb1["c2p_fallbacks"] - sb0["c2p_fallbacks"]) / calls
            by_block.append(row)
        run["groups_ms_per_step_by_block"] = by_block
        # end-to-end through the public API with host buffers: every job
        # uploads the primitives of the evolved state from pinned host
        # memory (rmhd_set_prims), steps once and reads the primitives back
        s.set_state(cons_w, prim_w)
        cons_h = torch.empty((14,) + wl.shape, dtype=torch.float64).pin_memory().numpy()
        prim_h = torch.empty((14,) + wl.shape, dtype=torch.float64).pin_memory().numpy()
        s.get_cons(cons_h)
        s.get_prims(prim_h)
        prim_in = torch.empty((14,) + wl.shape, dtype=torch.float64).pin_memory().numpy()
        prim_in[...] = prim_h
        ke = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            s.set_prims(prim_in)
            s.step(wl.dt, 1, sync=False)
            s.get_prims(prim_h)
        torch.cuda.synchronize()
        e2e_serial_s = time.perf_counter() - t0
        s.close()
        e2e_pipe = e2e_pipelined(R, torch, wl, prec, None, prim_in, 6, handles=3)
        e2e_state = e2e_pipelined(R, torch, wl, prec, cons_h, prim_in, 6)
        out[prec] = dict(ms=ms, groups=groups, stats=stats, clocks=sampler.summary(), iters=iters,
                         run=run, e2e=e2e_pipe, e2e_serial=N * ke / e2e_serial_s,
                         e2e_state=e2e_state, e2e_bytes=(14 * N * 8, 14 * N * 8))
    return wl, out


def run_slabs(args, rank, world, local):
    """N > 1: the 256^3 grid split into z-slabs over the ranks (one GPU
    each), halos of H layers exchanged point to point (NCCL) after every
    step (paper_2510_18968_b300.slabs).  Every rank times W warm-up and K
    timed steps (step + exchange) between a barrier and a synchronize on
    both sides; the job's time is the slowest rank's and the value counts
    the grid's cells once (strong scaling: the total work is fixed).
    End to end: each rank uploads its slab's primitives from pinned host
    memory, steps once with the exchange, and reads its slab back."""
    import torch
    import torch.distributed as dist
    import paper_2510_18968_b300 as R
    from paper_2510_18968_b300 import slabs as S

    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    wl = workload(args.n, args.imex)
    nz = wl.params["n"][2]
    H = S.halo_layers(wl.params)
    periodic = wl.params["bc"][2] == 0
    slab = S.make_slab(nz, world, rank, H, periodic)
    out = {}
    for prec in (["mixed", "fp64"] if args.precision == "both" else [args.precision]):
        P = dict(wl.params, precision=1 if prec == "mixed" else 0)
        s = S.slab_solver(R, P, wl.prim, None, None, slab)
        st = S.SolverStepper(s)
        ex = S.DistExchange(st, nz, H, periodic)
        for _ in range(args.warmup):
            st.step(wl.dt)
            ex.exchange()
        torch.cuda.synchronize()
        dist.barrier()
        sampler = ClockSampler(local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with sampler:
            torch.cuda.synchronize()
            e0.record()
            for _ in range(args.steps):
                st.step(wl.dt)
                ex.exchange()
            e1.record()
            torch.cuda.synchronize()
        ms = reduce_max_ms(e0.elapsed_time(e1), world, "cuda")
        # end to end through the public API, host buffers
        prim_h = torch.empty((14,) + s.shape, dtype=torch.float64).pin_memory().numpy()
        s.get_prims(prim_h)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ke = max(1, min(args.steps, 3))
        for _ in range(ke):
            s.set_prims(prim_h)
            st.step(wl.dt)
            ex.exchange()
            s.get_prims(prim_h)
        torch.cuda.synchronize()
        e2e_ms = reduce_max_ms(1e3 * (time.perf_counter() - t0), world, "cuda")
        out[prec] = dict(ms=ms, clocks=sampler.summary(), e2e_ms=e2e_ms, e2e_steps=ke,
                         slab_bytes=14 * 8 * int(np.prod(s.shape)),
                         halo=H, local_layers=slab.nz_local, owned_layers=slab.z1 - slab.z0)
        s.close()
    dist.destroy_process_group()
    return wl, out


def kernel_rooflines(wl, res, prec, steps):
    """Roofline of every kernel group from its live CUDA-event time."""
    hbm, kind = _peaks()
    g = res["groups"]
    N = wl.ncells
    nd = sum(1 for d in range(3) if wl.params["n"][d] > 1)
    imex = wl.params.get("imex", 0)
    rows, _, nflux = IMEX_ROWS[imex]
    # launches per step of each group: the stage-row group runs one recovery
    # kernel per row, the flux group of the stages one pass per formed F
    # before the last
    per_step = {"stage2_rhs_recovery": len(rows), "flux_stage2": nd * (nflux - 1),
                "flux_final": nd}
    out = {}
    for name, ms in g.items():
        if name == "ghost_fill" or ms <= 0.0:
            continue
        if name.startswith("flux"):
            per_launch_ms = ms / steps / per_step[name]   # one direction per launch
            faces = N                                 # ~one face per cell per direction
            if prec == "fp64":
                # the FP64 face kernel is bound by the FP64 pipe, not by HBM
                fl = FLUX_FLOPS_PER_FACE_BY_RECON[wl.params["recon"]] * faces
                ach = fl / (per_launch_ms * 1e-3) / 1e12
                out[name] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                             "peak_kind": "derived (148 SM x 2 DFMA/clk x 2.032 GHz)",
                             "launch_ms": per_launch_ms, "alg_fp64_flops_per_launch": fl,
                             "alg_bytes_per_launch": FLUX_FIELDS * 8 * faces}
                continue
            alg = FLUX_FIELDS * 4 * faces
            ach = alg / (per_launch_ms * 1e-3) / 1e9
            out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "peak_kind": kind, "launch_ms": per_launch_ms,
                         "alg_bytes_per_launch": alg,
                         "alg_flops_per_face": FLUX_FLOPS_PER_FACE_BY_RECON[wl.params["recon"]]}
        else:
            per_launch_ms = ms / steps / per_step.get(name, 1)
            f = fp64_flops(name, prec, res["iters"], imex) * N
            ach = f / (per_launch_ms * 1e-3) / 1e12
            out[name] = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                         "peak_kind": "derived (148 SM x 2 DFMA/clk x 2.032 GHz; measured "
                                      "1.111 TFLOP/s FP64 FMA at 1.94 GHz)",
                         "launch_ms": per_launch_ms, "alg_fp64_flops_per_launch": f,
                         "paper_iterations_per_recovery": res["iters"]}
    return out


# Pipe counters of the recovery kernels from one ncu capture of a 128^3
# launch of this workload (--set full): FP64-pipe cycles active and lane
# efficiency (threads per warp instruction / 32).  The FP64 pipe also runs
# what the algorithmic count leaves out (the Newton steps of divisions and
# square roots, compares, float <-> double conversions), so the pipe is near
# its limit while the algorithmic fraction reads lower.  Valid for the
# kernels as they are; re-measure after changing one.
NCU_PIPES = {
    ("stage1_recovery", "mixed"): {"fp64_pipe_busy": 0.7837, "lane_efficiency": 28.10 / 32,
                                   "source": "ncu --metrics, 128^3 launch of this workload"},
    ("stage2_rhs_recovery", "mixed"): {"fp64_pipe_busy": 0.7595, "lane_efficiency": 28.48 / 32,
                                       "source": "ncu --set full, 128^3 launch of this workload"},
    ("final_rhs_recovery", "mixed"): {"fp64_pipe_busy": 0.6589, "lane_efficiency": 30.90 / 32,
                                      "source": "ncu --metrics, 128^3 launch of this workload"},
}


def roofline(wl, res, prec, steps):
    ks = kernel_rooflines(wl, res, prec, steps)
    g = res["groups"]
    name = max((k for k in g if k != "ghost_fill"), key=g.get)
    r = dict(ks[name])
    r["kernel"] = name
    per_cell = TRAFFIC_PER_CELL.get((name, prec))
    r["traffic"] = None if per_cell is None else per_cell * wl.ncells
    r["traffic_unit"] = "bytes per launch (ncu, 128^3 launch scaled by cells)"
    if (name, prec) in NCU_PIPES and wl.params.get("imex", 0) == 0:
        r["ncu_pipes"] = dict(NCU_PIPES[(name, prec)])
    return r, ks


# Adjoint (gradient of a loss of the primitives after K steps with respect to
# the initial primitives and log sigma0) on the 128^3 Alfven cube (WENO5):
# algorithmic FP64 work of one face-flux adjoint taken as 3x the forward face
# work (the cheap-gradient bound of reverse mode), per face of each direction
# and stage.
ADJ_FLOPS_PER_FACE = 3 * FLUX_FLOPS_PER_FACE_BY_RECON[2]


def run_adjoint(args):
    import torch
    import paper_2510_18968_b300 as R
    n, K, every = args.adjoint_n, args.adjoint_steps, args.adjoint_every
    wl = W.alfven_diag(n=n, sigma=1e3)
    dx = wl.params["dx"]
    dV = dx[0] * dx[1] * dx[2]
    prim0 = np.ascontiguousarray(wl.prim)
    s = R.Solver(dict(wl.params, sigma0=2e3))
    s.set_prims(prim0)
    s.step(wl.dt, K)
    target = s.get_prims()[9].copy()
    s.close()
    s = R.Solver(wl.params)
    s.set_prims(prim0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.adjoint_forward(wl.dt, K, every)
    torch.cuda.synchronize()
    t_f = time.perf_counter() - t0
    PN = s.get_prims()
    lam = np.zeros_like(PN)
    lam[9] = 2.0 * (PN[9] - target) * dV
    loss = float(np.sum((PN[9] - target) ** 2) * dV)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grad, gls, groups = s.adjoint_backward(lam, profile=True)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    s.close()
    # the same gradient with the whole tape in HBM (no re-runs)
    s = R.Solver(wl.params)
    s.set_prims(prim0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.adjoint_forward(wl.dt, K, 0)
    torch.cuda.synchronize()
    t_f0 = time.perf_counter() - t0
    t0 = time.perf_counter()
    grad0, gls0, groups0 = s.adjoint_backward(lam, profile=True)
    torch.cuda.synchronize()
    t_b0 = time.perf_counter() - t0
    s.close()
    full_tape = {"forward_s": t_f0, "backward_s": t_b0, "kernel_ms": groups0,
                 "same_gradient": bool(np.array_equal(grad0, grad) and gls0 == gls)}
    N = wl.ncells
    nd = 3
    faces = nd * 2 * K * N          # faces of both stages of every step
    fl_ms = groups["adjoint_flux"]
    ach = ADJ_FLOPS_PER_FACE * faces / (fl_ms * 1e-3) / 1e12
    return {"workload": f"alfven_diag {n}^3 (WENO5+HLLE, sigma0=1e3, Gamma=4/3, periodic), "
                        f"{K} steps, checkpoints every {every}; loss = sum (B^y - B^y[sigma0="
                        f"2e3])^2 dx^3",
            "value": N * K / (t_f + t_b), "unit": "zone-updates/s (forward + gradient)",
            "forward_s": t_f, "backward_s": t_b, "backward_over_forward": t_b / t_f,
            "loss": loss, "dL_dlog_sigma0": gls, "grad_max": float(np.abs(grad).max()),
            "kernel_ms": groups, "full_tape": full_tape,
            "roofline": {"kernel": "k_adj_flux", "bound": "alu", "achieved": ach,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS,
                         "alg_fp64_flops_per_face": ADJ_FLOPS_PER_FACE,
                         "launch_ms": fl_ms / (nd * 2 * K), "traffic": None}}


def run_configs(args):
    """The other configurations: the 400-cell Brio-Wu shocktube (launch-bound:
    latency per step, one CUDA-graph replay per step against one launch
    sequence per step), the 128^3 Alfven cube and the 192^3 curved star
    (zone-updates/s of both paths, recovery statistics), and the 256^3 blast
    with each of the paper's IMEX schemes."""
    import torch
    import paper_2510_18968_b300 as R
    out = {}

    def timed(s, dt, k, graph=True):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        e0.record(st)
        if graph:
            s.step(dt, k, sync=False)
        else:
            for _ in range(k):
                s.step(dt, 1, sync=False)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    wl = W.brio_wu(n=400)
    s = R.Solver(wl.params)
    s.set_prims(np.ascontiguousarray(wl.prim))
    s.step(wl.dt, 20)
    ms_g = timed(s, wl.dt, 300)
    ms_l = timed(s, wl.dt, 300, graph=False)
    s.close()
    out["brio_wu_400"] = {"workload": "Brio-Wu 400 cells, minmod+HLLE, sigma=1e5, FP64",
                          "ms_per_step_graph": ms_g / 300, "ms_per_step_launches": ms_l / 300}
    for name, make in (("alfven_128", lambda: W.alfven_diag(n=128, sigma=1e4)),
                       ("lane_emden_192", lambda: W.lane_emden_star(n=192))):
        wl = make()
        d = {}
        for prec in ("mixed", "fp64"):
            s = R.Solver(dict(wl.params, precision=1 if prec == "mixed" else 0))
            if wl.alpha is not None:
                a, b, g, K = wl.metric_arrays()
                s.set_metric(np.ascontiguousarray(a), np.ascontiguousarray(b),
                             np.ascontiguousarray(g), np.ascontiguousarray(K))
            if wl.sigma_profile is not None:
                s.set_sigma(np.ascontiguousarray(wl.sigma_profile))
            s.set_prims(np.ascontiguousarray(wl.prim))
            s.step(wl.dt, 3)
            ms = timed(s, wl.dt, 10)
            st = s.stats()
            s.close()
            d[prec] = {"value": wl.ncells * 10 / (ms * 1e-3), "ms_per_step": ms / 10,
                       "paper_iterations_per_recovery": st["c2p_iterations"] / st["c2p_calls"],
                       "fallbacks": st["c2p_fallbacks"], "atmosphere_resets":
                       st["c2p_failures"] + st["atmo_floor_resets"]}
        d["unit"] = UNIT
        d["mixed_speedup"] = d["fp64"]["ms_per_step"] / d["mixed"]["ms_per_step"]
        out[name] = d
    # the paper's four IMEX schemes on the 256^3 blast (one more implicit
    # stage and face-flux evaluation than Table imex for the other three)
    wl = W.cyl_blast(n=256)
    d = {"workload": "cylindrical blast 256^3 (the headline workload), per IMEX scheme",
         "unit": UNIT}
    for scheme, label in ((0, "SSP2(2,2,2)"), (1, "SSP2(3,3,2)"), (2, "SSP3(3,3,2)"),
                          (3, "SSP3(4,3,3)")):
        e = {}
        wl.params["imex"] = scheme
        for prec in ("mixed", "fp64"):
            s = R.Solver(dict(wl.params, precision=1 if prec == "mixed" else 0))
            s.set_prims(np.ascontiguousarray(wl.prim))
            s.step(wl.dt, 3)
            ms = timed(s, wl.dt, 10)
            # kernel groups of three more steps (events between the groups)
            st0 = s.stats()
            groups = s.step_profiled(wl.dt, 3)
            st = s.stats()
            s.close()
            iters = ((st["c2p_iterations"] - st0["c2p_iterations"]) /
                     max(1, st["c2p_calls"] - st0["c2p_calls"]))
            ks = kernel_rooflines(wl, {"groups": groups, "iters": iters}, prec, 3)
            top = max((k for k in groups if k != "ghost_fill"), key=groups.get)
            e[prec] = {"value": wl.ncells * 10 / (ms * 1e-3), "ms_per_step": ms / 10,
                       "paper_iterations_per_recovery": iters,
                       "kernel_ms_per_step": {k: v / 3 for k, v in groups.items()},
                       "roofline": dict(ks[top], kernel=top)}
        d[label] = e
    out["imex_schemes_cyl_blast_256"] = d
    return out


def cpu_oracle_sample(nz, steps, imex=0):
    """The FP64 oracle on a z-slab (nz cells thick, same x-y plane and
    options) of the 256^3 workload; returns zone-updates/s and the sample."""
    import oracle
    wl = W.cyl_blast(n=256, nz=nz)
    wl.params["imex"] = imex
    a, b, g, K = wl.metric_arrays()
    m = oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(wl.params, m, prim)
    t0 = time.perf_counter()
    oracle.step(wl.params, m, cons, prim, wl.dt, steps)
    dt = time.perf_counter() - t0
    return wl.ncells * steps / dt, f"256x256x{nz} z-slab of the 256^3 workload, {steps} step(s)"


def _oracle_worker(nz, steps, barrier, out, imex=0):
    import oracle
    wl = W.cyl_blast(n=256, nz=nz)
    wl.params["imex"] = imex
    a, b, g, K = wl.metric_arrays()
    m = oracle.Metric(a.ravel(), b.reshape(3, -1), g.reshape(6, -1), K.reshape(6, -1))
    prim = np.ascontiguousarray(wl.prim.copy())
    cons = oracle.prim2con_grid(wl.params, m, prim)
    barrier.wait()
    t0 = time.perf_counter()
    oracle.step(wl.params, m, cons, prim, wl.dt, steps)
    out.put(wl.ncells * steps / (time.perf_counter() - t0))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_parallel(nz, steps, procs=None, imex=0):
    """The single-threaded FP64 oracle, unchanged, run as `procs` concurrent
    processes (spawned: the parent may hold a CUDA context), each on its own
    256 x 256 x nz z-slab of the 256^3 workload; they start together after
    set-up and the aggregate zone-updates/s is the sum of their rates."""
    import multiprocessing as mpr
    procs = procs or min(host_cores(), 64)
    ctx = mpr.get_context("spawn")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(nz, steps, barrier, out, imex))
          for _ in range(procs)]
    for p in ps:
        p.start()
    rates = [out.get() for _ in ps]
    for p in ps:
        p.join()
    return (sum(rates), procs, sum(rates) / procs,
            f"{procs} concurrent processes, each a 256x256x{nz} z-slab of the 256^3 workload, "
            f"{steps} step(s)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--no-run100", action="store_true",
                    help="skip the configuration's 100-step runs (short profiling runs)")
    ap.add_argument("--imex", type=int, default=0, choices=[0, 1, 2, 3],
                    help="IMEX scheme of the timed workload (0: SSP2(2,2,2), Table imex)")
    ap.add_argument("--adjoint-n", type=int, default=128)
    ap.add_argument("--adjoint-steps", type=int, default=60)
    ap.add_argument("--adjoint-every", type=int, default=10)
    args = ap.parse_args()
    rank, world, local = dist_env()
    cfg = {"workload": f"cyl_blast_{args.n}^3 (MC2+HLLE, sigma=1e3, Gamma=4/3, outflow, "
                       "dt=0.25 dx)", "grid": [args.n] * 3, "imex": IMEX_LABELS[args.imex],
           "l2": "inputs larger than L2 (state ~2 GB per array set)"}

    if args.impl == "reference":
        if rank != 0:
            return
        cpu_oracle_sample(2, 1, args.imex)   # warm-up: page in the oracle and its inputs
        vals = []
        for _ in range(args.steps):
            v, cores, per_core, sample = cpu_oracle_parallel(2, 1, imex=args.imex)
            vals.append(v)
        value = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * 256 ** 3 / value,
                "ms_per_step_kind": "extrapolated: 256^3 cells / the measured aggregate "
                                    "zone-update rate of the z-slab samples",
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "per_core": per_core, "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        wl, res = run_slabs(args, rank, world, local)
        if rank != 0:
            return
        head = "mixed" if "mixed" in res else "fp64"
        r = res[head]
        N = wl.ncells
        line = {"metric": METRIC, "value": N * args.steps / (r["ms"] * 1e-3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None,
                "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
                "config": dict(cfg, precision=head, parallelism=f"z-slabs x{world}",
                               halo_layers=r["halo"], local_layers=r["local_layers"],
                               owned_layers_rank0=r["owned_layers"],
                               timed_call="rmhd_step (one step) + halo exchange (NCCL "
                                          "point to point) per step")}
        if "fp64" in res and head != "fp64":
            line["fp64_value"] = N * args.steps / (res["fp64"]["ms"] * 1e-3)
            line["fp64_ms_per_step"] = res["fp64"]["ms"] / args.steps
        line["clocks"] = r["clocks"]
        line["e2e"] = {"value": N * r["e2e_steps"] / (r["e2e_ms"] * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": r["slab_bytes"] * world,
                       "d2h_bytes_per_step": r["slab_bytes"] * world,
                       "pipeline": "per rank: rmhd_set_prims of its slab from pinned memory, "
                                   "one step + exchange, rmhd_get_prims"}
        line["gpu_launches"] = (launches_per_step(wl) + 6) * args.steps
        print(json.dumps(line))
        return

    wl, res = run_ours(args, rank, world, local)
    if rank != 0:
        return
    head = "mixed" if "mixed" in res else "fp64"
    r = res[head]
    r["steps"] = args.steps
    N = wl.ncells
    value = job_value(N, args.steps, world, r["ms"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
            "config": dict(cfg, precision=head, parallelism=f"replicas x{world}",
                           timed_call="rmhd_step (CUDA-graph replay)",
                           window=f"steps {window_start(args) + 1}-"
                                  f"{window_start(args) + args.steps} of the {RUN_STEPS}-step "
                                  f"run from the initial data (untimed before it: "
                                  f"{window_start(args)} steps, the {args.warmup} warm-up "
                                  f"steps among them)")}
    # the configuration's whole RUN_STEPS-step run from the initial data,
    # both precisions (the cost per step grows as the blast evolves, so a
    # short early window overstates the run's mean rate)
    for prec, rr in res.items():
        run = rr["run"]
        key = "run100" if prec == head else f"{prec}_run100"
        line[key] = dict(value=job_value(N, run["steps"], world, run["ms"]),
                         ms_per_step=run["ms"] / run["steps"], unit=UNIT, precision=prec,
                         **{k: v for k, v in run.items() if k != "ms"})
    if "fp64" in res and head != "fp64":
        f = res["fp64"]
        line["fp64_value"] = job_value(N, args.steps, world, f["ms"])
        line["fp64_ms_per_step"] = f["ms"] / args.steps
        line["fp64"] = {"value": line["fp64_value"], "ms_per_step": line["fp64_ms_per_step"],
                        "mixed_speedup": f["ms"] / r["ms"],
                        "mixed_speedup_run100": f["run"]["ms"] / r["run"]["ms"]}
    line["roofline"], line["roofline_kernels"] = roofline(wl, r, head, args.steps)
    # the whole step against the compulsory state traffic of a fully fused
    # step (904 B per zone-update mixed, 1200 B FP64, flat metric)
    hbm, kind = _peaks()
    alg_b = ALG_BYTES_PER_ZONE[head]
    line["roofline"]["e2e_hbm_frac"] = alg_b * N * args.steps / (r["ms"] * 1e-3) / 1e9 / hbm
    line["roofline"]["e2e_hbm_frac_run100"] = (alg_b * N * r["run"]["steps"] / (r["run"]["ms"] * 1e-3)
                                               / 1e9 / hbm)
    line["roofline"]["e2e_alg_bytes_per_zone"] = alg_b
    line["roofline"]["kernel_timing"] = ("rmhd_step_profiled over the same window from the "
                                         "same state (events between kernel groups)")
    line["kernel_ms_per_step"] = {k: v / args.steps for k, v in r["groups"].items()}
    if "fp64" in res and head != "fp64":
        line["fp64"]["kernel_ms_per_step"] = {k: v / args.steps
                                             for k, v in res["fp64"]["groups"].items()}
        line["fp64"]["roofline_kernels"] = kernel_rooflines(wl, res["fp64"], "fp64", args.steps)
    line["recovery_stats"] = r["stats"]
    line["clocks"] = r["clocks"]
    line["e2e"] = {"value": world * r["e2e"], "unit": UNIT,
                   "h2d_bytes_per_step": r["e2e_bytes"][0], "d2h_bytes_per_step": r["e2e_bytes"][1],
                   "pipeline": "independent one-step jobs on 3 handles (own CUDA streams, own "
                               "host threads, staggered by one upload); per job: rmhd_set_prims "
                               "from pinned memory, step, rmhd_get_prims",
                   "serial_value": world * r["e2e_serial"],
                   "state_upload_value": world * r["e2e_state"],
                   "state_upload_handles": 2}
    # kernel launches inside the timed region, per step: three recovery
    # kernels and their deferred passes, ghost fills (primitives, and stage
    # currents when the charge flux uses them), one flux kernel per active
    # direction and stage
    line["gpu_launches"] = launches_per_step(wl) * args.steps
    if not args.no_adjoint:
        line["adjoint"] = run_adjoint(args)
    if not args.no_configs:
        line["configs"] = run_configs(args)
    if not args.no_cpu_baseline:
        v, cores, per_core, sample = cpu_oracle_parallel(2, 1, imex=args.imex)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "per_core": per_core, "sample": sample}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
