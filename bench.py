"""Throughput of the radiation step (transport + implicit source) on GB300.

Headline workload: the radiation-modified linear waves box at scale
(Sec. 3.6 setup): 256^3 jittered periodic Voronoi cells, 80 discrete
ordinates (S8), cell optical depth 1, cbar = 100, c = 1e4, a 1e-6 sinusoidal
temperature / radiation-energy perturbation along x (seeded, synthetic).
One "step" is one rt_step: the fused transport + source kernel over every
cell and angle.  Reported: cell-angle updates/s of the FP32 path (headline)
and of the FP64 path, each against the roofline of its algorithmic bytes or
flops; an end-to-end figure through the C ABI with host buffers; and the
CPU oracle timed on this host's cores (all of them and one).  The 128^3
shadows / crossing-beams box is timed beside it, with the van Leer,
adjoint, frequency-group and launch-bound thermal legs on the shadows box.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (the step has no cross-GPU exchange here); the
value is the sum over ranks divided by the slowest rank's time.
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-angle updates/s (transport+implicit source), FP32 vs FP64, % HBM roofline"
UNIT = "cell-angle updates/s"

# DRAM bytes (read + write) per launch of the step kernels, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, one launch, one
# pass); valid while the step kernel's device source has the recorded hash
# (else reported as null).  FP32: the 256^3 linear-wave launch itself
# (12.42 GB read + 6.15 GB written).  FP64: the 128^3 linear-wave launch
# (12.52 + 1.49 GB, mostly the flux-coefficient table) scaled by the cell
# count to 256^3 (the table, the rows and the gas all grow with the cells),
# taken when only the float instantiations' code differed from today's.
NCU_TRAFFIC = {("waves", 16777216, "fp32"): 18.57e9,
               ("waves", 16777216, "fp64"): 14.01e9 * 8}
NCU_SOURCE_SHA = "3210b6995f7435eb"
# FP64 arithmetic peak when the DGEMM probe cannot run: the nominal dense
# FP64 FMA rate of the GPU.
FP64_NOMINAL_GFLOPS = 1250.0


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("rt_step.cu", "rt_step_common.cuh", "rt_step_tile.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2002_08377_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_fp64_flops(n_cells, n_faces, n_angles):
    """Floating-point operations the FP64 step must do: per directed face and
    angle 2 (the upwind product and sum; the flux coefficients n_a . n_f cbar A_f
    are fixed for the mesh and tabulated once per state), per cell and angle 2
    for the update and 27 for the comoving source step."""
    directed = 2.0 * n_faces
    return 2.0 * directed * n_angles + 29.0 * n_cells * n_angles


def algorithmic_bytes(n_cells, n_faces, n_angles, real_bytes):
    """Bytes the method must move per step: one read and one write of every
    intensity, the per-cell gas state (V, rho, kappa_P, kappa_J, kappa_s, e,
    m, v read: 72 B; e, m written: 32 B) and every undirected face once
    (two int32 cell ids, A n (3 reals), A w.n (1 real)).  FP64 states also
    read their flux-coefficient table: A/2 doubles per directed face."""
    b = n_cells * (2 * real_bytes * n_angles + 104) + n_faces * (8 + 4 * real_bytes)
    if real_bytes == 8:
        b += 2 * n_faces * (n_angles // 2) * 8
    return b


def algorithmic_bytes_vl(n_cells, n_faces, n_angles, real_bytes):
    """Bytes one van Leer step must move: stage 1 is a first-order step over
    dt/2 (algorithmic_bytes); the gradient pass reads the stage-1 row of
    every cell, its face records (8 reals per directed face, the neighbour
    index inside) and the 8 reals of the inverse normal matrix, and writes
    three gradient rows; the reconstructed transport reads I^n, the stage-1
    row and its gradient rows, the face records again and the face slots
    (16 bytes per directed face for float states, the n_p . s table for
    double), and writes I*; the source-only stage reads I* and the gas and
    writes I^{n+1} and the gas."""
    s, N, F, A = real_bytes, n_cells, n_faces, n_angles
    stage1 = algorithmic_bytes(N, F, A, s)
    records = 2 * F * 8 * s
    slots = 2 * F * (16 if s == 4 else 8 * (A // 2))
    gradient = N * A * s * (1 + 3) + records + 8 * s * N
    transport = N * A * s * (1 + 1 + 3 + 1) + records + slots + N * s
    source = N * (2 * A * s + 104)
    return stage1 + gradient + transport + source


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and clock-event reasons during the timed region, via NVML
    (read-only queries) every few milliseconds."""
    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index=0, period=0.005):
        self.ok = False
        self.samples = []
        self.reasons = 0
        self.period = period
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            assert nv.nvmlInit_v2() == 0
            h = ctypes.c_void_p()
            assert nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) == 0
            mx = ctypes.c_uint()
            nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM = 1
            self.nv, self.h, self.max_mhz = nv, h, mx.value
            fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self.reason_fn = fn
            self.ok = True
        except Exception:
            self.max_mhz = None

    def _loop(self):
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                self.samples.append(clk.value)
            if self.reason_fn(self.h, ctypes.byref(rs)) == 0:
                self.reasons |= rs.value
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self._stop = threading.Event()
            self._t = threading.Thread(target=self._loop, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self._t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"]}
        names = [n for bit, n in self.REASONS.items() if self.reasons & bit and n != "gpu_idle"]
        return {"sm_mhz": float(statistics.median(self.samples)), "sm_max_mhz": self.max_mhz,
                "samples": len(self.samples), "reasons": names}


# ---------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world):
    """Largest x over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ms_per_rank, world):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time (weak scaling: every rank runs its own replica)."""
    ms = max_over_ranks(ms_per_rank, world)
    return units_per_rank * world / (ms * 1e-3), ms


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- workload
def make_workload(name="waves", n=None):
    from paper_2002_08377_gb300.inputs import shadows, waves
    if name == "waves":
        return waves(n=256 if n is None else n)
    return shadows(n=128 if n is None else n)


def describe(prob):
    n = prob.mesh.n[0]
    base = {"cells": prob.n_cells, "angles": prob.n_angles, "faces": prob.mesh.n_faces,
            "directed_faces_per_cell": round(2 * prob.mesh.n_faces / prob.n_cells, 3),
            "l2": "inputs larger than L2 (129 MB): intensities 2 x "
                  f"{prob.n_cells * prob.n_angles * 4 / 1e6:.0f} MB (FP32) + face slots"}
    if prob.name == "waves":
        base["workload"] = (f"radiation-modified linear waves at scale: {n}^3 jittered periodic "
                            "Voronoi cells, 80 level-symmetric angles (S8), cell optical depth 1, "
                            "cbar = 100, c = 1e4, 1e-6 sinusoidal T / E_r perturbation along x")
    else:
        base["workload"] = (f"shadows/crossing-beams box: {n}^3 jittered periodic Voronoi cells, "
                            "80 level-symmetric angles, 3 opaque spheres, 4 emitters, absorbing "
                            "layers, 2 beams, cbar = c = 1e3")
    return base


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(o, dt, budget_s, chunk):
    """Cell-angle updates/s of the FP64 oracle `o` on consecutive ranges of
    `chunk` cells of its workload (transport + source of those cells from
    the full state), until budget_s passes."""
    N, A = o.N, o.A
    done, t0 = 0, time.perf_counter()
    out = np.empty_like(o.I)
    c0 = 0
    while True:
        c1 = min(N, c0 + chunk)
        st, _ = o.sample_step(dt, c0, c1, out)
        if st != 0:
            raise RuntimeError(f"oracle step failed ({st})")
        done += (c1 - c0) * A
        c0 = 0 if c1 >= N else c1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return done / el, done, el


def mem_available():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) << 10
    except OSError:
        pass
    return None


def cpu_baseline(prob, dt, budget_s):
    """The oracle on all host cores and on one core, on bounded samples of
    the workload (ranges of cells of one step)."""
    import oracle
    # the oracle's state: two [N][A] double arrays, the face offsets and its
    # copies of the mesh arrays
    need = 2 * prob.n_cells * prob.n_angles * 8 + prob.mesh.n_faces * 120
    avail = mem_available()
    if avail is not None and avail < 1.3 * need:
        return {"unavailable": f"host memory: {avail >> 30} GB available, the oracle state of "
                               f"this workload needs about {need >> 30} GB"}
    o = oracle.Oracle(prob)
    N, A = o.N, o.A
    cores = oracle.set_threads(0)
    chunk = max(1, min(N, 1 << 18))
    v, done, el = cpu_oracle_rate(o, dt, budget_s, chunk)
    oracle.set_threads(1)
    v1, done1, el1 = cpu_oracle_rate(o, dt, max(2.0, budget_s / 3), max(1, chunk // 16))
    oracle.set_threads(cores)
    del o
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} cell-angle updates of the FP64 oracle ({el:.1f} s; ranges of "
                      f"{chunk} of the {N} cells x {A} angles of one step, transport + source)",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"{done1} cell-angle updates ({el1:.1f} s, ranges of "
                                      f"{max(1, chunk // 16)} cells)"}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    prob = make_workload(args.workload, args.n)
    dt = prob.cfl_dt()
    import oracle
    o = oracle.Oracle(prob)
    N, A = prob.n_cells, prob.n_angles
    sample = max(1, N // 64)  # each step: one sixty-fourth of the cells
    out = np.empty_like(o.I)
    for _ in range(args.warmup):
        o.sample_step(dt, 0, sample, out)
    t0 = time.perf_counter()
    for k in range(args.steps):
        c0 = (k * sample) % N
        o.sample_step(dt, c0, min(N, c0 + sample), out)
    el = time.perf_counter() - t0
    v = sample * A * args.steps / el
    cores = oracle.set_threads(0)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": describe(prob),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"cells [c0, c0+{sample}) of one step per timed step "
                                       f"(1/64 of the {N}-cell, {A}-angle workload)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
GRAPH_STEPS = 16  # RT_GRAPH_STEPS of include/rt.h


def warm_up(sol, dt, warmup):
    """warmup single steps, then two multi-step runs an odd step apart: these
    capture the step graphs of both buffer parities (rt_run / rt_launch
    replay them for every whole block of GRAPH_STEPS steps), so that no
    capture falls inside a timed region."""
    for _ in range(warmup):
        sol.step(dt)
    sol.run(GRAPH_STEPS, dt)
    sol.step(dt)
    sol.run(GRAPH_STEPS, dt)


def time_steps(sol, dt, steps, warmup, world, sampler=None):
    import torch
    warm_up(sol, dt, warmup)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stream = sol.stream
    l0 = sol.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    ctx = sampler if sampler is not None else _Null()
    with ctx:
        ev0.record(stream)
        sol.launch(steps, dt)  # back-to-back launches on the solver's stream
        ev1.record(stream)
        torch.cuda.synchronize()
    sol.sync()  # latched per-cell status of the timed steps
    barrier(world)
    launches = sol.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    return max_over_ranks(ms, world), launches


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


def e2e_rate(sol, prob, dt, steps, pipelined=True):
    """Through the C ABI with pinned host buffers: every step copies the
    intensities in, runs the step and copies them out.  pipelined: rt_step_io
    (the host copies run on the copy engines and overlap the neighbouring
    steps' GPU work), two output buffers in turn; otherwise rt_set_intensity,
    rt_step, rt_get_intensity, each synchronous."""
    import torch
    N, A = prob.n_cells, prob.n_angles
    host_in = torch.empty((N, A), dtype=torch.float32, pin_memory=True)
    host_in.numpy()[:] = prob.initial_intensity(np.float32)
    outs = [torch.empty((N, A), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    lib, st = sol.lib, sol.state
    pin = ctypes.c_void_p(host_in.data_ptr())
    pouts = [ctypes.c_void_p(o.data_ptr()) for o in outs]
    used = ctypes.c_double()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if pipelined:
        for k in range(steps):
            sol._check(lib.rt_step_io(st, dt, pin, pouts[k % 2]))
        sol._check(lib.rt_sync(st))
    else:
        for _ in range(steps):
            sol._check(lib.rt_set_intensity(st, pin, 0))
            sol._check(lib.rt_step(st, dt, ctypes.byref(used)))
            sol._check(lib.rt_get_intensity(st, pouts[0], 0))
    el = time.perf_counter() - t0
    nbytes = N * A * 4
    return N * A * steps / el, nbytes, nbytes


def groups_workload(n):
    """The shadows box on S6 with two frequency groups (96 angles in all):
    group 0 with 0.3 times and group 1 with 3 times the cells' opacities,
    group weights 0.4, 0.6, the intensities and boundary rows copied per
    group."""
    from paper_2002_08377_gb300.inputs import shadows
    prob = shadows(n=n, order=6)
    G = 2
    prob.n_groups = G
    prob.group_w = np.array([0.4, 0.6])
    sc = np.array([0.3, 3.0])
    for k in ("kappa_P", "kappa_J", "kappa_s"):
        setattr(prob, k, np.ascontiguousarray(getattr(prob, k)[:, None] * sc[None, :]))
    I = prob.initial_intensity()
    Ig = np.ascontiguousarray(np.concatenate([I, I], axis=1))
    prob.initial_intensity = lambda dtype=np.float64, _I=Ig: np.ascontiguousarray(_I.astype(dtype))
    prob.I0 = np.ascontiguousarray(np.tile(prob.I0, (1, G)))
    return prob


def groups_rate(n, steps, warmup, hbm_peak, peak_kind):
    """Steps of the two-group S6 shadows box (FP32): the transport sweep of
    all 96 angles, then the coupled source step."""
    import torch
    from paper_2002_08377_gb300.solver import RTSolver
    prob = groups_workload(n)
    N, Nf = prob.n_cells, prob.mesh.n_faces
    A = prob.n_groups * prob.n_angles
    dt = prob.cfl_dt()
    sol = RTSolver.from_problem(prob, "fp32")
    warm_up(sol, dt, warmup)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = sol.launch_count()
    ev0.record(sol.stream)
    sol.launch(steps, dt)
    ev1.record(sol.stream)
    torch.cuda.synchronize()
    sol.sync()
    ms = ev0.elapsed_time(ev1)
    launches = sol.launch_count() - l0
    sol.close()
    del sol
    torch.cuda.empty_cache()
    per = ms / steps
    # the grey byte model with all groups' intensities, plus 2 x 3 group opacities per cell
    B = algorithmic_bytes(N, Nf, A, 4) + N * 6 * 8
    achieved = B / (per * 1e-3) / 1e9
    return {"value": N * A * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": per, "steps": steps,
            "launches": launches, "dtype": "f32", "groups": prob.n_groups, "angles": A,
            "workload": "the shadows box on S6 with 2 frequency groups (96 angles)",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "algorithmic_bytes_per_step": B,
                         "peak_source": f"{peak_kind} HBM copy bandwidth"}}


def thermal_rate(world):
    """The thermal-equilibrium box (16^3 cells, S6, 100 steps; 4096 x 48
    intensities, 0.8 MB in FP32): a launch-bound case, timed as 100 steps
    through rt_launch with the step graphs replayed (6 replays of 16 steps,
    then 4 single launches) and with plain launches of the same kernels."""
    import torch
    from paper_2002_08377_gb300.inputs import thermal
    from paper_2002_08377_gb300.solver import RTSolver
    prob = thermal()
    N, A, steps = prob.n_cells, prob.n_angles, prob.n_steps
    dt = prob.cfl_dt()
    out = {"workload": f"thermal box: {N} cells x {A} angles, {steps} steps", "steps": steps}
    for prec in ("fp32", "fp64"):
        for plain in (0, 1):
            sol = RTSolver.from_problem(prob, prec, plain_launches=plain)
            ms, launches = time_steps(sol, dt, steps, 3, world)
            sol.close()
            key = f"{prec}_{'plain' if plain else 'graphs'}"
            out[key] = {"ms_per_step": ms / steps, "value": N * A * steps / (ms * 1e-3),
                        "launches": launches}
    out["value"] = out["fp32_graphs"]["value"]
    out["unit"] = UNIT
    return out


def adjoint_rate(prob, prec, dt, steps, warmup):
    """Reverse steps through rt_adjoint_step (the solver's call, caller-order
    device tensors, seeded cotangents): cell-angle reversals per second."""
    import torch
    from paper_2002_08377_gb300.solver import RTSolver
    sol = RTSolver.from_problem(prob, prec)
    N, A = prob.n_cells, prob.n_angles
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    I = sol.get_intensity(device=True)
    e, m = sol.gas_device()
    lI1 = torch.rand(N, A, dtype=sol.tdtype, device="cuda", generator=g)
    le1 = torch.rand(N, dtype=torch.float64, device="cuda", generator=g)
    lm1 = torch.rand(N, 3, dtype=torch.float64, device="cuda", generator=g)
    gP = torch.zeros(N, dtype=torch.float64, device="cuda")
    gJ = torch.zeros_like(gP)
    for _ in range(warmup):
        sol.adjoint_step(dt, I, e, m, lI1, le1, lm1, gP, gJ)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = sol.launch_count()
    ev0.record(sol.stream)
    for _ in range(steps):
        sol.adjoint_step(dt, I, e, m, lI1, le1, lm1, gP, gJ)
    ev1.record(sol.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = sol.launch_count() - l0
    sol.close()
    del sol
    torch.cuda.empty_cache()
    return {"value": N * A * steps / (ms * 1e-3), "unit": "cell-angle reversals/s",
            "ms_per_step": ms / steps, "steps": steps, "launches": launches,
            "dtype": "f32" if prec == "fp32" else "f64"}


def host_link_ceiling(n_bytes):
    """Plain copies of n_bytes between pinned host memory and the device
    (one cudaMemcpyAsync each way through torch), CUDA events, best of 3:
    the host-link rate an end-to-end step could at best reach."""
    import torch
    n = n_bytes // 4
    h = torch.empty(n, dtype=torch.float32, pin_memory=True)
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    best = {"h2d": 1e30, "d2h": 1e30}
    for _ in range(3):
        for k in ("h2d", "d2h"):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            if k == "h2d":
                d.copy_(h, non_blocking=True)
            else:
                h.copy_(d, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            best[k] = min(best[k], e0.elapsed_time(e1))
    # both directions at once, on two streams (what a pipelined step's copies
    # can share): wall time of the pair, best of 3
    h2 = torch.empty(n, dtype=torch.float32, pin_memory=True)
    d2 = torch.empty(n, dtype=torch.float32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    both = 1e30
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        both = min(both, (time.perf_counter() - t0) * 1e3)
    del h, d, h2, d2
    torch.cuda.empty_cache()
    out = {k: {"GB_per_s": 4 * n / (ms * 1e-3) / 1e9, "ms": ms, "bytes": 4 * n}
           for k, ms in best.items()}
    out["both_ways"] = {"GB_per_s": 8 * n / (both * 1e-3) / 1e9, "ms": both, "bytes": 8 * n,
                        "note": "one copy each way at the same time on two streams (wall time)"}
    return out


def fp64_peak_probe():
    """Measured FP64 arithmetic rate: cuBLAS DGEMM 8192^3 (2 N^3 flops), best
    of 3 after one warm-up, CUDA events.  The denominator of the FP64 step's
    ALU roofline (the nominal dense FP64 rate is 1.25 TFLOP/s)."""
    import torch
    n = 8192
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e9


def roofline(prec, N, Nf, A, per_ms, hbm_peak, peak_kind, fp64_peak, fp64_kind, traffic):
    """The roofline object of one precision's step kernel: HBM-bound for
    FP32 (algorithmic bytes / launch time), FP64-ALU-bound for FP64
    (algorithmic flops / launch time) with its HBM fraction beside."""
    rb = 4 if prec == "fp32" else 8
    B = algorithmic_bytes(N, Nf, A, rb)
    achieved = B / (per_ms * 1e-3) / 1e9
    if prec == "fp32":
        return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": B,
                "peak_source": f"{peak_kind} HBM copy bandwidth (of {peak_kind})"}
    F = algorithmic_fp64_flops(N, Nf, A)
    gf = F / (per_ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": gf, "peak": fp64_peak, "unit": "GFLOP/s",
            "frac": gf / fp64_peak, "traffic": traffic, "algorithmic_flops_per_launch": F,
            "peak_source": fp64_kind,
            "hbm": {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "algorithmic_bytes_per_launch": B}}


def time_workload(prob, precs, steps, warmup, world, hbm_peak, peak_kind, fp64_peak, fp64_kind,
                  sampler=None, e2e=False):
    """Both precisions' step on one workload: per precision the timed rate,
    its roofline and the state's device memory; with e2e, the end-to-end
    rate of the FP32 state through the C ABI with pinned host buffers."""
    import torch
    from paper_2002_08377_gb300.solver import RTSolver
    N, A, Nf = prob.n_cells, prob.n_angles, prob.mesh.n_faces
    dt = prob.cfl_dt()
    res = {}
    sha = kernel_source_sha()
    for key in precs:
        # "fp32_float_quartic": the FP32 state with the temperature solved in float
        prec = "fp64" if key == "fp64" else "fp32"
        sol = RTSolver.from_problem(prob, prec, float_quartic=int(key == "fp32_float_quartic"))
        k = steps if prec == "fp32" else max(3, steps // 5)
        ms, launches = time_steps(sol, dt, k, max(3, warmup), world,
                                  sampler if key == "fp32" else None)
        per = ms / k
        tr = NCU_TRAFFIC.get((prob.name, N, key)) if NCU_SOURCE_SHA == sha else None
        res[key] = {"value": N * A * k * world / (ms * 1e-3), "ms_per_step": per, "steps": k,
                    "launches": launches, "device_bytes": sol.device_bytes(),
                    "roofline": roofline(prec, N, Nf, A, per, hbm_peak, peak_kind, fp64_peak,
                                         fp64_kind, tr)}
        if key == "fp32" and e2e:
            # the pipelined loop over as many steps as the device-timed region
            # (its first input and last output copy are not overlapped); the
            # synchronous sequence over at most 10
            k_e2e, k_seq = max(3, steps), max(3, min(10, steps))
            e2e_rate(sol, prob, dt, 2)  # the copy streams, their events and staging arrays
            e2e_v, bi, bo = e2e_rate(sol, prob, dt, k_e2e)
            seq_v, _, _ = e2e_rate(sol, prob, dt, k_seq, pipelined=False)
            res["e2e"] = {"value": e2e_v * world, "unit": UNIT, "h2d_bytes_per_step": bi,
                          "d2h_bytes_per_step": bo, "steps": k_e2e,
                          "api": "rt_step_io (pinned host rows in and out every step, copied by "
                                 "the copy engines while the neighbouring steps run), then rt_sync",
                          "sequential": {"value": seq_v * world, "steps": k_seq,
                                         "api": "rt_set_intensity, rt_step, rt_get_intensity "
                                                "per step, each synchronous"}}
        sol.close()
        del sol
        torch.cuda.empty_cache()
    return res


def radhydro_rate(n, steps, warmup):
    """The linear-wave box (n^3, S8) with the gas dynamics on (FP32
    radiation, double hydro): rt_radhydro_step = one van Leer hydro step at
    the gas Courant step, then the radiation subcycled under it at its own
    Courant step.  Reports ms per hydro step alone and per radiation-hydro
    step (hydro + n_sub radiation steps)."""
    import torch
    from paper_2002_08377_gb300.inputs import waves
    from paper_2002_08377_gb300.solver import RTSolver
    prob = waves(n=n)
    sol = RTSolver.from_problem(prob, "fp32", hydro=1)
    dt_rad = prob.cfl_dt()
    dt = sol.hydro_dt(0.3)
    n_sub = int(np.ceil(dt / dt_rad))
    for _ in range(warmup):
        sol.radhydro_step(dt, n_sub)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(sol.stream)
    for _ in range(steps):
        sol.hydro_step(dt)
    ev[1].record(sol.stream)
    ev[2].record(sol.stream)
    for _ in range(steps):
        sol.radhydro_step(dt, n_sub)
    ev[3].record(sol.stream)
    torch.cuda.synchronize()
    out = {"workload": f"linear-wave box {n}^3 x 80 angles with the gas dynamics (FP32 radiation)",
           "n_sub": n_sub, "steps": steps, "cells": prob.n_cells, "faces": prob.mesh.n_faces,
           "hydro_ms_per_step": ev[0].elapsed_time(ev[1]) / steps,
           "radhydro_ms_per_step": ev[2].elapsed_time(ev[3]) / steps,
           "device_bytes": sol.device_bytes()}
    sol.close()
    del sol
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the shadows box and its van Leer / adjoint / group / thermal legs")
    ap.add_argument("--only", choices=["fp32", "fp64", "fp32_float_quartic"], default=None,
                    help="time one precision of one workload only (profiling runs)")
    ap.add_argument("--workload", choices=["waves", "shadows"], default="waves",
                    help="the headline workload (waves: the 256^3 linear-wave box)")
    ap.add_argument("--n", type=int, default=None,
                    help="lattice cells per axis of the headline workload (default: its full "
                         "size; smaller for profiler captures)")
    ap.add_argument("--shadows-n", type=int, default=128,
                    help="lattice cells per axis of the shadows box of the extra legs")
    args = ap.parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2002_08377_gb300 import build as rtbuild
    from paper_2002_08377_gb300.solver import RTSolver
    rtbuild.build()

    hbm_peak, peak_kind = measured_peaks()
    if args.only is not None:
        prob = make_workload(args.workload, args.n)
        r = time_workload(prob, (args.only,), args.steps, args.warmup, world, hbm_peak, peak_kind,
                          FP64_NOMINAL_GFLOPS, "nominal dense FP64 rate", None, False)[args.only]
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": r["value"], "unit": UNIT,
                              "ms_per_step": r["ms_per_step"], "dtype": args.only,
                              "config": describe(prob), "roofline": r["roofline"],
                              "device_bytes": r["device_bytes"],
                              "note": "single-precision profiling run"}), flush=True)
        return

    try:
        fp64_peak = fp64_peak_probe()
        fp64_kind = "measured cuBLAS DGEMM 8192^3 FP64 rate on this GPU (of measured)"
    except Exception as ex:  # no DGEMM: the nominal figure
        fp64_peak, fp64_kind = FP64_NOMINAL_GFLOPS, f"nominal dense FP64 rate ({ex})"

    sampler = ClockSampler(index=0)
    prob = make_workload(args.workload, args.n)
    N, A = prob.n_cells, prob.n_angles
    dt = prob.cfl_dt()
    head = time_workload(prob, ("fp32", "fp64", "fp32_float_quartic"), args.steps, args.warmup,
                         world, hbm_peak, peak_kind, fp64_peak, fp64_kind, sampler,
                         not args.no_e2e)
    link = None
    if not args.no_e2e:
        link = host_link_ceiling(N * A * 4)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(prob, dt, args.cpu_budget)
    head_cfg = describe(prob)
    del prob

    extras = None
    if not args.no_extras:
        sprob = make_workload("shadows", args.shadows_n)
        sN, sA, sNf = sprob.n_cells, sprob.n_angles, sprob.mesh.n_faces
        sdt = sprob.cfl_dt()
        sh = time_workload(sprob, ("fp32", "fp64"), args.steps, args.warmup, world, hbm_peak,
                           peak_kind, fp64_peak, fp64_kind)
        extras = {"config": describe(sprob), "fp32": sh["fp32"], "fp64": sh["fp64"]}
        # the van Leer integrator with limited linear reconstruction (FP32)
        sprob.integrator = 1
        sol = RTSolver.from_problem(sprob, "fp32")
        k = max(3, args.steps // 5)
        ms, launches = time_steps(sol, sdt, k, max(3, args.warmup), world)
        per = ms / k
        B = algorithmic_bytes_vl(sN, sNf, sA, 4)
        achieved = B / (per * 1e-3) / 1e9
        extras["van_leer"] = {
            "value": sN * sA * k * world / (ms * 1e-3), "ms_per_step": per, "steps": k,
            "launches": launches, "dtype": "f32",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "algorithmic_bytes_per_step": B,
                         "bytes_model": "first-order stage + gradient rows + reconstructed "
                                        "transport + source stage (algorithmic_bytes_vl)",
                         "peak_source": f"{peak_kind} HBM copy bandwidth"}}
        sol.close()
        del sol
        sprob.integrator = 0
        torch.cuda.empty_cache()
        # one reverse step (rt_adjoint_step: forward transport sweep, source
        # reverse, transposed sweep, caller-order permutes) per timed step
        adj = {}
        for prec in ("fp32", "fp64"):
            k = max(3, args.steps // 10) if prec == "fp32" else 3
            r = adjoint_rate(sprob, prec, sdt, k, 2)
            r["over_forward_step"] = r["ms_per_step"] / sh[prec]["ms_per_step"]
            adj[prec] = r
        extras["adjoint"] = adj
        del sprob
        extras["groups"] = groups_rate(args.shadows_n, max(3, args.steps // 5), 3, hbm_peak,
                                       peak_kind)
        extras["thermal"] = thermal_rate(world)
        extras["radhydro"] = radhydro_rate(args.shadows_n, 3, 1)

    r32, r64 = head["fp32"], head["fp64"]
    line = {"metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world,
            "steps": r32["steps"], "warmup": max(3, args.warmup), "ms_per_step": r32["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": head_cfg, "roofline": r32["roofline"],
            "cpu_baseline": cpu, "e2e": head.get("e2e"), "host_link": link,
            "gpu_launches": r32["launches"], "device_bytes": r32["device_bytes"],
            "clocks": sampler.summary(),
            "fp32_float_quartic": {
                "value": head["fp32_float_quartic"]["value"],
                "ms_per_step": head["fp32_float_quartic"]["ms_per_step"],
                "frac": head["fp32_float_quartic"]["roofline"]["frac"],
                "note": "the FP32 state with float_quartic = 1 (temperature solved in float in "
                        "every lane); the headline solves it in double"},
            "fp64": {"value": r64["value"], "ms_per_step": r64["ms_per_step"],
                     "steps": r64["steps"], "dtype": "f64", "launches": r64["launches"],
                     "device_bytes": r64["device_bytes"], "roofline": r64["roofline"],
                     "fp32_over_fp64": r32["value"] / r64["value"]},
            "shadows": extras}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
