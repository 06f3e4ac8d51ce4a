"""Benchmark of the matrix-free SEM-NI monodomain time step on GB300.

One benchmark step = one full time step of the partitioned scheme
(Section 3, Algorithm 1) on the ~2 M DOF operator-sweep slab at p = 4
(20 x 7 x 3 mm, 83 x 29 x 13 hexahedra, 2,064,933 nodes, vertices perturbed by
+-10 % of h, fibre angle rotating -60 -> +60 degrees through z):
  fused ionic update + right-hand side  ->  flexible FP64 PCG to
  ||r|| <= 1e-10 ||b|| with the mixed-precision multigrid V-cycle.

Prints ONE JSON line (rank 0).  ``value`` is whole-job DOF-steps per second
(nodes advanced by one time step per second, summed over ranks) of the
mixed-precision solver.  The same line carries
  - the plain FP64 paths on the same slab from the same state: Jacobi-CG, and
    multigrid PCG with an all-FP64 V-cycle on the same hierarchy (so the
    precision speed-up is measured at equal preconditioning);
  - ``roofline`` for the kernel that takes the most time in the step, timed
    live with CUDA events on its launching stream inside the timed region;
  - ``configs``: the other workloads, timed by CUDA events in the same run --
    the p = 1..6 operator sweep (~2 M DOFs each), the 8.57 M DOF FP64-GMG
    monodomain run, and the ~30 M DOF mixed-precision runs at p = 4 and 6;
  - ``cpu_baseline``: the CPU oracle on the machine's host cores.

``--impl reference`` times the CPU oracle itself as the reference arm.
``--sweep`` / ``--workload`` run one of the extra workloads alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SEM operator GDOF/s and monodomain steps/s, mixed vs FP64 at 1e-8; % roofline"
UNIT = "GDOF-steps/s"
DT = 0.05            # ms
RTOL = 1e-10
MAXIT = 2000
STIM_RADIUS = 1.5    # mm
STIM_AMP = 50.0      # mV/ms
STIM_T_OFF = 1.0     # ms
SLAB_LENGTHS = W.SLAB_LENGTHS_MM
MG_DTYPE = {"fp32": "f32", "bf16": "f32 arithmetic / bf16 metric", "fp64": "f64",
            "tc": "f32 vectors / bf16 metric / bf16 tensor-core contractions with f32 accumulation"}
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64: 152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz

# DRAM bytes (read + write) per launch from one ncu capture of the kernel on the
# p = 4 SEM-NI slab of 2,064,933 nodes, each with the hash of the kernel sources it
# was taken from: a figure whose kernel code has changed since is reported as null
# (kernel_source_hash below; comments do not count).
NCU_TRAFFIC = {(4, "LGL"): (273.026304e6 + 12.97408e6, "apply")}
NCU_TRAFFIC_SMOOTHER = {(4, "LGL", "bf16"): (88.765696e6 + 1.543936e6, "apply")}
NCU_SOURCE_HASH = {"apply": "9c6bd0526832d33d"}
KERNEL_SOURCES = {"apply": ("sem_apply_kernel.cuh", "sem_apply_fp32.cu", "sem_apply_fp64.cu",
                            "sem_internal.cuh")}


def _code_only(text: str) -> str:
    """C++ source without its comments and blank lines (string literals in these
    files hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def _per_s(amount, ms):
    """amount per second over ms milliseconds (NaN when nothing was timed)."""
    return amount / (ms * 1e-3) if ms > 0 else float("nan")


def kernel_source_hash(kind: str) -> str:
    """First 16 hex digits of the sha256 of the code (comments left out) of the
    CUDA sources of a kernel family."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2205_05136_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(table, key):
    """DRAM bytes per launch of the captured kernel, or None when there is no
    capture or its kernel sources changed after it."""
    ent = table.get(key)
    if ent is None:
        return None
    val, kind = ent
    return val if kernel_source_hash(kind) == NCU_SOURCE_HASH.get(kind) else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def apply_flops_per_element(p: int, quad: str) -> int:
    """Algorithmic flops of one element apply with plain sum factorization:
    SEM-NI 6 sweeps of 2 n^4, SEM 12 sweeps, plus 22 n^3 at the quadrature points."""
    n = p + 1
    sweeps = 6 if quad == "LGL" else 12
    return sweeps * 2 * n ** 4 + 22 * n ** 3


def apply_bytes_per_element_fp32(p: int, metric: str = "fp32") -> int:
    """Algorithmic HBM bytes of one FP32 element apply: 7 metric values per
    quadrature point (4 bytes, or 2 with the bf16 metric), the int32 map, and
    u read + y written once per node (4 bytes each).  The tensor-core kernel
    ("tc", bf16 metric) takes node indices from the slab's numbering and reads
    no map."""
    n = p + 1
    mb = 2 if metric in ("bf16", "tc") else 4
    mapb = 0 if metric == "tc" else 4 * n ** 3
    return 7 * mb * n ** 3 + mapb + 8 * p ** 3


def apply_bytes_per_element(p: int) -> int:
    """Algorithmic HBM bytes of one FP64 element apply: 7 metric doubles per
    quadrature point, the int32 map, and u read + y written once per node."""
    n = p + 1
    return 56 * n ** 3 + 4 * n ** 3 + 16 * p ** 3


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, maxmhz, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                maxmhz = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": maxmhz, "reasons": sorted(reasons),
                "samples": len(mhz)}


def workload_name(p, quad, s, ndofs):
    """The workload string of the JSON line's config (the same for both arms)."""
    return (f"monodomain BDF2 time step, {'SEM-NI' if quad == 'LGL' else 'SEM'} Q{p} slab "
            f"20x7x3 mm, {s.nx}x{s.ny}x{s.nz} hexahedra, {ndofs} DOFs, +-10% vertex perturbation, "
            f"fibres -60..+60 deg, dt {DT} ms, CG rtol {RTOL}")


def workload(p=4):
    s = W.sweep_slab(p)
    ne = s.n_elements
    tissue = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
    centre = W.seeded_point(s.lengths, STIM_RADIUS, seed=W.SEED_STIM)
    return s, tissue, centre


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(p, quad, target_s):
    """Times the oracle's element-by-element apply (dense local matrices) over a
    bounded sample of the workload's elements; returns (seconds per element,
    elements timed)."""
    from oracle import mesh as Mh
    s, tissue, _ = workload(p)
    sp_ = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    u = W.uniform_vector(sp_.ndofs, -85.0, 20.0, seed=W.SEED_U)
    Mh.apply_element_by_element(sp_, tissue, u, 30.0, 1.0, elements=range(2))  # tables, caches
    t0 = time.perf_counter()
    done = 0
    e = 0
    while True:
        Mh.apply_element_by_element(sp_, tissue, u, 30.0, 1.0, elements=range(e, e + 8))
        e = (e + 8) % sp_.nelem
        done += 8
        if time.perf_counter() - t0 >= target_s:
            break
    return (time.perf_counter() - t0) / done, done


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_timed(p, quad, target_s, offset, barrier, queue):
    """One oracle process: set-up, then (after every process is ready) the
    element-by-element apply over consecutive elements from `offset` for
    target_s seconds; puts (elements, seconds) on the queue."""
    from oracle import mesh as Mh
    s, tissue, _ = workload(p)
    sp_ = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
    u = W.uniform_vector(sp_.ndofs, -85.0, 20.0, seed=W.SEED_U)
    Mh.apply_element_by_element(sp_, tissue, u, 30.0, 1.0, elements=range(2))  # tables, caches
    barrier.wait()
    e = offset % sp_.nelem
    done = 0
    t0 = time.perf_counter()
    while True:
        n = min(8, sp_.nelem - e)
        Mh.apply_element_by_element(sp_, tissue, u, 30.0, 1.0, elements=range(e, e + n))
        e = (e + n) % sp_.nelem
        done += n
        if time.perf_counter() - t0 >= target_s:
            break
    queue.put((done, time.perf_counter() - t0))


def run_oracle_parallel(p, quad, target_s, workers):
    """Times the oracle's element-by-element apply in `workers` single-thread
    processes at once (spawned, no GPU), each on its own stretch of elements;
    returns the elements per second of all processes together and the list of
    (elements, seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                            "CUDA_VISIBLE_DEVICES")}
    for k in saved:
        os.environ[k] = "" if k == "CUDA_VISIBLE_DEVICES" else "1"
    try:
        barrier = ctx.Barrier(workers)
        q = ctx.Queue()
        procs = [ctx.Process(target=_oracle_timed, args=(p, quad, target_s, k * 1009, barrier, q))
                 for k in range(workers)]
        for pr in procs:
            pr.start()
        res = [q.get(timeout=900) for _ in procs]
        for pr in procs:
            pr.join(timeout=60)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sum(d / t for d, t in res), res


def _oracle_worker(p, quad, target_s):
    sec, done = oracle_sample(p, quad, target_s)
    print(json.dumps({"sec_per_element": sec, "elements": done}))


def run_oracle_subprocess(p, quad, target_s):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, "-c",
           f"import bench; bench._oracle_worker({p}, {quad!r}, {target_s})"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_equivalent(sec_per_element, nelem, ndofs, applies_per_step):
    """Oracle DOF-steps/s: one step needs `applies_per_step` applies over all elements."""
    step_s = sec_per_element * nelem * applies_per_step
    return ndofs / step_s / 1e9, step_s


# --------------------------------------------------------------- GPU arm
def init_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, ws, dist


def time_arm(slab, precond, args, dist, dev, clocks=False):
    """Warm-up, then K timed time steps from the rest state; returns
    (ms, stats, u after the run, state, clock summary)."""
    import torch
    state = slab.new_state(-85.0, 1.0)
    stream = torch.cuda.current_stream()
    state.step(DT, args.warmup, rtol=RTOL, maxit=MAXIT, precond=precond)
    # restarts the library's sampling of apply timings (one solve in ten, the
    # first timed step included), so that every timed run has samples
    slab.set_timing(True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(dev) if clocks else None
    if clk:
        clk.__enter__()
    ev0.record(stream)
    stats = state.step(DT, args.steps, rtol=RTOL, maxit=MAXIT, precond=precond)
    ev1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    u, h, _ = state.get()
    return ms, stats, (u, h), state, (clk.summary() if clk else None)


def field_errors(u, h, u_ref, h_ref):
    """Relative L2 and Linf differences of u and h against a reference run."""
    import torch
    return {"u_rel_l2": float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref)),
            "u_rel_linf": float((u - u_ref).abs().max() / u_ref.abs().max()),
            "h_rel_l2": float(torch.linalg.norm(h - h_ref) / torch.linalg.norm(h_ref)),
            "h_rel_linf": float((h - h_ref).abs().max() / h_ref.abs().max())}


def oracle_step_config1(nsteps=100):
    """The oracle's own time step (Section 3, Algorithm 1: ionic update, right-hand
    side, exact sparse solve) on the small slab workload -- 8 x 4 x 2 Q2 SEM-NI
    elements, 765 DOFs, corner stimulus, dt 0.05 ms -- timed end to end on one host
    core for `nsteps` steps."""
    from oracle import mesh as Mh
    from oracle import monodomain as MD
    s = W.slab(8, 4, 2, SLAB_LENGTHS, perturb=0.0, seed=W.SEED_MESH)
    tissue = W.constant_tissue(s, 0.12, 0.03, 0.0)
    o = Mh.SlabSpace(s.flat_vertices(), s.nx, s.ny, s.nz, 2, "LGL")
    box = (0.0, 0.0, 0.0, 1.5, 1.5, 1.5)
    t0 = time.perf_counter()
    md = MD.Monodomain(o, tissue, DT, region=("box", box), amplitude=STIM_AMP, t_on=0.0, t_off=STIM_T_OFF)
    t1 = time.perf_counter()
    md.run(MD.rest_state(o.ndofs), nsteps)
    t2 = time.perf_counter()
    return {"workload": "monodomain BDF2 steps, SEM-NI Q2 slab 20x7x3 mm, 8x4x2 hexahedra, 765 DOFs, "
                        "corner stimulus 50 mV/ms for 1 ms, dt 0.05 ms",
            "steps": nsteps, "cores": 1, "setup_s": t1 - t0, "seconds": t2 - t1,
            "steps_per_s": nsteps / (t2 - t1), "value": o.ndofs * nsteps / (t2 - t1) / 1e9,
            "unit": UNIT, "kind": "oracle",
            "sample": "oracle.monodomain.Monodomain.run: assembled M and K, sparse LU solves (numpy/scipy fp64)"}


def run_gpu(args):
    import torch
    rank, ws, dist = init_dist()
    dev = torch.cuda.current_device()
    from paper_2205_05136_gb300 import build as gbuild
    if rank == 0:
        gbuild.build()
    if dist is not None:
        dist.barrier()
    import paper_2205_05136_gb300 as gb
    from paper_2205_05136_gb300 import capi

    p, quad = args.p, args.quad
    s, tissue, centre = workload(p)
    slab = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad, device=dev)
    slab.set_tissue(*tissue)
    slab.set_ionic()
    slab.set_stimulus("sphere", (*centre, STIM_RADIUS), STIM_AMP, 0.0, STIM_T_OFF)
    slab.set_timing(True)
    n_d, n_e = slab.ndofs, slab.nelem
    prec = {"fp32": gb.SEM_PREC_FP32, "bf16": gb.SEM_PREC_FP32_BF16, "fp64": gb.SEM_PREC_FP64,
            "tc": gb.SEM_PREC_BF16_TC}[args.mg_precision]
    mg = (args.mg_degree, args.mg_coarse_degree, args.mg_min_coarse_dofs)

    # plain FP64 path: Jacobi-CG with the FP64 operator
    capi.sem_set_operator_precision(slab.ctx, gb.SEM_PREC_FP64)
    capi.sem_set_gmg(slab.ctx, *mg, prec)
    ms64 = msg64 = float("nan")
    if args.arms in ("all", "fp64"):
        ms64, st64, f64, state64, clk64 = time_arm(slab, gb.SEM_PC_JACOBI, args, dist, dev,
                                                   clocks=args.arms == "fp64")
        state64.close()
        # all-FP64 multigrid PCG on the hierarchy of the mixed path (FP64 operator and V-cycle)
        capi.sem_set_gmg(slab.ctx, *mg, gb.SEM_PREC_FP64)
        msg64, stg64, fg64, stateg64, _ = time_arm(slab, gb.SEM_PC_GMG, args, dist, dev)
        stateg64.close()
    if args.arms == "fp64":  # report the plain FP64 path alone
        msmx, stats, fmx, clk = ms64, st64, f64, clk64
        state = slab.new_state(-85.0, 1.0)
        state.step(DT, 2, rtol=RTOL, maxit=MAXIT)
    else:
        # mixed-precision path: flexible FP64 CG (operator in double-float arithmetic unless
        # --op-precision fp64) preconditioned by the low-precision multigrid V-cycle
        capi.sem_set_operator_precision(
            slab.ctx, gb.SEM_PREC_DF64 if args.op_precision == "df64" else gb.SEM_PREC_FP64)
        capi.sem_set_gmg(slab.ctx, *mg, prec)
        msmx, stats, fmx, state, clk = time_arm(slab, gb.SEM_PC_GMG, args, dist, dev, clocks=True)
    if args.arms == "mixed":
        st64 = stg64 = stats
        f64 = fg64 = fmx

    ms = msmx
    value = ws * n_d * args.steps / (ms * 1e-3) / 1e9
    iters = stats.cg_iters / max(args.steps, 1)
    apply_ms = stats.apply_ms / max(stats.n_apply, 1)
    flops = n_e * apply_flops_per_element(p, quad)
    achieved_tf = _per_s(flops, apply_ms) / 1e12 if apply_ms > 0 else None
    algo_bytes = n_e * apply_bytes_per_element(p)
    apply64_ms = st64.apply_ms / max(st64.n_apply, 1)
    pk = peaks()
    hbm_peak = pk.get("hbm_gbs", 6780.0)
    outer_is_df = args.arms != "fp64" and args.op_precision == "df64"
    outer = {
        "kernel": f"sem_apply_kernel<P={p},{quad},{'df64' if outer_is_df else 'f64'},dot> (outer CG operator)",
        "launches": int(stats.cg_iters), "timed": int(stats.n_apply), "avg_ms": apply_ms if apply_ms > 0 else None,
        "total_ms": apply_ms * stats.cg_iters,
        "fp64_equivalent_tflops": achieved_tf,
        "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": algo_bytes,
    }
    kernels = {"outer_apply": outer}
    dominant = "outer_apply"
    if stats.n_smoother_apply > 0:
        sm_ms = stats.smoother_apply_ms / stats.n_smoother_apply
        sm_bytes = n_e * apply_bytes_per_element_fp32(p, args.mg_precision)
        per_vcycle = 2 * args.mg_degree  # fine-level applies per V-cycle (one V-cycle per PCG iteration)
        kernels["smoother_apply"] = {
            "kernel": smoother_kernel_name(p, quad, args.mg_precision),
            "timed": int(stats.n_smoother_apply), "avg_ms": sm_ms,
            "total_ms_est": sm_ms * per_vcycle * stats.cg_iters,
            "algorithmic_bytes_per_launch": sm_bytes,
            "achieved_gbs": sm_bytes / (sm_ms * 1e-3) / 1e9,
        }
        if kernels["smoother_apply"]["total_ms_est"] > outer["total_ms"]:
            dominant = "smoother_apply"
    if dominant == "smoother_apply":
        ksm = kernels["smoother_apply"]
        roofline = {"bound": "hbm", "achieved": ksm["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": ksm["achieved_gbs"] / hbm_peak,
                    "traffic": ncu_traffic(NCU_TRAFFIC_SMOOTHER, (p, quad, args.mg_precision)),
                    "kernel": ksm["kernel"],
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst figure"}
    elif outer_is_df:
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_tf / FP64_PEAK_TFLOPS if achieved_tf else None, "traffic": None,
                    "kernel": outer["kernel"],
                    "peak_note": ("FP64-equivalent flops of the double-float operator, which runs on the FP32 pipe, "
                                  "against the nominal native FP64 peak of 1.25 TFLOP/s")}
    else:
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_tf / FP64_PEAK_TFLOPS if achieved_tf else None,
                    "traffic": args.traffic if args.traffic is not None else ncu_traffic(NCU_TRAFFIC, (p, quad)),
                    "kernel": outer["kernel"],
                    "peak_note": "nominal FP64 1.25 TFLOP/s (no FP64 figure in MEASURED_PEAKS.json; DFMA probe measured 1.19)"}
    roofline["algorithmic_flops_per_launch"] = flops if dominant == "outer_apply" else None
    roofline["algorithmic_bytes_per_launch"] = (algo_bytes if dominant == "outer_apply"
                                                else kernels["smoother_apply"]["algorithmic_bytes_per_launch"])

    # end to end through the public C ABI with host buffers (page-locked), one
    # step per call, continuing from the device state reached above: each call
    # reads u^n, u^{n-1}, h^n, h^{n-1} from host memory and writes u^{n+1},
    # h^{n+1} to host memory; the caller rotates three host arrays per field
    ck = state.checkpoint()
    hu = [ck["u_prev"].cpu().pin_memory(), ck["u"].cpu().pin_memory(),
          torch.empty(n_d, dtype=torch.float64).pin_memory()]
    hh = [ck["h_prev"].cpu().pin_memory(), ck["h"].cpu().pin_memory(),
          torch.empty(n_d, dtype=torch.float64).pin_memory()]
    n2 = ck["n"]
    n_e2e = max(1, min(args.steps, 50))
    # one untimed call first (it creates the context's host-step buffers, stream
    # and events); the timed calls continue from its result
    capi.sem_step_host_out(slab.ctx, hu[1], hu[0], hh[1], hh[0], hu[2], hh[2], n2, DT, RTOL, 0.0,
                           MAXIT, gb.SEM_PC_JACOBI if args.arms == "fp64" else gb.SEM_PC_GMG)
    hu = [hu[1], hu[2], hu[0]]
    hh = [hh[1], hh[2], hh[0]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_carried = 0
    for k in range(n_e2e):
        st_k = capi.sem_step_host_out(slab.ctx, hu[1], hu[0], hh[1], hh[0], hu[2], hh[2], n2 + 1 + k, DT, RTOL, 0.0,
                                      MAXIT, gb.SEM_PC_JACOBI if args.arms == "fp64" else gb.SEM_PC_GMG)
        e2e_carried += st_k.carried_solves
        hu = [hu[1], hu[2], hu[0]]
        hh = [hh[1], hh[2], hh[0]]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = n_d * n_e2e / e2e_s / 1e9 * ws
    state.close()
    slab.close()
    torch.cuda.empty_cache()

    # the other workloads, in the same run (each timed by CUDA events)
    configs = None
    if not args.no_extra:
        t_extra = time.perf_counter()
        configs = {"sweep_2m": sweep_records(args, steps=args.extra_apply_steps),
                   "gmg8m": gmg8m_record(args, nsteps=args.gmg8m_steps),
                   "mixed30m": mixed30m_records(args, nsteps=args.mixed30m_steps)}
        configs["wall_s"] = time.perf_counter() - t_extra

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cores = host_cores()
            rate, res = run_oracle_parallel(p, quad, args.cpu_seconds, cores)
            applies = st64.cg_iters / max(args.steps, 1) + 1.0
            step_s = n_e * applies / rate
            cpu = {"value": n_d / step_s / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": (f"apply-rate extrapolation: oracle element-by-element apply (dense local matrices, "
                              f"numpy fp64) in {cores} single-thread processes at once, {args.cpu_seconds:.0f} s each, "
                              f"{sum(d for d, _ in res)} of this slab's {n_e} elements in all "
                              f"({rate:.0f} elements/s together, {res[0][0] / res[0][1]:.0f} per process); "
                              f"scaled to one Jacobi-CG time step of {applies:.2f} applies, the FP64 Jacobi-CG "
                              f"count measured above ({step_s:.0f} s/step)")}
        except Exception as exc:  # report, never fail the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": f"failed: {exc}"}
        try:
            cpu["step_config1"] = oracle_step_config1()
        except Exception as exc:
            cpu["step_config1"] = {"failed": str(exc)}

    speed_j = ms64 / msmx
    speed_g = msg64 / msmx
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64 vectors, residuals, inner products, ionic exp; "
                  f"{'double-float (f32 pairs)' if outer_is_df else 'f64'} operator; "
                  f"{MG_DTYPE[args.mg_precision]} multigrid V-cycle"),
        "data": "synthetic",
        "config": {
            "workload": workload_name(p, quad, s, n_d),
            "solver": (f"flexible FP64 PCG ({args.op_precision} operator) + {args.mg_precision} GMG V-cycle "
                       f"(p-then-h coarsening down to {args.mg_min_coarse_dofs} nodes, "
                       f"Chebyshev({args.mg_degree}), coarse Chebyshev({args.mg_coarse_degree}))"),
            "p": p, "quadrature": quad, "ndofs": n_d, "nelem": n_e,
            "parallelism": f"replicas x{ws}",
            "l2": f"inputs larger than L2: {n_e * 7 * (p + 1) ** 3 * 8 / 1e6:.0f} MB FP64 metric streamed per apply",
        },
        "steps_per_s": args.steps / (ms * 1e-3),
        "cg_iters_per_step": iters,
        "apply_gdofs": _per_s(n_d, apply_ms) / 1e9 if apply_ms > 0 else None,
        "apply_ms": apply_ms,
        "fp64_path": {"solver": "Jacobi-CG, FP64 operator", "value": ws * n_d * args.steps / (ms64 * 1e-3) / 1e9,
                      "unit": UNIT, "ms_per_step": ms64 / args.steps,
                      "cg_iters_per_step": st64.cg_iters / max(args.steps, 1),
                      "apply_ms": apply64_ms,
                      "apply_gdofs": _per_s(n_d, apply64_ms) / 1e9 if apply64_ms > 0 else None},
        "fp64_gmg_path": {"solver": (f"flexible PCG, FP64 operator + FP64 GMG V-cycle on the same hierarchy "
                                     f"(Chebyshev({args.mg_degree}), coarse Chebyshev({args.mg_coarse_degree}))"),
                          "value": ws * n_d * args.steps / (msg64 * 1e-3) / 1e9, "unit": UNIT,
                          "ms_per_step": msg64 / args.steps,
                          "cg_iters_per_step": stg64.cg_iters / max(args.steps, 1)},
        "mixed_vs_fp64": {"speedup": speed_g, "speedup_vs_fp64_gmg": speed_g, "speedup_vs_fp64_jacobi": speed_j,
                          "vs_fp64_gmg": field_errors(fmx[0], fmx[1], fg64[0], fg64[1]),
                          "vs_fp64_jacobi": field_errors(fmx[0], fmx[1], f64[0], f64[1]),
                          # the two FP64 solvers against each other: the part of vs_fp64_jacobi that
                          # comes from the solvers' different iterates at rtol, not from the precision
                          "fp64_gmg_vs_fp64_jacobi": field_errors(fg64[0], fg64[1], f64[0], f64[1]),
                          "rel_l2_u_diff": field_errors(fmx[0], fmx[1], fg64[0], fg64[1])["u_rel_l2"],
                          "note": ("speedup = FP64-GMG step time / mixed step time (same hierarchy, so the "
                                   "precision alone); u and h after warm-up + timed steps of each path from the "
                                   "same start state")},
        "roofline": roofline,
        "kernels": kernels,
        "fp64_apply_roofline": {"bound": "alu", "kernel": f"sem_apply_kernel<P={p},{quad},f64,dot> (plain FP64 path)",
                                "achieved": _per_s(flops, apply64_ms) / 1e12, "peak": FP64_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": _per_s(flops, apply64_ms) / 1e12 / FP64_PEAK_TFLOPS,
                                "traffic": ncu_traffic(NCU_TRAFFIC, (p, quad))} if args.arms != "mixed" else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * n_d,
                "d2h_bytes_per_step": 2 * 8 * n_d, "steps": n_e2e,
                "carried_solves": int(e2e_carried),
                "call": "sem_step_host_out (page-locked host arrays, rotated by the caller)"},
        "gpu_launches": int(stats.kernel_launches),
        "clocks": clk,
        "configs": configs,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def smoother_kernel_name(p, quad, mg_precision):
    if mg_precision == "tc" and quad == "LGL" and 2 <= p <= 4:
        return f"sem_apply_tc_kernel<P={p}> (SEM-NI, bf16 metric, mma.sync bf16 -> f32; fine-level V-cycle apply)"
    return (f"{'sem_apply_pipe_kernel' if p <= 4 else 'sem_apply_kernel'}<P={p},{quad},f32,"
            f"{'bf16' if mg_precision in ('bf16', 'tc') else 'f32'} metric> (fine-level V-cycle apply)")


def _timed_applies(slab, u, y, steps, precision, flush):
    """Median CUDA-event time (s) of `steps` applies y = (30 M + K) u, each after an
    L2 flush (a 256 MB write), after 3 untimed applies."""
    import torch
    for _ in range(3):
        slab.apply(u, 30.0, 1.0, precision=precision, out=y)
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        slab.apply(u, 30.0, 1.0, precision=precision, out=y)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(ts)


def sweep_records(args, steps=10, ps=(1, 2, 3, 4, 5, 6)):
    """Operator-apply sweep, p = 1..6, SEM-NI and SEM, ~2 M DOFs each, 20 x 7 x 3 mm,
    perturbed, rotating fibres, u ~ U[-1, 1]: FP64 (and double-float, FP32, FP32 +
    bf16 metric) apply times, GDOF/s and the FP64 fraction of peak."""
    import torch
    import paper_2205_05136_gb300 as gb
    out = []
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for p in ps:
        for quad in ("LGL", "LG"):
            s, tissue, _ = workload(p)
            slab = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad)
            slab.set_tissue(*tissue)
            u = torch.tensor(W.uniform_vector(slab.ndofs, seed=W.SEED_U), device="cuda")
            y = torch.empty_like(u)
            t = _timed_applies(slab, u, y, steps, gb.SEM_PREC_FP64, flush)
            flops = slab.nelem * apply_flops_per_element(p, quad)
            rec = {"p": p, "quad": quad, "ndofs": slab.ndofs, "nelem": slab.nelem,
                   "apply_ms": t * 1e3, "gdofs": slab.ndofs / t / 1e9,
                   "tflops_algorithmic": flops / t / 1e12,
                   "frac_fp64_peak": flops / t / 1e12 / FP64_PEAK_TFLOPS,
                   "gbs_algorithmic": slab.nelem * apply_bytes_per_element(p) / t / 1e9}
            ydf = torch.empty_like(u)
            tdf = _timed_applies(slab, u, ydf, steps, gb.SEM_PREC_DF64, flush)
            rec["df64_apply_ms"] = tdf * 1e3
            rec["df64_gdofs"] = slab.ndofs / tdf / 1e9
            rec["df64_rel_diff_vs_fp64"] = float(torch.linalg.norm(ydf - y) / torch.linalg.norm(y))
            u32 = u.float()
            for prec, name in ((gb.SEM_PREC_FP32, "fp32"), (gb.SEM_PREC_FP32_BF16, "fp32_bf16")):
                y32 = torch.empty_like(u32)
                t32 = _timed_applies(slab, u32, y32, steps, prec, flush)
                rec[f"{name}_apply_ms"] = t32 * 1e3
                rec[f"{name}_gdofs"] = slab.ndofs / t32 / 1e9
                rec[f"{name}_rel_diff_vs_fp64"] = float(torch.linalg.norm(y32.double() - y) / torch.linalg.norm(y))
            out.append(rec)
            slab.close()
            del u, y, ydf, u32
            torch.cuda.empty_cache()
    return out


def run_sweep(args):
    from paper_2205_05136_gb300 import build as gbuild
    gbuild.build()
    for rec in sweep_records(args, steps=args.steps, ps=args.sweep_p):
        print(json.dumps(dict(sweep=True, **rec)), flush=True)


def _slab_ctx(gb, s, p, quad, tissue, dev=0):
    slab = gb.Slab(s.flat_vertices(), s.nx, s.ny, s.nz, p, quad, device=dev)
    slab.set_tissue(*tissue)
    slab.set_ionic()
    return slab


def _timed_run(st, nsteps, precond, maxit=MAXIT):
    """nsteps time steps on the current stream between two CUDA events; (s, stats)."""
    import torch
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    stats = st.step(DT, nsteps, rtol=RTOL, maxit=maxit, precond=precond)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e-3, stats


def gmg8m_record(args, nsteps=200):
    """Monodomain run on a 40 x 20 x 6 mm slab at p = 4 (128 x 64 x 16 elements,
    8.57 M DOFs), rotating fibres, `nsteps` steps of 0.05 ms (200: 10 ms), seeded
    stimulus ball r = 1.5 mm, flexible PCG with the p-then-h multigrid (p 4 -> 2 -> 1,
    then h-levels down to 2,000 nodes; Chebyshev 3, coarsest level Chebyshev 10), in two
    arms on the same hierarchy: all FP64 (operator and V-cycle), and mixed
    (double-float outer operator, bf16-metric FP32 V-cycle); activation times tracked
    inside the timed run; relative L2 / Linf differences of u and h after the run."""
    import torch
    import paper_2205_05136_gb300 as gb
    from paper_2205_05136_gb300 import capi
    s = W.slab(128, 64, 16, (40.0, 20.0, 6.0), perturb=0.1, seed=W.SEED_MESH)
    ne = s.n_elements
    tissue = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
    slab = _slab_ctx(gb, s, 4, args.quad, tissue)
    centre = W.seeded_point(s.lengths, STIM_RADIUS, seed=W.SEED_STIM)
    slab.set_stimulus("sphere", (*centre, STIM_RADIUS), STIM_AMP, 0.0, STIM_T_OFF)
    slab.set_timing(True)
    out = {"workload": (f"40x20x6 mm slab, 128x64x16 Q4 SEM-NI elements, {slab.ndofs} DOFs, +-10% perturbation, "
                        f"fibres -60..+60 deg, {nsteps} steps of {DT} ms from rest, stimulus ball r 1.5 mm"),
           "ndofs": slab.ndofs, "steps": nsteps,
           "solver": "flexible PCG rtol 1e-10, GMG p 4->2->1 then h down to 2,000 nodes, Chebyshev(3), coarse Chebyshev(10)"}
    finals = {}
    rest = {"u": torch.full((slab.ndofs,), -85.0, dtype=torch.float64, device="cuda"),
            "u_prev": torch.full((slab.ndofs,), -85.0, dtype=torch.float64, device="cuda"),
            "h": torch.ones(slab.ndofs, dtype=torch.float64, device="cuda"),
            "h_prev": torch.ones(slab.ndofs, dtype=torch.float64, device="cuda"), "n": 0}
    for name, op, prec in (("fp64", gb.SEM_PREC_FP64, gb.SEM_PREC_FP64),
                           ("mixed", gb.SEM_PREC_DF64, gb.SEM_PREC_FP32_BF16)):
        capi.sem_set_operator_precision(slab.ctx, op)
        capi.sem_set_gmg(slab.ctx, 3, 10, 2000, prec)
        info = capi.sem_gmg_info(slab.ctx, 1.5 / DT)
        st = slab.new_state(-85.0, 1.0)
        st.step(DT, 3, rtol=RTOL, maxit=MAXIT, precond=gb.SEM_PC_GMG)  # warm-up, then back to rest
        st.restore(rest)
        st.track_activation(True)  # activation times (Eq. tau) on the way, inside the timed run
        el, stats = _timed_run(st, nsteps, gb.SEM_PC_GMG)
        u, h, n = st.get()
        tau, dmax = st.activation()
        finals[name] = (u, h, tau, dmax)
        out["levels"] = {"p": info["p"], "dims": info["dims"], "ndofs": info["ndofs"]}
        out[name] = {"seconds": el, "steps_per_s": nsteps / el, "gdof_steps_per_s": slab.ndofs * nsteps / el / 1e9,
                     "cg_iters_per_step": stats.cg_iters / nsteps,
                     "u_max_mV": float(u.max()), "activated_fraction": float((u > -40.0).double().mean()),
                     "outer_apply_ms": stats.apply_ms / max(stats.n_apply, 1)}
        st.close()
    (u64, h64, tau64, d64), (umx, hmx, taumx, dmx) = finals["fp64"], finals["mixed"]
    act = d64 > 10.0  # nodes the front reached (upstroke faster than 10 mV/ms)
    if bool(act.any()):
        out["activation"] = {"activated_nodes": int(act.sum()),
                             "tau_ms_min": float(tau64[act].min()), "tau_ms_max": float(tau64[act].max()),
                             "mixed_same_tau_fraction": float((taumx[act] == tau64[act]).double().mean()),
                             "mixed_max_abs_tau_diff_ms": float((taumx[act] - tau64[act]).abs().max()),
                             "mixed_dudt_max_rel_diff": float(((dmx - d64)[act].abs() / d64[act]).max())}
    out["mixed"].update(field_errors(umx, hmx, u64, h64))
    out["mixed"]["speedup_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    slab.close()
    del finals, rest
    torch.cuda.empty_cache()
    return out


def run_gmg8m(args):
    from paper_2205_05136_gb300 import build as gbuild
    gbuild.build()
    print(json.dumps(gmg8m_record(args, nsteps=args.steps if args.steps != 200 else 200)), flush=True)


def mixed30m_records(args, nsteps=5, cases=((4, (207, 72, 31)), (6, (137, 48, 21))), sampled_rows=True):
    """Mixed precision at ~30 M DOFs (p = 4: 207 x 72 x 31; p = 6: 137 x 48 x 21), each
    arm from the rest state with the stimulus on: one untimed BDF1 step, then `nsteps`
    timed steps.  Arms: FP64 Jacobi-CG; flexible PCG with an all-FP64 GMG V-cycle; the
    mixed solver (double-float outer operator, bf16-metric FP32 V-cycle) on the same
    hierarchy (Chebyshev 6, coarse Chebyshev 6, coarsening down to 300,000 nodes).
    Per-field relative L2 and Linf of u and h against the FP64-GMG arm; sampled
    operator rows against the oracle."""
    import torch
    import paper_2205_05136_gb300 as gb
    from paper_2205_05136_gb300 import capi
    from oracle import mesh as Mh
    recs = []
    for p, dims in cases:
        s = W.slab(*dims, SLAB_LENGTHS, perturb=0.1, seed=W.SEED_MESH)
        ne = s.n_elements
        tissue = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
        slab = _slab_ctx(gb, s, p, args.quad, tissue)
        centre = W.seeded_point(s.lengths, STIM_RADIUS, seed=W.SEED_STIM)
        slab.set_stimulus("sphere", (*centre, STIM_RADIUS), STIM_AMP, 0.0, STIM_T_OFF)
        out = {"workload": (f"mixed precision, {'SEM-NI' if args.quad == 'LGL' else 'SEM'} Q{p} slab 20x7x3 mm, "
                            f"{dims[0]}x{dims[1]}x{dims[2]} hexahedra, {slab.ndofs} DOFs, +-10% perturbation, "
                            f"fibres -60..+60 deg, 1 + {nsteps} steps of {DT} ms from rest"),
               "p": p, "ndofs": slab.ndofs, "nelem": ne, "steps": nsteps}
        uvec = W.uniform_vector(slab.ndofs, seed=W.SEED_U)
        ut = torch.tensor(uvec, device="cuda")
        y64 = slab.apply(ut, 30.0, 1.0)
        if sampled_rows:
            o = Mh.SlabSpace(s.flat_vertices(), *dims, p, args.quad)
            idx = W.seeded_indices(slab.ndofs, 16, seed=7)
            ref = Mh.sampled_rows(o, tissue, uvec, idx, 30.0, 1.0)
            yi = y64[torch.tensor(idx, device="cuda")].cpu().numpy()
            out["apply_rel_err_fp64_vs_oracle_sampled"] = float(np.abs(yi - ref).max() / np.abs(ref).max())
        for prec, name in ((gb.SEM_PREC_FP32, "fp32"), (gb.SEM_PREC_FP32_BF16, "bf16")):
            yl = slab.apply(ut.float(), 30.0, 1.0, precision=prec).double()
            out[f"apply_rel_l2_{name}_vs_fp64"] = float(torch.linalg.norm(yl - y64) / torch.linalg.norm(y64))
            del yl
        del ut, y64
        results = {}
        for name, pc, op, prec in (("fp64_jacobi", gb.SEM_PC_JACOBI, gb.SEM_PREC_FP64, None),
                                   ("fp64_gmg", gb.SEM_PC_GMG, gb.SEM_PREC_FP64, gb.SEM_PREC_FP64),
                                   ("mixed", gb.SEM_PC_GMG, gb.SEM_PREC_DF64, gb.SEM_PREC_FP32_BF16)):
            capi.sem_set_operator_precision(slab.ctx, op)
            if prec is not None:
                capi.sem_set_gmg(slab.ctx, 6, 6, 300000, prec)
            st = slab.new_state(-85.0, 1.0)
            st.step(DT, 1, rtol=RTOL, maxit=MAXIT * 4, precond=pc)  # warm-up (BDF1)
            el, stt = _timed_run(st, nsteps, pc, maxit=MAXIT * 4)
            u, h, _ = st.get()
            results[name] = (u, h)
            out[name] = {"ms_per_step": el / nsteps * 1e3, "cg_iters_per_step": stt.cg_iters / nsteps,
                         "gdof_steps_per_s": slab.ndofs * nsteps / el / 1e9}
            st.close()
        ug, hg = results["fp64_gmg"]
        for name in ("mixed", "fp64_jacobi"):
            u, h = results[name]
            out[name].update({f"{k}_vs_fp64_gmg": v for k, v in field_errors(u, h, ug, hg).items()})
        out["mixed"]["speedup_vs_fp64_gmg"] = out["fp64_gmg"]["ms_per_step"] / out["mixed"]["ms_per_step"]
        out["mixed"]["speedup_vs_fp64_jacobi"] = out["fp64_jacobi"]["ms_per_step"] / out["mixed"]["ms_per_step"]
        recs.append(out)
        slab.close()
        del results
        torch.cuda.empty_cache()
    return recs


def run_mixed30m(args):
    from paper_2205_05136_gb300 import build as gbuild
    gbuild.build()
    for rec in mixed30m_records(args, nsteps=args.steps if args.steps != 200 else 10):
        print(json.dumps(rec), flush=True)


def run_adjoint(args):
    """Adjoint at p = 3 on a 140 x 49 x 21 deformed slab (3.99 M DOFs), 200 steps,
    checkpoint every 20, 64 seeded sensors; target from conductivities perturbed
    by U[0.8, 1.2] per element; gradient checked by central differences
    (h = 1e-6) on 16 seeded elements x (sigma_l, sigma_t, theta)."""
    import torch
    import paper_2205_05136_gb300 as gb
    from paper_2205_05136_gb300 import build as gbuild, capi
    gbuild.build()
    nsteps = args.steps if args.steps != 20 else 200
    s = W.slab(140, 49, 21, SLAB_LENGTHS, perturb=0.1, seed=W.SEED_MESH)
    ne = s.n_elements
    base = (np.full(ne, 0.12), np.full(ne, 0.03), W.transmural_fiber_angles(s))
    slab = _slab_ctx(gb, s, 3, args.quad, base)
    centre = W.seeded_point(s.lengths, STIM_RADIUS, seed=W.SEED_STIM)
    slab.set_stimulus("sphere", (*centre, STIM_RADIUS), STIM_AMP, 0.0, STIM_T_OFF)
    capi.sem_set_gmg(slab.ctx, 3, 8, 40000, gb.SEM_PREC_FP32)
    sensors = torch.tensor(W.seeded_indices(slab.ndofs, 64, seed=W.SEED_SENSORS), dtype=torch.int32)
    dev = torch.device("cuda")
    u0 = torch.full((slab.ndofs,), -85.0, dtype=torch.float64, device=dev)
    h0 = torch.ones(slab.ndofs, dtype=torch.float64, device=dev)
    kw = dict(checkpoint_every=20, rtol=1e-12, maxit=4 * MAXIT, precond=gb.SEM_PC_GMG)
    pl, pt = W.perturbed_conductivities(base[0], base[1])
    with torch.no_grad():
        target = gb.traces(slab, torch.tensor(pl, device=dev), torch.tensor(pt, device=dev),
                           torch.tensor(base[2], device=dev), u0, h0, DT, nsteps, sensors, **kw)
    prm = [torch.tensor(b, device=dev, requires_grad=True) for b in base]

    def loss_of(params):
        T = gb.traces(slab, params[0], params[1], params[2], u0, h0, DT, nsteps, sensors, **kw)
        return 0.5 * DT * torch.sum((T - target) ** 2)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = loss_of(prm)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    grads = [p.grad.detach().cpu().numpy() for p in prm]
    elems = W.seeded_indices(ne, 16, seed=W.SEED_FD)
    checks, worst = [], 0.0
    h = 1e-6
    with torch.no_grad():
        for k in range(3):
            scale = np.abs(grads[k]).max()
            for e in elems:
                vals = []
                for sgn in (1.0, -1.0):
                    q = [t.detach().clone() for t in prm]
                    q[k][e] += sgn * h
                    vals.append(float(loss_of(q)))
                fd = (vals[0] - vals[1]) / (2 * h)
                err = abs(grads[k][e] - fd) / max(abs(fd), 1e-3 * scale)
                worst = max(worst, err)
                checks.append((k, int(e), float(grads[k][e]), fd))
    print(json.dumps({
        "workload": "adjoint p=3 140x49x21 (3.99 M DOFs), 200 steps, checkpoint 20, 64 sensors",
        "ndofs": slab.ndofs, "steps": nsteps, "loss": float(L), "forward_s": t_fwd, "backward_s": t_bwd,
        "fd_checks": len(checks), "fd_max_rel_dev": worst, "fd_h": h, "fd_samples": checks[:6]}),
        flush=True)
    slab.close()


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on this workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, quad = args.p, args.quad
    s, _, _ = workload(p)
    nel = s.n_elements
    ndofs = (p * s.nx + 1) * (p * s.ny + 1) * (p * s.nz + 1)
    # applies per time step: the FP64 Jacobi-CG iterations per step that the GPU arm
    # measures on this workload (32.6) plus the residual apply
    applies = args.ref_applies_per_step
    per_step = max(1.0, min(8.0, 150.0 / max(args.steps + args.warmup, 1)))
    cores = host_cores()
    vals = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, res = run_oracle_parallel(p, quad, per_step, cores)
        wall = time.perf_counter() - t0
        step_s = nel * applies / rate
        if k >= args.warmup:
            vals.append((ndofs / step_s / 1e9, step_s, wall))
    v = statistics.median(x[0] for x in vals)
    sample = (f"apply-rate extrapolation: each bench step runs the oracle's element-by-element apply (numpy fp64) "
              f"in {cores} single-thread processes at once for ~{per_step:.0f} s over this slab's {nel} elements; "
              f"value = DOF-steps/s of a full time step of {applies} applies at that rate "
              f"(extrapolated {statistics.median(x[1] for x in vals):.0f} s per time step)")
    cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
           "extrapolated_s_per_time_step": statistics.median(x[1] for x in vals)}
    try:
        cpu["step_config1"] = oracle_step_config1()
    except Exception as exc:
        cpu["step_config1"] = {"failed": str(exc)}
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(x[2] for x in vals) * 1e3,
        "ms_per_step_note": "wall time of one bench step (one bounded oracle sample, process start-up included)",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(p, quad, s, ndofs), "p": p, "quadrature": quad,
                   "ndofs": ndofs, "nelem": nel},
        "cpu_baseline": cpu,
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--quad", default="LGL", choices=["LGL", "LG"])
    ap.add_argument("--cpu-seconds", type=float, default=2.0,
                    help="seconds of oracle work per host core for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per apply launch from an ncu capture of the current kernel")
    ap.add_argument("--ref-applies-per-step", type=float, default=33.0)
    ap.add_argument("--mg-precision", default="bf16", choices=["fp32", "bf16", "fp64", "tc"])
    ap.add_argument("--op-precision", default="df64", choices=["df64", "fp64"],
                    help="arithmetic of the outer CG operator in the mixed path")
    ap.add_argument("--arms", default="all", choices=["all", "mixed", "fp64"],
                    help="time the mixed-precision multigrid path, the plain FP64 paths, or all")
    ap.add_argument("--mg-degree", type=int, default=6)
    # tuned on the 2 M DOF slab at dt = 0.05 ms (mass-dominated operator): a degree-6
    # Chebyshev smoother on the p = 4 level and the p = 2 level (266,085 nodes) as the
    # coarsest level, smoothed by Chebyshev(5), give 3 PCG iterations per step and the
    # shortest step time with that count (coarse degrees 2..8: 3.13, 4, 3.17, 3, 3, -, 3
    # iterations)
    ap.add_argument("--mg-coarse-degree", type=int, default=5)
    ap.add_argument("--mg-min-coarse-dofs", type=int, default=300000)
    ap.add_argument("--workload", default="timestep", choices=["timestep", "gmg8m", "mixed30m", "adjoint"],
                    help="extra measurements of the multigrid, mixed-precision and adjoint workloads")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (operator sweep, 8.57 M and ~30 M DOF runs)")
    ap.add_argument("--extra-apply-steps", type=int, default=5, help="timed applies per sweep entry")
    ap.add_argument("--gmg8m-steps", type=int, default=200)
    ap.add_argument("--mixed30m-steps", type=int, default=5)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--sweep-p", type=int, nargs="*", default=[1, 2, 3, 4, 5, 6])
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not args.sweep:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "gmg8m":
        run_gmg8m(args)
    elif args.workload == "mixed30m":
        run_mixed30m(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
