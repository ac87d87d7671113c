"""Benchmark of the ACM-HD flux-reconstruction RHS on GB300.

One step = one fused right-hand-side evaluation R = -div F(U) + S(U) (face
trace kernel + fused kernel) of the 3-D Taylor-Green workload: p = 3 hexes
(4^3 Gauss-Legendre points), 64^3 periodic mesh on [-pi, pi]^3, 13
variables, FP32.  Metric: GDOF-RHS/s = n_elem * (p+1)^3 * 13 / t / 1e9.

Printed as one JSON line (rank 0).  Besides `value` (device-resident
inputs, CUDA events around exactly --steps steps) it carries:
  e2e           the same metric through fr_rhs_host (pinned host buffers,
                host->device and device->host copies inside the timed region)
  roofline      the fused kernel's algorithmic bytes / its event-timed
                duration, against the measured HBM copy bandwidth
  unfused/fp64  the six-kernel Table-1 pipeline and the FP64 fused RHS,
                timed the same way (context for the fused-vs-unfused ratio)
  cpu_baseline  the FP64 oracle timed on this host's cores on a bounded
                sample of the same workload
  clocks        nvidia-smi samples taken during the timed region

Multi-GPU (torchrun): every rank evaluates its own replica of the workload
(the RHS of one mesh has a halo exchange that is not built), so the value
is the DOF total over all ranks / the slowest rank's time ("weak").

--impl reference times the FP64 oracle itself on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "hex_p3_64cube"
METRIC = "GDOF-RHS/s"


def _rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def _init_dist(backend):
    """Process group of a torchrun launch (RANK, WORLD_SIZE and MASTER_* from
    the environment); None for a single process."""
    _, _, world = _rank_env()
    if world == 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist


def _max_over_ranks(dist, seconds, device):
    """The job's time: the slowest rank's (replicas run independently)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / seconds


def _reference_runs_here():
    """The reference arm runs on rank 0 only; other ranks exit without work."""
    rank, _, world = _rank_env()
    return world == 1 or rank == 0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _source_digest():
    """Digest of the fused RHS kernel's code (comments and blank lines
    dropped), to tell whether the committed ncu counters still describe it."""
    h = hashlib.sha256()
    for name in ("k_fused.cu", "fused_tile.cuh", "fr_device.cuh", "xface_layout.h"):
        with open(os.path.join(ROOT, "paper_2107_14027_gb300", "csrc", name)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per fused launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "fused_hex_p3_64cube.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        if prof.get("source_digest") == _source_digest():
            return float(prof["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


_ORACLE_PIECE = """
import sys, time
sys.path.insert(0, {root!r})
from oracle import fr
from paper_2107_14027_gb300 import workloads as W
cfg = W.WORKLOADS[{workload!r}]
n = ({n_side},) * 3
h = (cfg['hi'][0] - cfg['lo'][0]) / cfg['n'][0]
lo = (cfg['lo'][0],) * 3
hi = (cfg['lo'][0] + h * {n_side},) * 3
U = W.taylor_green(n, lo, hi, cfg['order'])
mesh = fr.Mesh(n, lo, hi)
prm = fr.Params(cfg['zeta'], cfg['nu'], cfg['t_r'])
def one():
    fr.rhs(U, mesh, cfg['order'], prm)
"""

_ORACLE_WORKER = _ORACLE_PIECE + """
def work(seconds):
    one()
    t0 = time.perf_counter(); k = 0
    while time.perf_counter() - t0 < seconds:
        one(); k += 1
    return k, time.perf_counter() - t0
"""


def _cpu_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    return env


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _cpu_baseline_runs(n_side, seconds):
    """The FP64 oracle RHS on an n_side^3 p = 3 piece of the workload, timed
    (a) in one single-threaded process and (b) in one single-threaded process
    per host core at once (a spawned pool, started from a fresh interpreter,
    so no GPU state is inherited).  Returns a dict of both rates (GDOF/s)."""
    code = _ORACLE_WORKER.format(root=ROOT, workload=WORKLOAD, n_side=n_side) + f"""
import json, multiprocessing as mp, os
if __name__ == "__main__":
    dof = U.size
    k, t = work({seconds})
    single = dof * k / t / 1e9
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.map(work, [{seconds}] * cores)
        wall = time.perf_counter() - t0
    allc = dof * sum(r[0] for r in res) / wall / 1e9
    print(json.dumps({{"single": single, "single_reps": k, "single_s": t / k, "all": allc,
                      "cores": cores, "all_reps": sum(r[0] for r in res), "wall": wall}}))
"""
    path = os.path.join("/tmp", f"acmhd_oracle_baseline_{os.getpid()}.py")
    with open(path, "w") as f:
        f.write(code)
    try:
        r = subprocess.run([sys.executable, path], capture_output=True, text=True, env=_cpu_env(),
                           timeout=900)
    finally:
        os.unlink(path)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def _err_vs_oracle(U, R, mesh_n, cfg, elems):
    """Per-variable error of the timed output R (sampled columns `elems`)
    against the oracle's per-element path on the same FP32-rounded input
    (part of the CPU-baseline leg): RMS error over RMS of the oracle's
    result (plain) and over RMS of the summed terms (scaled)."""
    from oracle import acmhd, fr
    from oracle.ops1d import Ops1D
    order = cfg["order"]
    mesh = fr.Mesh(mesh_n, cfg["lo"], cfg["hi"])
    prm = fr.Params(cfg["zeta"], cfg["nu"], cfg["t_r"])
    U64 = U.astype(np.float64)
    t0 = time.perf_counter()
    R_ref = fr.rhs_dense(U64, mesh, order, prm, elems=elems)
    t_ref = time.perf_counter() - t0
    ops = Ops1D(order)
    m = ops.m
    Dt = ops.D - np.outer(ops.dhl, ops.lm) - np.outer(ops.dhr, ops.lp)
    Ue = U64[:, :, elems].reshape(U.shape[0], m, m, m, len(elems))
    B = np.abs(acmhd.source(Ue, prm.T))
    for a in range(3):
        F = np.abs(acmhd.flux(Ue, a, prm.zeta, prm.nu, prm.T))
        ax = 3 - a
        B = B + (2.0 / mesh.h[a]) * np.moveaxis(np.tensordot(np.abs(Dt), F, axes=([1], [ax])),
                                                0, ax)
    B = B.reshape(U.shape[0], m ** 3, len(elems))
    diff = np.sqrt(np.mean((R - R_ref) ** 2, axis=(1, 2)))
    ref = np.sqrt(np.mean(R_ref ** 2, axis=(1, 2)))
    scale = np.sqrt(np.mean(B ** 2, axis=(1, 2)))
    names = ["P", "u", "v", "w"] + [f"{g}{x}" for g in "qrs" for x in "xyz"]
    # the plain relative error means something only where the result does not
    # cancel far below its summed terms: ||R|| / ||B|| >= 8 u / tol (FP32:
    # u = 2^-24, tol = 2e-5); other rows (the exact-gradient auxiliary rows,
    # P of the divergence-free field) are held to the scaled bound alone
    ratio = ref / np.maximum(scale, 1e-300)
    thr = 8 * 2.0 ** -24 / 2e-5
    plain = diff / np.maximum(ref, 1e-300)
    return {"elements": int(len(elems)), "oracle": "FP64 per-element (dense) path",
            "plain": {k: (float(v) if r >= thr else None)
                      for k, v, r in zip(names, plain, ratio)},
            "plain_rows_threshold": {"R_over_B_min": thr,
                                     "R_over_B": {k: float(r) for k, r in zip(names, ratio)},
                                     "note": "null: the row's result cancels below 8u/tol of "
                                             "its summed terms (the noise-free Taylor-Green "
                                             "field: every row); the scaled error holds"},
            "scaled": {k: float(v) for k, v in zip(names, diff / np.maximum(scale, 1e-300))},
            "max_scaled": float(np.max(diff / np.maximum(scale, 1e-300))),
            "oracle_s": t_ref}


def run_reference(args):
    if not _reference_runs_here():
        return
    _, _, world = _rank_env()
    # one oracle RHS on a 12^3-element p = 3 sample of the 64^3 workload per step
    n_side = 12
    code_steps = args.warmup + args.steps
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
from oracle import fr
from paper_2107_14027_gb300 import workloads as W
cfg = W.WORKLOADS[{WORKLOAD!r}]
n = ({n_side},) * 3
h = (cfg['hi'][0] - cfg['lo'][0]) / cfg['n'][0]
lo = (cfg['lo'][0],) * 3
hi = (cfg['lo'][0] + h * {n_side},) * 3
U = W.taylor_green(n, lo, hi, cfg['order'])
mesh = fr.Mesh(n, lo, hi)
prm = fr.Params(cfg['zeta'], cfg['nu'], cfg['t_r'])
ts = []
for i in range({code_steps}):
    t0 = time.perf_counter(); fr.rhs(U, mesh, cfg['order'], prm); ts.append(time.perf_counter() - t0)
print(json.dumps({{"t": sum(ts[{args.warmup}:]), "dof": U.size}}))
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    value = res["dof"] * args.steps / res["t"] / 1e9
    sample = f"FP64 oracle RHS on a {n_side}^3-element p=3 piece of the 64^3 TGV workload per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * res["t"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "order": 3, "mesh": [64, 64, 64], "nvars": 13},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def _time_loop(fn, stream, steps, warmup, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3  # seconds


def run_gpu(args):
    import torch
    rank, local_rank, world = _rank_env()
    torch.cuda.set_device(local_rank)
    dist = _init_dist("nccl")

    from paper_2107_14027_gb300 import abi
    from paper_2107_14027_gb300 import workloads as W
    cfg = W.WORKLOADS[WORKLOAD]
    n, order, nv = cfg["n"], cfg["order"], 13
    m = order + 1
    dof = int(np.prod(n)) * m ** 3 * nv

    # CPU baseline first (fresh processes; no GPU state inherited)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline_runs(16, 10.0)

    stream = torch.cuda.current_stream()
    U32 = W.taylor_green(n, cfg["lo"], cfg["hi"], order, dtype=np.float32)
    ctx = abi.fr_create(n, cfg["lo"], cfg["hi"], order, nv, cfg["zeta"], cfg["nu"], cfg["t_r"],
                        abi.FR_F32, abi.FR_CORR_DG)
    stride, ne, nbytes = abi.fr_layout(ctx)
    Ud = abi.pack_state(ctx, U32, abi.FR_F32)
    Rd = abi.new_state(ctx, abi.FR_F32)

    def step():
        abi.fr_rhs(ctx, Ud, Rd, stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # warm-up, then exactly --steps timed steps, clocks sampled meanwhile
    for _ in range(args.warmup):
        step()
    barrier()
    with ClockSampler(local_rank) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
        t_total = ev0.elapsed_time(ev1) / 1e3
        if args.steps * (t_total / max(args.steps, 1)) < 1.0:
            # keep the sampler alive for a few samples on very short runs
            time.sleep(0.5)
    t_max = _max_over_ranks(dist, t_total, "cuda")
    value = _job_rate(dof * args.steps, world, t_max) / 1e9

    # error of the timed output against the oracle on sampled elements
    # (mesh corners, the last tile, 250 seeded others): CPU-baseline leg
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(0)
        elems = np.unique(np.concatenate([[0, n[0] - 1, ne - n[0], ne - 1, (ne - 1) // 32 * 32],
                                          rng.choice(ne, 250, replace=False)]))
        idx = torch.as_tensor(elems, device="cuda")
        Rs = Rd[:, :ne].index_select(1, idx).cpu().numpy().astype(np.float64)
        err = _err_vs_oracle(U32, Rs.reshape(nv, m ** 3, len(elems)), n, cfg, elems)

    # per-kernel timing on the launching stream: the trace kernel alone
    # (fr_trace) and the fused kernel alone (fr_rhs_volume, reading the
    # traces of the same U)
    K = max(args.steps, 10)
    t_rhs_only = t_total / args.steps
    trace_s = _time_loop(lambda: abi.fr_trace(ctx, Ud, stream), stream, K, 2, torch) / K
    fused_s = _time_loop(lambda: abi.fr_rhs_volume(ctx, Ud, Rd, stream), stream, K, 2, torch) / K

    # algorithmic bytes of one fused launch (FP32), the method's own: read U
    # (n_v m^3 per element), write R (n_v m^3), and read the neighbours' face
    # traces of the 1 + 2d variables the normal flux needs on each of the 2d
    # faces (the paper's sparsity of the ACM-HD flux, Sec. 3).  The dense
    # model (all n_v variables on all faces, n_v (2 m^3 + 6 m^2)) is kept as
    # a second figure.
    d = 3
    alg_bytes = ne * (2 * nv * m ** 3 + 2 * d * (1 + 2 * d) * m ** 2) * 4
    dense_bytes = ne * nv * (2 * m ** 3 + 6 * m ** 2) * 4
    hbm, peak_kind = _peaks()
    achieved = alg_bytes / fused_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": _profiled_traffic(),
                "kernel": "fused_kernel<3,4,float>", "peak_source": peak_kind,
                "alg_bytes_per_launch": alg_bytes,
                "byte_model": "per element 4 (2 n_v m^3 + 2d (1+2d) m^2)",
                "dense_model": {"bytes_per_launch": dense_bytes,
                                "achieved": dense_bytes / fused_s / 1e9,
                                "frac": dense_bytes / fused_s / 1e9 / hbm,
                                "model": "per element 4 n_v (2 m^3 + 6 m^2)"}}
    # the whole RHS (trace + fused) on the same sparse model: U read twice,
    # R written, traces written and read once
    rhs_bytes = ne * (3 * nv * m ** 3 + 2 * 2 * d * (1 + 2 * d) * m ** 2) * 4
    rhs_roofline = {"bytes_per_rhs": rhs_bytes, "achieved": rhs_bytes / t_rhs_only / 1e9,
                    "frac": rhs_bytes / t_rhs_only / 1e9 / hbm}

    # unfused pipeline and FP64 fused, same stream
    t_unf = _time_loop(lambda: abi.fr_rhs_unfused(ctx, Ud, Rd, stream), stream, K, 2, torch) / K
    abi.fr_destroy(ctx)
    del Ud, Rd
    torch.cuda.empty_cache()

    U64 = U32.astype(np.float64)
    ctx64 = abi.fr_create(n, cfg["lo"], cfg["hi"], order, nv, cfg["zeta"], cfg["nu"], cfg["t_r"],
                          abi.FR_F64, abi.FR_CORR_DG)
    Ud64 = abi.pack_state(ctx64, U64, abi.FR_F64)
    Rd64 = abi.new_state(ctx64, abi.FR_F64)
    t64 = _time_loop(lambda: abi.fr_rhs(ctx64, Ud64, Rd64, stream), stream, max(K // 2, 5), 2,
                     torch) / max(K // 2, 5)
    t64_fused = _time_loop(lambda: abi.fr_rhs_volume(ctx64, Ud64, Rd64, stream), stream,
                           max(K // 2, 5), 2, torch) / max(K // 2, 5)
    abi.fr_destroy(ctx64)
    # the same RHS in the double-float mode (FP64 storage, ~48-bit arithmetic)
    ctxdf = abi.fr_create(n, cfg["lo"], cfg["hi"], order, nv, cfg["zeta"], cfg["nu"], cfg["t_r"],
                          abi.FR_DF64, abi.FR_CORR_DG)
    tdf = _time_loop(lambda: abi.fr_rhs(ctxdf, Ud64, Rd64, stream), stream, max(K // 2, 5), 2,
                     torch) / max(K // 2, 5)
    tdf_fused = _time_loop(lambda: abi.fr_rhs_volume(ctxdf, Ud64, Rd64, stream), stream,
                           max(K // 2, 5), 2, torch) / max(K // 2, 5)
    abi.fr_destroy(ctxdf)
    del Ud64, Rd64
    torch.cuda.empty_cache()
    # FMA peaks of this GPU (probe kernel), FP64 and FP32
    probe = {p: _fma_peak(abi, p, stream, torch) for p in (abi.FR_F64, abi.FR_F32)}
    # FP64 is arithmetic-bound on GB300: the fused kernel's algorithmic flops
    # (per point 42 m + 195: 21 flux components contracted along their axis,
    # 2 m flops each; corrections; flux and source) against the FP64 peak
    flops64 = ne * m ** 3 * (42 * m + 195)
    fp64_roofline = {"bound": "alu", "achieved": flops64 / t64_fused / 1e12,
                     "peak": probe[abi.FR_F64] / 1e12, "unit": "TFLOP/s",
                     "frac": flops64 / t64_fused / probe[abi.FR_F64],
                     "kernel": "fused_kernel<3,4,double>", "flops_per_launch": flops64,
                     "flop_model": "per point 42 m + 195",
                     "peak_source": "measured by the FMA probe kernel (fr_fma_probe)"}

    # end to end through the public host-buffer call
    ctx = abi.fr_create(n, cfg["lo"], cfg["hi"], order, nv, cfg["zeta"], cfg["nu"], cfg["t_r"],
                        abi.FR_F32, abi.FR_CORR_DG)
    stride, ne, nbytes = abi.fr_layout(ctx)
    Uh = torch.empty((nbytes // 4,), dtype=torch.float32, pin_memory=True)
    Uh.view(-1, stride)[:, :ne].copy_(torch.from_numpy(U32.reshape(-1, ne)))
    Rh = torch.empty_like(Uh).pin_memory()
    Ke = max(args.steps // 2, 3)
    for _ in range(2):
        abi.fr_rhs_host(ctx, Uh, Rh, stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        abi.fr_rhs_host(ctx, Uh, Rh, stream)
    barrier()
    te = time.perf_counter() - t0
    te_max = _max_over_ranks(dist, te, "cuda")
    e2e = {"value": _job_rate(dof * Ke, world, te_max) / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "call": "fr_rhs_host"}
    abi.fr_destroy(ctx)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "order": order, "mesh": list(n), "nvars": nv,
                       "elements": int(np.prod(n)), "dof": dof, "precision": "fp32",
                       "l2": "inputs larger than L2 (state 872 MB, traces 705 MB)",
                       "parallelism": f"replicas{world}"},
            "e2e": e2e,
            "roofline": roofline,
            "rhs_roofline": rhs_roofline,
            "kernels_ms": {"fused": 1e3 * fused_s, "trace": 1e3 * trace_s,
                           "rhs": 1e3 * t_rhs_only},
            "unfused": {"value": dof / t_unf / 1e9, "ms": 1e3 * t_unf,
                        "fused_speedup": t_unf / t_rhs_only},
            "fp64": {"value": dof / t64 / 1e9, "ms": 1e3 * t64, "fused_ms": 1e3 * t64_fused,
                     "roofline": fp64_roofline},
            "df64": {"value": dof / tdf / 1e9, "ms": 1e3 * tdf, "fused_ms": 1e3 * tdf_fused,
                     "speedup_over_fp64": t64 / tdf,
                     "arithmetic": "double-float (two FP32, ~48 bits), FP64 storage"},
            "fma_peak_tflops": {"fp64": probe[abi.FR_F64] / 1e12,
                                "fp32": probe[abi.FR_F32] / 1e12},
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
        }
        if err is not None:
            out["err_vs_oracle"] = err
        if cpu is not None:
            out["cpu_baseline"] = {
                "value": cpu["all"], "unit": "GDOF/s", "cores": cpu["cores"], "kind": "oracle",
                "cpu_model": _cpu_model(), "nproc": os.cpu_count(),
                "single_core": {"value": cpu["single"], "cores": 1, "reps": cpu["single_reps"],
                                "s_per_rhs": cpu["single_s"]},
                "sample": (f"FP64 numpy oracle RHS (sum-factorised) on a 16^3-element p=3 piece "
                           f"of the workload: one process per core ({cpu['cores']}), "
                           f"{cpu['all_reps']} RHS in {cpu['wall']:.1f} s; single core "
                           f"{cpu['single_reps']} RHS, {cpu['single_s']:.2f} s each")}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def _fma_peak(abi, precision, stream, torch):
    """FLOP/s of the FMA probe kernel, iterations sized to about 20 ms."""
    out = torch.zeros(152 * 8 * 8 * 4, dtype=torch.float64, device="cuda")
    iters = 64
    for _ in range(4):
        flops = abi.fr_fma_probe(precision, iters, out, stream)
        t = _time_loop(lambda: abi.fr_fma_probe(precision, iters, out, stream), stream, 3, 1,
                       torch) / 3
        if t > 0.01:
            break
        iters = int(iters * min(64.0, 0.02 / max(t, 1e-6)))
    t = _time_loop(lambda: abi.fr_fma_probe(precision, iters, out, stream), stream, 10, 2,
                   torch) / 10
    return flops / t


class _DualSolver:
    """One dual-time solver of the 3-D Taylor-Green workload: the stepping
    context (FP32 unless --dual-precision 64), an FP64 twin for the stretch
    below the FP32 rounding floor, and their pseudo solvers (P-multigrid
    cycles, with Anderson mixing in the FP64 phase, unless --dual-solver
    rk4)."""

    def __init__(self, abi, args, prec, U0, n, lo, hi, order):
        self.abi, self.args, self.prec = abi, args, prec
        zeta, nu, t_r = 2.5, 1.0 / 1600.0, 5e-3
        self.refine = prec == abi.FR_F32 and args.dual_tol < _TOL_SWITCH
        self.c = abi.fr_create(n, lo, hi, order, 13, zeta, nu, t_r, prec)
        twin = abi.FR_DF64 if args.dual_twin == "df64" else abi.FR_F64
        self.c64 = abi.fr_create(n, lo, hi, order, 13, zeta, nu, t_r, twin) if self.refine \
            else None
        self.U = abi.pack_state(self.c, U0, prec)
        self.U64 = abi.new_state(self.c64, abi.FR_F64) if self.refine else None
        self.pm = [None, None]
        if args.dual_solver != "rk4":
            factors = None
            if args.dual_pmg_factors:
                fs = [float(x) for x in args.dual_pmg_factors.split(",")]
                factors = {order - i: f for i, f in enumerate(fs)}
            for j, c in enumerate((self.c, self.c64)):
                if c is None:
                    continue
                self.pm[j] = abi.fr_pmg_create(c, 1)
                abi.fr_pmg_set_dtau(self.pm[j], factors, True)
                if (args.dual_pmg_bottom != 4 or args.dual_pmg_post != 7) and order > 1:
                    sched = [(q, 1) for q in range(order, 1, -1)] + [(1, args.dual_pmg_bottom)]
                    sched += [(q, 1) for q in range(2, order)] + [(order, args.dual_pmg_post)]
                    abi.fr_pmg_set_cycle(self.pm[j], sched)
                last = j == 1 or not self.refine
                if args.dual_solver == "pmg-aa" and last:
                    abi.fr_pmg_set_anderson(self.pm[j], args.dual_anderson)

    def step(self, dt, guess, cap, mlp=None):
        """One physical step; returns (status, stats, wall seconds)."""
        import torch
        a = self.args
        if a.dual_solver != "rk4":
            cap = max(1, cap // a.dual_pmg_iters_per_cycle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, s = self.abi.fr_dual_step(self.c, self.U, dt, a.dual_dtau, a.dual_tol, cap,
                                      check_every=5, guess=guess, refine=self.c64,
                                      U_refine=self.U64, tol_switch=_TOL_SWITCH, mlp=mlp,
                                      allow_noconv=True, pmg=self.pm[0], refine_pmg=self.pm[1])
        torch.cuda.synchronize()
        return st, s, time.perf_counter() - t0

    def destroy(self):
        for x in self.pm:
            if x is not None:
                self.abi.fr_pmg_destroy(x)
        self.abi.fr_destroy(self.c)
        if self.c64 is not None:
            self.abi.fr_destroy(self.c64)


_TOL_SWITCH = 5e-6


def _dual_case(args):
    n, order = (args.dual_mesh,) * 3, args.dual_order
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    return n, order, lo, hi


def _dual_config(args, workload, extra):
    cfg = {"workload": workload, "order": args.dual_order, "mesh": [args.dual_mesh] * 3,
           "dt": 1e-2, "bdf": 2, "tol": args.dual_tol, "tol_switch": _TOL_SWITCH,
           "dtau": args.dual_dtau, "solver": args.dual_solver,
           "pseudo": {"rk4": "classical RK4, fixed dtau (iters = RK4 steps)",
                      "pmg": "P-multigrid cycles p..1 (iters = cycles)",
                      "pmg-aa": "P-multigrid cycles p..1, Anderson mixing in the FP64 phase "
                                "(iters = cycles)"}[args.dual_solver],
           "anderson": args.dual_anderson if args.dual_solver == "pmg-aa" else 0,
           "fp64_twin": args.dual_twin,
           "pmg_factors": args.dual_pmg_factors or "1.75^(p-q)",
           "pmg_bottom_iterations": args.dual_pmg_bottom,
           "pmg_finest_post_iterations": args.dual_pmg_post}
    cfg.update(extra)
    return cfg


def _rec(k, st, s, wall):
    return {"step": k, "wall_s": wall, "iters": s.iters, "iters_fp64": s.iters_refine,
            "res": s.res, "res_switch": s.res_switch, "guess": s.guess_used,
            "res_guess": list(s.res_guess), "mlp_weight": s.mlp_weight,
            "res_blend": s.res_blend, "converged": st == 0}


def run_dual(args):
    """Learned vs plain initial guess on the dual-time workload (3-D p = 4,
    48^3 Taylor-Green, BDF2 dt = 1e-2, FP32 RHS with an FP64 twin below the
    FP32 floor, residual tolerance --dual-tol = 1e-6).  Solver A takes 3
    steps, then --dual-collect-steps more while element samples are
    collected; the network is trained (newest 10 % of the samples held out
    for validation, Adam with decoupled weight decay, the epoch count with
    the lowest validation loss kept by saving and reloading the network);
    then a fork B of A (same history) takes the held-out steps with the
    learned guess while A takes them with the plain extrapolation.  Metric:
    wall-seconds per held-out physical step (host clock around
    fr_dual_step, device synchronised)."""
    import tempfile
    import torch
    from paper_2107_14027_gb300 import abi
    from paper_2107_14027_gb300 import workloads as W
    n, order, lo, hi = _dual_case(args)
    prec = abi.FR_F64 if args.dual_precision == 64 else abi.FR_F32
    U0 = W.taylor_green(n, lo, hi, order, dtype=np.float32 if prec == abi.FR_F32 else np.float64)
    A = _DualSolver(abi, args, prec, U0, n, lo, hi, order)
    B = _DualSolver(abi, args, prec, U0, n, lo, hi, order)
    n_warm, n_collect, n_held = 3, args.dual_collect_steps, args.dual_held_steps
    per_step = max(1, args.dual_samples // n_collect)
    cap_samples = per_step * n_collect
    abi.fr_dual_init(A.c, A.U)
    net = abi.fr_mlp_create(A.c, args.dual_hidden, cap_samples, seed=2021)
    if args.dual_mlp_degree >= 0:
        abi.fr_mlp_set_output_degree(net, args.dual_mlp_degree)
    log = {"A": [], "B": []}

    def step(S, name, k, guess, cap, mlp=None):
        st, s, wall = S.step(1e-2, guess, cap, mlp)
        rec = _rec(k, st, s, wall)
        log[name].append(rec)
        print(json.dumps({"solver": name, **rec}), file=sys.stderr, flush=True)

    k = 0
    for _ in range(n_warm + n_collect):
        k += 1
        step(A, "A", k, abi.FR_GUESS_EXTRAPOLATE, args.dual_train_iters)
        if k > n_warm:
            abi.fr_mlp_collect(net, per_step, seed=1000 + k)
    # training: newest 10 % held out; keep the epoch count with the lowest
    # validation loss (saved and reloaded)
    n_val = max(1, cap_samples // 10)
    abi.fr_mlp_set_training(net, n_val, args.dual_wd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    curve, best = [], (float("inf"), 0)
    path = os.path.join(tempfile.mkdtemp(prefix="acmhd_mlp_"), "best.bin")
    loss0 = abi.fr_mlp_train(net, 1, args.dual_lr)
    done = 1
    while done < args.dual_epochs:
        chunk = min(args.dual_val_every, args.dual_epochs - done)
        tl = abi.fr_mlp_train(net, chunk, args.dual_lr)
        done += chunk
        vl = abi.fr_mlp_validation_loss(net)
        curve.append({"epochs": done, "train_loss": tl, "val_loss": vl})
        if vl < best[0]:
            best = (vl, done)
            abi.fr_mlp_save(net, path)
    if os.path.exists(path):
        abi.fr_mlp_destroy(net)
        net = abi.fr_mlp_load(A.c, path, capacity=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    abi.fr_dual_copy(B.c, A.c)
    for _ in range(n_held):
        k += 1
        step(A, "A", k, abi.FR_GUESS_EXTRAPOLATE, args.dual_held_iters)
        step(B, "B", k, abi.FR_GUESS_MLP, args.dual_held_iters, net)
    wa = float(np.mean([r["wall_s"] for r in log["A"][-n_held:]]))
    wb = float(np.mean([r["wall_s"] for r in log["B"]]))
    d = 3
    Va, Vb = abi.new_velocity(A.c, d, order), abi.new_velocity(B.c, d, order)
    abi.fr_dual_velocity(A.c, Va)
    abi.fr_dual_velocity(B.c, Vb)
    dv = float((Va - Vb).abs().max().item())
    out = {
        "metric": f"wall-s per physical step at {args.dual_tol:g} residual", "value": wb,
        "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "dtype": "f64" if prec == abi.FR_F64 else "f32+f64", "data": "synthetic",
        "config": _dual_config(args, f"hex_p{order}_{args.dual_mesh}cube_dual", {
            "max_iter_train_steps": args.dual_train_iters,
            "max_iter_held_steps": args.dual_held_iters,
            "mlp": {"hidden": args.dual_hidden, "samples": cap_samples, "validation": n_val,
                    "epochs": args.dual_epochs, "best_epochs": best[1], "lr": args.dual_lr,
                    "weight_decay": args.dual_wd, "output_degree": args.dual_mlp_degree,
                    "train_s": t_train, "loss_first": loss0,
                    "curve": curve}}),
        "plain_wall_s": wa, "learned_wall_s": wb, "speedup": wa / wb,
        "held_out_steps": n_held, "max_velocity_difference": dv,
        "steps": {"plain": log["A"], "learned": log["B"]},
    }
    print(json.dumps(out))
    abi.fr_mlp_destroy(net)
    A.destroy()
    B.destroy()


def run_dual_steps(args):
    """--dual-steps physical steps of the dual-time workload with the plain
    extrapolated guess (the workload's 200-step run), pseudo-iterations and
    wall-seconds per step logged; for the first --dual-fp64-ref steps an
    FP64-only solver (FP64 RHS, same solver otherwise) runs the same steps
    from the same initial state and the largest velocity difference between
    the two is logged: the error of the FP32 + FP64-twin result against an
    FP64 run."""
    import torch
    from paper_2107_14027_gb300 import abi
    from paper_2107_14027_gb300 import workloads as W
    n, order, lo, hi = _dual_case(args)
    prec = abi.FR_F64 if args.dual_precision == 64 else abi.FR_F32
    U0 = W.taylor_green(n, lo, hi, order, dtype=np.float32)
    S = _DualSolver(abi, args, prec, U0 if prec == abi.FR_F32 else U0.astype(np.float64), n, lo,
                    hi, order)
    abi.fr_dual_init(S.c, S.U)
    R = None
    if args.dual_fp64_ref > 0:
        R = _DualSolver(abi, args, abi.FR_F64, U0.astype(np.float64), n, lo, hi, order)
        abi.fr_dual_init(R.c, R.U)
    d = 3
    V, Vr = abi.new_velocity(S.c, d, order), (abi.new_velocity(R.c, d, order) if R else None)
    log = []
    for k in range(1, args.dual_steps + 1):
        st, s, wall = S.step(1e-2, abi.FR_GUESS_EXTRAPOLATE, args.dual_held_iters)
        rec = _rec(k, st, s, wall)
        if R is not None and k <= args.dual_fp64_ref:
            st64, s64, wall64 = R.step(1e-2, abi.FR_GUESS_EXTRAPOLATE, args.dual_held_iters)
            abi.fr_dual_velocity(S.c, V)
            abi.fr_dual_velocity(R.c, Vr)
            rec["fp64_ref"] = {"converged": st64 == 0, "iters": s64.iters, "wall_s": wall64,
                               "res": s64.res,
                               "max_velocity_error": float((V - Vr).abs().max().item()),
                               "rms_velocity_error": float(torch.sqrt(((V - Vr) ** 2).mean()))}
        log.append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)
    walls = [r["wall_s"] for r in log]
    out = {
        "metric": f"wall-s per physical step at {args.dual_tol:g} residual",
        "value": float(np.mean(walls)), "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "dtype": "f64" if prec == abi.FR_F64 else "f32+f64", "data": "synthetic",
        "config": _dual_config(args, f"hex_p{order}_{args.dual_mesh}cube_dual_steps",
                               {"steps": args.dual_steps, "fp64_reference_steps": args.dual_fp64_ref,
                                "max_iter": args.dual_held_iters}),
        "converged_steps": int(sum(r["converged"] for r in log)),
        "total_wall_s": float(np.sum(walls)),
        "max_fp64_velocity_error": max([r["fp64_ref"]["max_velocity_error"] for r in log
                                        if "fp64_ref" in r] or [None]),
        "steps": log,
    }
    print(json.dumps(out))
    S.destroy()
    if R is not None:
        R.destroy()


def run_profile_case(args):
    """A smaller copy of the workload (N^3 elements, same order and
    variables) for ncu captures: warm-up + steps fused RHS calls only."""
    import torch
    from paper_2107_14027_gb300 import abi
    from paper_2107_14027_gb300 import workloads as W
    cfg = W.WORKLOADS[WORKLOAD]
    n = (args.mesh,) * 3
    U = W.taylor_green(n, cfg["lo"], cfg["hi"], cfg["order"], dtype=np.float32)
    ctx = abi.fr_create(n, cfg["lo"], cfg["hi"], cfg["order"], 13, cfg["zeta"], cfg["nu"],
                        cfg["t_r"], abi.FR_F32, abi.FR_CORR_DG)
    Ud = abi.pack_state(ctx, U, abi.FR_F32)
    Rd = abi.new_state(ctx, abi.FR_F32)
    stream = torch.cuda.current_stream()
    t = _time_loop(lambda: abi.fr_rhs(ctx, Ud, Rd, stream), stream, args.steps, args.warmup, torch)
    abi.fr_destroy(ctx)
    dof = int(np.prod(n)) * 64 * 13
    print(json.dumps({"profile_case": f"hex_p3_{args.mesh}cube", "ms_per_rhs": 1e3 * t / args.steps,
                      "gdof_s": dof * args.steps / t / 1e9}))


def run_sweep(args):
    """Order sweep p = 1..6 on 3-D Taylor-Green meshes of about 38M points per
    variable (168^3 .. 48^3; 67^3 at p = 4), 13 variables, FP32: the fused
    RHS (trace + volume kernel) against the six unfused stage kernels, with
    each kernel's time and the fused RHS's fraction of the HBM roofline for
    its own minimum traffic (read U once, write R once, write and read the
    stored face traces once)."""
    import torch
    from paper_2107_14027_gb300 import abi
    from paper_2107_14027_gb300 import workloads as W
    peak, peak_src = _peaks()
    stream = torch.cuda.current_stream()
    rows = []
    orders = [int(x) for x in args.sweep_orders.split(",")]
    for order in orders:
        nside = W.ORDER_SWEEP_MESH[order]
        n = (nside,) * 3
        lo, hi = (-np.pi,) * 3, (np.pi,) * 3
        prec = abi.FR_F64 if args.sweep_precision == 64 else abi.FR_F32
        nside = args.sweep_mesh or nside
        n = (nside,) * 3
        U = W.taylor_green(n, lo, hi, order,
                           dtype=np.float64 if prec == abi.FR_F64 else np.float32)
        ctx = abi.fr_create(n, lo, hi, order, 13, 2.5, 1 / 1600, 5e-3, prec, 0)
        stride, ne, nbytes = abi.fr_layout(ctx)
        Ud = abi.pack_state(ctx, U, prec)
        Rd = abi.new_state(ctx, prec)
        K, Wm = args.steps, args.warmup
        t_rhs = _time_loop(lambda: abi.fr_rhs(ctx, Ud, Rd, stream), stream, K, Wm, torch) / K
        t_tr = _time_loop(lambda: abi.fr_trace(ctx, Ud, stream), stream, K, Wm, torch) / K
        t_vol = _time_loop(lambda: abi.fr_rhs_volume(ctx, Ud, Rd, stream), stream, K, Wm,
                           torch) / K
        Ku = max(2, K // 4)
        t_unf = _time_loop(lambda: abi.fr_rhs_unfused(ctx, Ud, Rd, stream), stream, Ku, 2,
                           torch) / Ku
        abi.fr_destroy(ctx)
        del Ud, Rd
        torch.cuda.empty_cache()
        m = order + 1
        dof = ne * m ** 3 * 13
        # own minimum of the two-kernel RHS: U read once, R written once, the
        # y/z face traces (7 slots, 4 faces) written and read once
        b = 8 if prec == abi.FR_F64 else 4
        own = ne * (2 * 13 * m ** 3 + 2 * 4 * 7 * m * m) * b
        rows.append({"order": order, "mesh": nside, "gdof_s": dof / t_rhs / 1e9,
                     "fused_tflops": ne * m ** 3 * (42 * m + 195) / t_vol / 1e12,
                     "unfused_gdof_s": dof / t_unf / 1e9, "fused_speedup": t_unf / t_rhs,
                     "ms": {"rhs": 1e3 * t_rhs, "trace": 1e3 * t_tr, "volume": 1e3 * t_vol,
                            "unfused": 1e3 * t_unf},
                     "own_min_gb": own / 1e9, "hbm_frac_own": own / t_rhs / 1e9 / peak})
    print(json.dumps({"metric": "GDOF-RHS/s, order sweep, fused vs unfused", "unit": "GDOF/s",
                      "higher_is_better": True, "n_gpus": 1,
                      "dtype": "f64" if args.sweep_precision == 64 else "f32", "data": "synthetic",
                      "steps": args.steps, "warmup": args.warmup, "peak_gbs": peak,
                      "peak_source": peak_src, "orders": rows}))


def run_mlp(args):
    """The network's GEMMs at the inference shapes of the dual-time workload
    (p = 4, 48^3: 110,592 elements, 4875 -> 256 -> 256 -> 1625 features):
    C[N x M] = W[N x K] . X[K x M] in BF16 with FP32 accumulation through
    fr_gemm_bf16, with the tensor-memory kernel (tcgen05, the default) and the
    warp-level mma.sync kernel, against the measured cuBLAS BF16 peak; then
    the backward orientations at the training shapes (5,000 samples), which
    the mma.sync kernels serve."""
    import torch
    from paper_2107_14027_gb300 import abi
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        pk = json.load(f)
    peak = float(pk.get("bf16_tflops", 1900.0))
    stream = torch.cuda.current_stream()
    M = 110592
    out = {}
    layers = [int(x) for x in args.mlp_layers.split(",") if x]
    kernels = [k for k in args.mlp_kernels.split(",") if k]
    shapes = {1: (256, 4875, 4880), 2: (256, 256, 256), 3: (1625, 256, 256)}
    for kind, label in ((abi.FR_GEMM_AUTO, "tcgen05"), (abi.FR_GEMM_MMA_SYNC, "mma_sync")):
        if label not in kernels:
            continue
        abi.fr_gemm_set_kernel(kind)
        rows, tot_flop, tot_s = [], 0.0, 0.0
        for N, K, lda in (shapes[li] for li in layers):
            W = torch.zeros(N, lda, device="cuda", dtype=torch.bfloat16)
            W[:, :K] = (torch.randn(N, K, device="cuda") * 0.05).to(torch.bfloat16)
            X = torch.randn(K, M, device="cuda").to(torch.bfloat16)
            C = torch.empty(N, M, device="cuda", dtype=torch.float32)
            fn = lambda: abi.fr_gemm_bf16(0, 0, N, M, K, W, lda, X, M, C, M, stream)
            t = _time_loop(fn, stream, args.steps, args.warmup, torch) / args.steps
            abi.fr_gemm_check(stream)
            ref = (W[:, :K].float() @ X.float())
            err = float((C - ref).abs().max() / ref.abs().max())
            flop = 2.0 * N * M * K
            rows.append({"N": N, "M": M, "K": K, "ms": 1e3 * t, "tflops": flop / t / 1e12,
                         "frac_of_measured_bf16": flop / t / 1e12 / peak,
                         "hbm_bytes_min": 2.0 * K * M + 2.0 * N * lda + 4.0 * N * M,
                         "max_rel_err_vs_fp32": err})
            tot_flop += flop
            tot_s += t
            del W, X, C, ref
        out[label] = {"tflops": tot_flop / tot_s / 1e12, "ms": 1e3 * tot_s, "layers": rows}
    # backward products of one training step at 5,000 samples
    n, bw = 5000, {}
    for kind, label in ((abi.FR_GEMM_AUTO, "tcgen05"), (abi.FR_GEMM_MMA_SYNC, "mma_sync")):
        if label not in kernels or layers != [1, 2, 3]:
            continue
        abi.fr_gemm_set_kernel(kind)
        rows = []
        for name, am, bm, N, Mo, K in (("dW1", 0, 1, 256, 4875, n), ("dH1", 1, 0, 256, n, 256),
                                        ("dW3", 0, 1, 1625, 256, n), ("dH2", 1, 0, 256, n, 1625)):
            A = (torch.randn(N, K, device="cuda") if am == 0 else
                 torch.randn(K, N, device="cuda")).to(torch.bfloat16)
            B = (torch.randn(K, Mo, device="cuda") if bm == 0 else
                 torch.randn(Mo, K, device="cuda")).to(torch.bfloat16)
            C = torch.empty(N, Mo, device="cuda", dtype=torch.float32)
            lda = K if am == 0 else N
            ldb = Mo if bm == 0 else K
            fn = lambda: abi.fr_gemm_bf16(am, bm, N, Mo, K, A, lda, B, ldb, C, Mo, stream)
            t = _time_loop(fn, stream, args.steps, args.warmup, torch) / args.steps
            abi.fr_gemm_check(stream)
            flop = 2.0 * N * Mo * K
            rows.append({"gemm": name, "N": N, "M": Mo, "K": K, "ms": 1e3 * t,
                         "tflops": flop / t / 1e12, "frac_of_measured_bf16": flop / t / 1e12 / peak})
            del A, B, C
        bw[label] = rows
    abi.fr_gemm_set_kernel(abi.FR_GEMM_AUTO)
    first = out.get("tcgen05") or out.get("mma_sync") or {"tflops": None}
    print(json.dumps({"metric": "BF16 GEMM TFLOP/s, MLP inference shapes", "unit": "TFLOP/s",
                      "value": first["tflops"], "higher_is_better": True, "n_gpus": 1,
                      "dtype": "bf16", "data": "synthetic", "steps": args.steps,
                      "warmup": args.warmup, "peak_tflops": peak, "peak_source": "measured",
                      "kernel": "tcgen05.mma kind::f16 128x256 tiles, TMEM accumulators, TMA",
                      "inference": out, "backward_training_5000": bw}))


def run_rk(args):
    """RK4 pseudo-steps (fr_rk_step) on an N^3 Taylor-Green mesh of order p,
    FP32: the fused-stage schedule (RK4 combination and next-stage traces in
    the volume kernel) against the separate trace + volume + update kernels.
    One pseudo-step is four RHS evaluations."""
    import torch
    from paper_2107_14027_gb300 import abi
    from paper_2107_14027_gb300 import workloads as W
    order = args.rk_order
    nside = args.rk_mesh or W.ORDER_SWEEP_MESH[order]
    n = (nside,) * 3
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    U = W.taylor_green(n, lo, hi, order, dtype=np.float32)
    ctx = abi.fr_create(n, lo, hi, order, 13, 2.5, 1 / 1600, 5e-3, abi.FR_F32, 0)
    stride, ne, _ = abi.fr_layout(ctx)
    stream = torch.cuda.current_stream()
    dof = ne * (order + 1) ** 3 * 13
    res, outs = {}, {}
    for name, sched in (("fused_stage", abi.FR_SCHEDULE_FUSED_STAGE),
                        ("separate", abi.FR_SCHEDULE_TWO_KERNELS)):
        abi.fr_set_schedule(ctx, sched)
        Ud = abi.pack_state(ctx, U, abi.FR_F32)
        abi.fr_rk_step(ctx, Ud, 1e-4, stream)
        outs[name] = Ud.clone()
        for _ in range(args.warmup):
            abi.fr_rk_step(ctx, Ud, 1e-4, stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            abi.fr_rk_step(ctx, Ud, 1e-4, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        res[name] = {"ms_per_step": ms, "gdof_s": 4 * dof / ms / 1e6}
    same = bool(torch.equal(outs["fused_stage"][:, :ne], outs["separate"][:, :ne]))
    abi.fr_destroy(ctx)
    auto = "fused_stage" if order <= 2 else "separate"
    print(json.dumps({
        "metric": "GDOF-RHS/s in RK4 pseudo-steps (4 RHS per step)", "value": res[auto]["gdof_s"],
        "unit": "GDOF/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"hex_p{order}_{nside}cube_rk4", "order": order, "mesh": list(n),
                   "auto_schedule": auto},
        "fused_stage": res["fused_stage"], "separate": res["separate"],
        "fused_over_separate": res["separate"]["ms_per_step"] / res["fused_stage"]["ms_per_step"],
        "bitwise_equal_after_one_step": same}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mesh", type=int, default=None,
                    help="profiling only: run fr_rhs on an N^3 mesh and print its timing")
    ap.add_argument("--workload", default="rhs",
                    choices=["rhs", "dual", "dual-steps", "rk", "sweep", "mlp"],
                    help="rhs: the fused RHS (default); dual: BDF2 dual time stepping, "
                         "plain vs learned initial guess; dual-steps: N dual-time steps with "
                         "the plain guess, error against an FP64 run; rk: RK4 pseudo-steps, fused "
                         "stage vs separate update; sweep: orders 1..6, fused vs unfused; "
                         "mlp: the network's tensor-core GEMMs")
    ap.add_argument("--sweep-orders", default="1,2,3,4,5,6")
    ap.add_argument("--sweep-precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--sweep-mesh", type=int, default=0,
                    help="elements per direction for every order (default: ~38M points)")
    ap.add_argument("--mlp-layers", default="1,2,3",
                    help="mlp workload: which inference layers to time (1, 2, 3)")
    ap.add_argument("--mlp-kernels", default="tcgen05,mma_sync",
                    help="mlp workload: GEMM kernels to time")
    ap.add_argument("--rk-order", type=int, default=3)
    ap.add_argument("--rk-mesh", type=int, default=None,
                    help="elements per direction (default: the order sweep's mesh)")
    ap.add_argument("--dual-mesh", type=int, default=48)
    ap.add_argument("--dual-order", type=int, default=4)
    ap.add_argument("--dual-dtau", type=float, default=1e-3)
    ap.add_argument("--dual-precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--dual-hidden", type=int, default=256)
    ap.add_argument("--dual-lr", type=float, default=1e-3)
    ap.add_argument("--dual-collect-steps", type=int, default=8)
    ap.add_argument("--dual-held-steps", type=int, default=5)
    ap.add_argument("--dual-samples", type=int, default=5000)
    ap.add_argument("--dual-epochs", type=int, default=400)
    ap.add_argument("--dual-train-iters", type=int, default=1200,
                    help="pseudo-iteration cap of the steps before the held-out ones")
    ap.add_argument("--dual-held-iters", type=int, default=1200,
                    help="pseudo-iteration cap of the held-out steps")
    ap.add_argument("--dual-solver", default="pmg-aa", choices=["rk4", "pmg", "pmg-aa"],
                    help="pseudo solver: RK4 steps, P-multigrid cycles, or cycles with "
                         "Anderson mixing in the FP64 phase (default)")
    ap.add_argument("--dual-twin", default="f64", choices=["df64", "f64"],
                    help="arithmetic of the FP64 twin below the FP32 floor: double-float "
                         "(FP64 storage, ~48-bit arithmetic on the FP32 pipes) or FP64")
    ap.add_argument("--dual-pmg-factors", default="",
                    help="pseudo-step multipliers for orders p, p-1, .., 1 (default 1.75^(p-q))")
    ap.add_argument("--dual-anderson", type=int, default=8, help="Anderson memory (pmg-aa)")
    ap.add_argument("--dual-pmg-post", type=int, default=1,
                    help="RK4 iterations on the finest order on the way up a cycle (the "
                         "paper's cycle: 7)")
    ap.add_argument("--dual-pmg-bottom", type=int, default=32,
                    help="iterations on order 1 per cycle (the paper's cycle: 4; measured "
                         "better: 32 with one on the finest order going up)")
    ap.add_argument("--dual-pmg-iters-per-cycle", type=int, default=10,
                    help="fine-iteration equivalents of one cycle, to turn the iteration "
                         "caps into cycle caps")
    ap.add_argument("--dual-wd", type=float, default=1e-2, help="weight decay of the network")
    ap.add_argument("--dual-mlp-degree", type=int, default=-1,
                    help="project the learned corrections onto degree <= q per element (-1: off)")
    ap.add_argument("--dual-val-every", type=int, default=25,
                    help="epochs between validation-loss checks")
    ap.add_argument("--dual-steps", type=int, default=200,
                    help="physical steps of --workload dual-steps")
    ap.add_argument("--dual-fp64-ref", type=int, default=0,
                    help="dual-steps: run an FP64-only solver beside for this many steps")
    ap.add_argument("--dual-tol", type=float, default=1e-6,
                    help="residual tolerance; below the FP32 floor (5e-6) an FP64 twin refines")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mesh is not None:
        run_profile_case(args)
    elif args.workload == "dual":
        run_dual(args)
    elif args.workload == "dual-steps":
        run_dual_steps(args)
    elif args.workload == "rk":
        run_rk(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "mlp":
        run_mlp(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
