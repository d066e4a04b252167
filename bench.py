"""Benchmark of the Moebius domain-wall hopping kernel (Dhop) on GB300.

Workload: Moebius DWF (M5 = 1.8, b = 1.5, c = 0.5) Dhop at 32^3 x 64 x Ls = 12,
FP32 storage, one right-hand side, links U = exp(i 0.3 H), Gaussian source,
seed 5.  One step = one application of Dhop to the whole 5D field (the paper's
"Domain Wall kernel", 1320 flop per 5D site update, Table 3).

Prints one JSON line: throughput in GFlop/s (1320-flop convention), the HBM
roofline of the kernel against the measured copy bandwidth, an end-to-end
figure through the host-buffer C entry point, the CPU oracle as a baseline,
and the SM clocks sampled during the timed region.  The fused D, D^+ and
D^+D applies, the FP16-storage Dhop and the Wilson Dslash (the same kernel at
Ls = 1) are timed too and reported under "ops"; "batched" is the 12-RHS
workload at 16^3 x 32 x 12, "cg" the FP64 / mixed CG on D^+D at 24^4 x 16 and
"cg_eo" the even-odd preconditioned solve of D x = eta on the same lattice
(--no-cg skips those; --cg-full adds the CGs on the benchmark lattice).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Möbius DWF Dhop GFlop/s & % HBM roofline; mixed vs FP64 CG time to 1e-10"
DIMS = (32, 32, 32, 64)
LS = 12
M5, B, C = 1.8, 1.5, 0.5
MF = 0.01
SEED = 5
FLOP_DHOP = 1320           # per 5D site update (Table 3)
FLOP_D_MOBIUS = 1320 + 192  # + (b + cK) on the input (3 x 24) and the diagonal (5 x 24)


def bytes_per_site(real_bytes: int, Ls: int, nrhs: int = 1) -> float:
    """Algorithmic HBM bytes per 5D site update: read psi once (24 reals), write
    once (24 reals), 4 links x 18 reals per 4D site shared by Ls*nrhs updates."""
    return real_bytes * (48 + 72.0 / (Ls * nrhs))


# DRAM traffic of one Dhop launch, from a one-pass ncu capture of the full-size
# workload (dram__bytes_read.sum + dram__bytes_write.sum).  The record names the
# tile it was taken with and a digest of the stencil sources; when either no
# longer matches, the traffic is reported as null.
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "dslash_dhop_f32_32x32x32x64_ls12_dram.md")


def kernel_digest() -> str:
    """sha256 (first 16 hex digits) over the code of the stencil kernel sources:
    comments and whitespace are left out, so only a change of the code voids a
    traffic record."""
    csrc = os.path.join(ROOT, "paper_2112_01852_gb300", "csrc")
    names = sorted(n for n in os.listdir(csrc)
                   if n.startswith("dw_dslash") or n == "dw_common.cuh")
    h = hashlib.sha256()
    for n in names:
        h.update(n.encode())
        with open(os.path.join(csrc, n), encoding="utf-8") as f:
            code = f.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(tile, dims, Ls):
    """Bytes per launch from the traffic record if it applies to this kernel,
    tile and workload, else None."""
    try:
        with open(TRAFFIC_RECORD) as f:
            kv = dict(m.groups() for m in re.finditer(r"^- (\w+): (.+?)\s*$", f.read(), re.M))
        rec_tile = tuple(int(v) for v in kv["tile"].split(","))
        rec_dims = tuple(int(v) for v in kv["dims"].split(","))
        if (rec_tile != tuple(tile) or rec_dims != tuple(dims) or int(kv["Ls"]) != Ls
                or kv["source_digest"] != kernel_digest()):
            return None
        return float(kv["dram_read_bytes"]) + float(kv["dram_write_bytes"])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper half of the observed clocks
        loaded = [v for v in sm if v >= 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as tdist
        tdist.barrier()


def _max_over_ranks(ws, v):
    """Max of a host scalar over the ranks (NCCL: via a CUDA tensor; gloo: CPU)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as tdist
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ws, ms_local, units_local):
    """Whole-job figure of N independent replicas: every rank processes
    units_local units in ms_local; the job takes the slowest rank's time."""
    ms = _max_over_ranks(ws, ms_local)
    return ms, units_local * ws / (ms * 1e-3)


def time_op(fn, steps, warmup, stream):
    """Mean ms per call over `steps` calls with CUDA events on `stream`."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def time_op_flushed(fn, steps, warmup, stream, flush):
    """Mean ms per call over `steps` calls, each timed alone with CUDA events on
    `stream` after `flush` (a device buffer larger than L2) has been rewritten, so
    that no input of the call is L2-resident when it starts."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def paper_context():
    """The paper's Domain Wall kernel rates on one A64FX node (Table 2, Sec. 4.2),
    from the committed fixture: context for the GPU figures, not a target."""
    path = os.path.join(ROOT, "tests", "golden", "table2_dwf_gflops.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t) for t in line.split()]
            rows.append({"dims": v[:4], "Ls": v[4], "dp_1rank": v[5], "sp_1rank": v[6],
                         "dp_4ranks": v[7], "sp_4ranks": v[8]})
    return {"hardware": "one A64FX node (QPACE 4), 48 cores, HBM2 1 TB/s",
            "unit": "GFlop/s", "source": "Table 2", "domain_wall_kernel": rows}


def cpu_baseline(psi, U, budget_s=12.0):
    """The FP64 oracle's Dhop on the host cores: whole-lattice applies until the
    time budget is spent (at least one)."""
    import oracle
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.dhop(psi, U, DIMS, LS)
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = (time.perf_counter() - t0) / n
    V5 = int(np.prod(DIMS)) * LS
    return {"value": FLOP_DHOP * V5 / dt / 1e9, "unit": "GFlop/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d whole-lattice FP64 Dhop apply(s) at 32^3x64xLs12 (%.1f s each)" % (n, dt)}


def oracle_timings(psi, U, budget_s=6.0):
    """The FP64 oracle's D on the host cores at the benchmark lattice (whole-
    lattice applies until the time budget is spent), and its CG on D^+D to 1e-10
    at 4^4 x Ls=8 (the small lattice whose oracle CG finishes in a second):
    context beside the GPU numbers, not a target."""
    import oracle
    from paper_2112_01852_gb300 import inputs
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.dw(psi, U, DIMS, LS, M5, B, C, [MF])
        n += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = (time.perf_counter() - t0) / n
    V5 = int(np.prod(DIMS)) * LS
    dims1, ls1 = (4, 4, 4, 4), 8
    U1 = inputs.exp_su3_field(dims1, seed=1)
    b1 = inputs.gaussian_fermion(dims1, ls1, 1, seed=1)
    t1 = time.perf_counter()
    x1, iters, res = oracle.cg(b1, U1, dims1, ls1, M5, B, C, [MF], tol=1e-10)
    cg_s = time.perf_counter() - t1
    return {"cores": oracle.num_threads(), "kind": "oracle",
            "D": {"value": FLOP_D_MOBIUS * V5 / dt / 1e9, "unit": "GFlop/s",
                  "sample": "%d whole-lattice FP64 Moebius D apply(s) at %sxLs%d "
                            "(%.1f s each)" % (n, "x".join(str(d) for d in DIMS), LS, dt)},
            "cg_4x4x4x4_ls8": {"seconds": cg_s, "iters": int(_first(iters)),
                               "resid": float(_first(res)), "tol": 1e-10}}


def _first(v):
    return v[0] if isinstance(v, (list, tuple, np.ndarray)) else v


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload, each step a bounded
    sample of the lattice (a fixed set of 4D sites, all slices)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2112_01852_gb300 import inputs
    oracle.build()
    V4 = int(np.prod(DIMS))
    U = inputs.exp_su3_field(DIMS, seed=SEED)
    psi = inputs.gaussian_fermion(DIMS, LS, 1, seed=SEED)
    nsite = min(65536, V4)  # 4D sites per step (x Ls = 786432 site updates at full size)
    rng = np.random.default_rng(0)
    sites = np.sort(rng.choice(V4, size=nsite, replace=False))
    for _ in range(args.warmup):
        oracle.dhop(psi, U, DIMS, LS, sites=sites)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dhop(psi, U, DIMS, LS, sites=sites)
    dt = (time.perf_counter() - t0) / args.steps
    val = FLOP_DHOP * nsite * LS / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFlop/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(),
        "cpu_baseline": {"value": val, "unit": "GFlop/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "%d random 4D sites x Ls=%d per step of the %s lattice"
                                   % (nsite, LS, "x".join(str(d) for d in DIMS))},
        "e2e": {"value": val, "unit": "GFlop/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


CG_DIMS, CG_LS, CG_SEED = (24, 24, 24, 24), 16, 3
BATCH_DIMS, BATCH_LS, BATCH_SEED = (16, 16, 16, 32), 12, 4
BATCH_MASSES = [0.005] * 5 + [0.01] * 4 + [0.02] * 2 + [0.05]


def _warm(solve, x):
    """One short solve (a few iterations) before the timed one: the solver tunes
    the tiles of its inner operator on first use and keeps them per lattice, so
    the timed solve measures the solve alone.  Returns its wall time (tuning
    included)."""
    import torch
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solve(x, 3)
    return time.perf_counter() - t0


def bench_cg(args, dims=None, Ls=None, seed=None):
    """CG on D^+D x = b to a true residual of 1e-10 (default 24^4 x Ls=16, m_f =
    0.01): plain FP64 against mixed FP32 and mixed FP16-storage, wall time of the
    whole dw_cg_solve call; every solution's residual is recomputed by the oracle."""
    import oracle
    import torch
    from paper_2112_01852_gb300 import dw, inputs
    from paper_2112_01852_gb300.lattice import Lattice
    dims = CG_DIMS if dims is None else dims
    Ls = CG_LS if Ls is None else Ls
    seed = CG_SEED if seed is None else seed
    U = inputs.exp_su3_field(dims, seed=seed)
    rhs = inputs.gaussian_fermion(dims, Ls, 1, seed=seed)
    lat = Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F64)
    lat.load_gauge(U)
    bdev = lat.pack(rhs)
    out = {"workload": "mobius_cg_%s_ls%d_mf%g" % ("x".join(str(d) for d in dims), Ls, MF),
           "tol": 1e-10}
    for name, mode in (("f64", dw.DW_F64), ("mixed_f32", dw.DW_F32), ("mixed_f16", dw.DW_F16)):
        x = lat.empty(1)
        warm = _warm(lambda v, n: lat.cg(v, bdev, [MF], nrhs=1, tol=1e-10, maxit=n, mode=mode),
                     x)
        x.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("cg_%s" % name)
        t0 = time.perf_counter()
        status, stats = lat.cg(x, bdev, [MF], nrhs=1, tol=1e-10, maxit=40000, mode=mode)
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        xs = lat.unpack(x)
        Ax = oracle.dwdagdw(xs, U, dims, Ls, M5, B, C, [MF])
        res = float(np.linalg.norm((rhs - Ax).ravel()) / np.linalg.norm(rhs.ravel()))
        out[name] = {"seconds": wall, "first_call_seconds": warm, "status": status,
                     "iters": stats[0].iters, "reliable_updates": stats[0].reliable_updates,
                     "converged": stats[0].converged, "true_resid": stats[0].true_resid,
                     "oracle_resid": res}
        del x
    out["speedup_mixed_f32"] = out["f64"]["seconds"] / out["mixed_f32"]["seconds"]
    out["speedup_mixed_f16"] = out["f64"]["seconds"] / out["mixed_f16"]["seconds"]
    lat.close()
    return out


def bench_eo(args, dims=None, Ls=None, seed=None, f64=True):
    """D x = eta (default 24^4 x Ls=16, m_f = 0.01) to 1e-10: even-odd
    preconditioned CG (FP64 unless f64 is False, mixed FP32 / FP16) against plain
    mixed-FP32 CG on D^+D x = D^+ eta; every solution's residual |eta - D x| / |eta|
    is recomputed by the oracle."""
    import oracle
    import torch
    from paper_2112_01852_gb300 import dw, inputs
    from paper_2112_01852_gb300.lattice import Lattice
    dims = CG_DIMS if dims is None else dims
    Ls = CG_LS if Ls is None else Ls
    seed = CG_SEED if seed is None else seed
    U = inputs.exp_su3_field(dims, seed=seed)
    eta = inputs.gaussian_fermion(dims, Ls, 1, seed=seed)
    lat = Lattice(dims, Ls, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F64)
    lat.load_gauge(U)
    e = lat.pack(eta)
    out = {"workload": "mobius_solve_D_%s_ls%d_mf%g" % ("x".join(str(d) for d in dims),
                                                         Ls, MF), "tol": 1e-10}

    def resid(x):
        r = oracle.dw(lat.unpack(x), U, dims, Ls, M5, B, C, [MF]) - eta
        return float(np.linalg.norm(r.ravel()) / np.linalg.norm(eta.ravel()))

    modes = (("eo_f64", dw.DW_F64),) if f64 else ()
    for name, mode in modes + (("eo_mixed_f32", dw.DW_F32), ("eo_mixed_f16", dw.DW_F16)):
        x = lat.empty(1)
        warm = _warm(lambda v, n: lat.solve_eo(v, e, [MF], nrhs=1, tol=1e-10, maxit=n,
                                               mode=mode), x)
        x.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("solve_%s" % name)
        t0 = time.perf_counter()
        status, stats = lat.solve_eo(x, e, [MF], nrhs=1, tol=1e-10, maxit=40000, mode=mode)
        wall = time.perf_counter() - t0
        torch.cuda.nvtx.range_pop()
        out[name] = {"seconds": wall, "first_call_seconds": warm, "status": status,
                     "iters": stats[0].iters,
                     "reliable_updates": stats[0].reliable_updates,
                     "true_resid": stats[0].true_resid, "oracle_resid": resid(x)}
        del x
    # the same system without preconditioning: CG on D^+D x = D^+ eta.  Its stopping
    # test is on the normal equations, so its tolerance is lowered (and the solve
    # rerun from zero) until the residual of D x = eta itself is at most 1e-10, the
    # target the even-odd solve meets; the last, successful solve is the one timed.
    b = lat.empty(1)
    dw.dw_apply_Ddag(lat.handle, b.data_ptr(), e.data_ptr(), [MF], 1)
    y = lat.empty(1)
    _warm(lambda v, n: lat.cg(v, b, [MF], nrhs=1, tol=1e-10, maxit=n, mode=dw.DW_F32), y)
    tol_u = 1e-10
    for _ in range(5):
        y.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status, stats = lat.cg(y, b, [MF], nrhs=1, tol=tol_u, maxit=40000, mode=dw.DW_F32)
        wall = time.perf_counter() - t0
        r_full = resid(y)
        if r_full <= 1e-10:
            break
        tol_u *= max(1e-3, min(0.5, 0.5 * 1e-10 / r_full))
    out["unprec_mixed_f32"] = {"seconds": wall, "status": status, "iters": stats[0].iters,
                               "cg_tol": tol_u, "oracle_resid": r_full}
    out["speedup_eo_vs_unprec_mixed_f32"] = wall / out["eo_mixed_f32"]["seconds"]
    lat.close()
    return out


def bench_batched(args):
    """12 right-hand sides over 4 masses (5/4/2/1) at 16^3 x 32 x Ls=12, FP32:
    one batched Dhop / D^+D launch per step, and one batched mixed-FP32 CG solve
    of all 12 systems (residuals recomputed by the oracle)."""
    import oracle
    import torch
    from paper_2112_01852_gb300 import dw, inputs
    from paper_2112_01852_gb300.lattice import Lattice
    nrhs = len(BATCH_MASSES)
    U = inputs.exp_su3_field(BATCH_DIMS, seed=BATCH_SEED)
    rhs = inputs.gaussian_fermion(BATCH_DIMS, BATCH_LS, nrhs, seed=BATCH_SEED)
    V5 = int(np.prod(BATCH_DIMS)) * BATCH_LS
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    lat = Lattice(BATCH_DIMS, BATCH_LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F32)
    lat.load_gauge(U)
    x = lat.pack(rhs)
    y = lat.empty(nrhs)
    tile = lat.tune(dw.DW_OP_DHOP, nrhs)
    ms = time_op(lambda: dw.dw_apply_Dhop(lat.handle, y.data_ptr(), x.data_ptr(), nrhs, sh),
                 max(5, args.steps // 2), 3, stream)
    bps = bytes_per_site(4, BATCH_LS, nrhs)
    out = {"workload": "mobius_batched_16x16x16x32_ls12_12rhs_f32", "nrhs": nrhs,
           "masses": BATCH_MASSES, "dhop": {"ms": ms, "gflops": FLOP_DHOP * V5 * nrhs / ms / 1e6,
                                            "gbs": bps * V5 * nrhs / ms / 1e6, "tile": tile}}
    ms2 = time_op(lambda: dw.dw_apply_DdagD(lat.handle, y.data_ptr(), x.data_ptr(),
                                            BATCH_MASSES, nrhs, sh), max(5, args.steps // 4), 3,
                  stream)
    out["ddagd"] = {"ms": ms2, "gflops": 2 * FLOP_D_MOBIUS * V5 * nrhs / ms2 / 1e6}
    lat.close()
    del x, y
    lat = Lattice(BATCH_DIMS, BATCH_LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F64)
    lat.load_gauge(U)
    bdev = lat.pack(rhs)
    xs = lat.empty(nrhs)
    _warm(lambda v, n: lat.cg(v, bdev, BATCH_MASSES, nrhs=nrhs, tol=1e-10, maxit=n,
                              mode=dw.DW_F32), xs)
    xs.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, stats = lat.cg(xs, bdev, BATCH_MASSES, nrhs=nrhs, tol=1e-10, maxit=40000,
                           mode=dw.DW_F32)
    wall = time.perf_counter() - t0
    sol = lat.unpack(xs, nrhs)
    Ax = oracle.dwdagdw(sol, U, BATCH_DIMS, BATCH_LS, M5, B, C, BATCH_MASSES)
    res = [float(np.linalg.norm((rhs[r] - Ax[r]).ravel()) / np.linalg.norm(rhs[r].ravel()))
           for r in range(nrhs)]
    out["cg_mixed_f32"] = {"seconds": wall, "status": status,
                           "iters": [s.iters for s in stats],
                           "reliable_updates": [s.reliable_updates for s in stats],
                           "max_oracle_resid": max(res)}
    # the same 12 systems solved one after another (one RHS per solve)
    seq, seq_res, seq_iters = 0.0, [], []
    one = lat.empty(1)
    _warm(lambda v, n: lat.cg(v, lat.pack(rhs[0]), [BATCH_MASSES[0]], nrhs=1, tol=1e-10,
                              maxit=n, mode=dw.DW_F32), one)
    for r in range(nrhs):
        br = lat.pack(rhs[r])
        one.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st1 = lat.cg(one, br, [BATCH_MASSES[r]], nrhs=1, tol=1e-10, maxit=40000,
                        mode=dw.DW_F32)
        seq += time.perf_counter() - t0
        seq_iters.append(st1[0].iters)
        sol1 = lat.unpack(one)
        A1 = oracle.dwdagdw(sol1, U, BATCH_DIMS, BATCH_LS, M5, B, C, [BATCH_MASSES[r]])
        seq_res.append(float(np.linalg.norm((rhs[r] - A1[0]).ravel())
                             / np.linalg.norm(rhs[r].ravel())))
    out["cg_sequential_mixed_f32"] = {"seconds": seq, "iters": seq_iters,
                                      "max_oracle_resid": max(seq_res)}
    out["batched_over_sequential_time"] = wall / seq
    lat.close()
    return out


def _config():
    name = "mobius_dwf_dhop_%s_ls%d_f32" % ("x".join(str(d) for d in DIMS), LS)
    return {"workload": name, "dims": list(DIMS), "Ls": LS,
            "nrhs": 1, "kind": "mobius", "M5": M5, "b": B, "c": C, "mf": MF,
            "links": "exp(i 0.3 H)", "seed": SEED, "prec": "f32",
            "l2": "inputs larger than L2 (2.42 GB FP32 field vs 129 MB L2)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dims", default=None,
                    help="Lx,Ly,Lz,Lt override (profiling runs on a smaller lattice)")
    ap.add_argument("--Ls", type=int, default=None)
    ap.add_argument("--main-only", action="store_true",
                    help="time only the FP32 Dhop (no other operators, e2e, CG or CPU leg)")
    ap.add_argument("--tile", default=None,
                    help="spt,tx[,variant[,zblk[,sgrp]]]: fixed Dhop tile instead of tuning")
    ap.add_argument("--layout", default="spin_pair", choices=["spin_pair", "complex"],
                    help="FP32 quad layout of the timed Dhop (complex: the interleaved-"
                         "complex layout of the ablation)")
    ap.add_argument("--prec", default="f32", choices=["f32", "f16"],
                    help="storage of the timed Dhop with --main-only (profiling runs)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="right-hand sides of the timed Dhop with --main-only (profiling runs)")
    ap.add_argument("--op", default="dhop", choices=["dhop", "d", "ddag"],
                    help="operator timed with --main-only (profiling runs; --tile applies "
                         "to it): the hopping term, D or D^+ at mass m_f")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--solvers-only", action="store_true",
                    help="run only the CG and even-odd solver legs (profiling runs); "
                         "prints their JSON")
    ap.add_argument("--cg-full", action="store_true",
                    help="also run the three CGs on the benchmark lattice (minutes)")
    args = ap.parse_args()
    if not args.main_only and (args.prec != "f32" or args.nrhs != 1 or args.op != "dhop"):
        ap.error("--prec, --nrhs and --op apply to --main-only runs")
    global DIMS, LS
    if args.dims:
        DIMS = tuple(int(v) for v in args.dims.split(","))
    if args.Ls:
        LS = args.Ls
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2112_01852_gb300 import build as cuda_build
    from paper_2112_01852_gb300 import dw, inputs
    from paper_2112_01852_gb300.lattice import Lattice
    cuda_build.build()
    if args.solvers_only:
        out = {"cg": bench_cg(args), "cg_eo": bench_eo(args)}
        if args.cg_full:
            out["cg_full"] = bench_cg(args, DIMS, LS, SEED)
            out["cg_eo_full"] = bench_eo(args, DIMS, LS, SEED, f64=False)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0

    NR = args.nrhs
    prec = dw.DW_F16 if args.prec == "f16" else dw.DW_F32
    V4 = int(np.prod(DIMS))
    V5 = V4 * LS
    U = inputs.exp_su3_field(DIMS, seed=SEED)
    psi = inputs.gaussian_fermion(DIMS, LS, NR, seed=SEED)

    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    lat = Lattice(DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=prec)
    lat.load_gauge(U)
    if args.layout == "complex":
        dw.dw_set_complex_layout(lat.handle, 1)
    x = lat.pack(psi)
    y = lat.empty(NR)
    tiles = {}
    main_op = {"dhop": dw.DW_OP_DHOP, "d": dw.DW_OP_D, "ddag": dw.DW_OP_DDAG}[args.op]
    if args.tile:
        tv = [int(v) for v in args.tile.split(",")] + [0, 0, 1][len(args.tile.split(",")) - 2:]
        spt, tx, var, zb, sg = tv[:5]
        lat.set_tile(main_op, spt, tx, var, nrhs=NR, zblk=zb, sgrp=sg)
        tiles[main_op] = (spt, tx, var, zb, sg)
    else:
        tiles[main_op] = lat.tune(main_op, NR)
    if not args.main_only:
        for op in (dw.DW_OP_D, dw.DW_OP_DDAG):
            tiles[op] = lat.tune(op, 1)

    mfs = [MF] * NR
    if main_op == dw.DW_OP_DHOP:
        def dhop():
            dw.dw_apply_Dhop(lat.handle, y.data_ptr(), x.data_ptr(), NR, sh)
    elif main_op == dw.DW_OP_D:  # profiling runs of the other operators (--main-only)
        def dhop():
            dw.dw_apply_D(lat.handle, y.data_ptr(), x.data_ptr(), mfs, NR, sh)
    else:
        def dhop():
            dw.dw_apply_Ddag(lat.handle, y.data_ptr(), x.data_ptr(), mfs, NR, sh)

    # warm-up and timed region (barrier + synchronize on both sides)
    for _ in range(args.warmup):
        dhop()
    torch.cuda.synchronize()
    _barrier(ws)
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("dhop_timed")
    e0.record(stream)
    for _ in range(args.steps):
        dhop()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    _barrier(ws)
    clocks = sampler.stop()
    ms, sites_per_s = aggregate(ws, e0.elapsed_time(e1) / args.steps, V5 * NR)
    gflops = (FLOP_DHOP if main_op == dw.DW_OP_DHOP else FLOP_D_MOBIUS) * sites_per_s / 1e9

    # roofline of the Dhop kernel (one launch per step)
    peak, peak_kind = _peaks()
    bps = bytes_per_site(2 if prec == dw.DW_F16 else 4, LS, NR)
    alg_bytes = bps * V5 * NR
    achieved = alg_bytes / (ms * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": gflops, "unit": "GFlop/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": _config(),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (recorded_traffic(tiles[dw.DW_OP_DHOP], DIMS, LS)
                                 if main_op == dw.DW_OP_DHOP else None),
                     "peak_source": peak_kind,
                     "bytes_per_site": bps, "sites_per_launch": V5 * NR},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "tile": tiles[main_op],
    }
    if args.main_only or args.layout != "spin_pair":
        line["op"] = args.op
        line["layout"] = args.layout
        line["dtype"] = "f16" if prec == dw.DW_F16 else "f32"
        line["config"]["nrhs"] = NR
        line["config"]["prec"] = line["dtype"]
        if rank == 0:
            print(json.dumps(line), flush=True)
        lat.close()
        return 0

    # other operators on the same lattice (kernel-only, same event method)
    mf = [MF]
    ops = {}
    ops["D"] = time_op(lambda: dw.dw_apply_D(lat.handle, y.data_ptr(), x.data_ptr(), mf, 1, sh),
                       args.steps, 3, stream)
    ops["Ddag"] = time_op(
        lambda: dw.dw_apply_Ddag(lat.handle, y.data_ptr(), x.data_ptr(), mf, 1, sh),
        args.steps, 3, stream)
    ops["DdagD"] = time_op(
        lambda: dw.dw_apply_DdagD(lat.handle, y.data_ptr(), x.data_ptr(), mf, 1, sh),
        max(5, args.steps // 2), 3, stream)
    def op_line(ms, flop, nbytes):
        gbs = nbytes / ms / 1e6
        return {"ms": ms, "gflops": flop / ms / 1e6, "gbs": gbs, "frac": gbs / peak,
                "bytes_per_launch": nbytes}

    ops_out = {
        "peak_gbs": peak, "peak_source": peak_kind + " copy bandwidth (MEASURED_PEAKS hbm_gbs)",
        "D": op_line(ops["D"], FLOP_D_MOBIUS * V5, alg_bytes),
        "Ddag": op_line(ops["Ddag"], FLOP_D_MOBIUS * V5, alg_bytes),
        "DdagD": op_line(ops["DdagD"], 2 * FLOP_D_MOBIUS * V5, 2 * alg_bytes),
        "tiles": {"Dhop": tiles[dw.DW_OP_DHOP], "D": tiles.get(dw.DW_OP_D),
                  "Ddag": tiles.get(dw.DW_OP_DDAG)},
    }
    # layout ablation: the same Dhop with interleaved-complex quads (the RIRI
    # counterpart) at its own tuned tile, beside the spin-pair (RRII-like) default
    latc = Lattice(DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F32)
    latc.load_gauge(U)
    dw.dw_set_complex_layout(latc.handle, 1)
    xc = latc.pack(psi)
    yc = latc.empty(1)
    tc = latc.tune(dw.DW_OP_DHOP, 1)
    msc = time_op(lambda: dw.dw_apply_Dhop(latc.handle, yc.data_ptr(), xc.data_ptr(), 1, sh),
                  args.steps, 3, stream)
    ops_out["layout_ablation"] = {
        "spin_pair": dict(op_line(ms, FLOP_DHOP * V5, alg_bytes), tile=tiles[dw.DW_OP_DHOP]),
        "interleaved_complex": dict(op_line(msc, FLOP_DHOP * V5, alg_bytes), tile=tc),
    }
    del xc, yc
    latc.close()

    # FP16-storage Dhop on the same lattice
    lat16 = Lattice(DIMS, LS, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F16)
    lat16.load_gauge(U)
    x16 = lat16.pack(psi)
    y16 = lat16.empty(1)
    lat16.tune(dw.DW_OP_DHOP, 1)
    ms16 = time_op(lambda: dw.dw_apply_Dhop(lat16.handle, y16.data_ptr(), x16.data_ptr(), 1, sh),
                   args.steps, 3, stream)
    ops_out["Dhop_f16"] = {"ms": ms16, "gflops": FLOP_DHOP * V5 / ms16 / 1e6,
                           "gbs": bytes_per_site(2, LS) * V5 / ms16 / 1e6,
                           "frac": bytes_per_site(2, LS) * V5 / ms16 / 1e6 / peak}
    del x16, y16
    lat16.close()

    # Wilson Dslash: the same kernel at Ls = 1 on the same 4D lattice.  Its field
    # (201 MB) and links (100 MB) would largely stay in L2 between back-to-back
    # launches, so each launch is timed alone after an L2 flush.  The fraction is
    # taken on the bytes the kernel must move: spinor in and out and two-row
    # (12-real) links, 384 B per site (the 18-real model gives 480 B).
    latw = Lattice(DIMS, 1, kind=dw.DW_MOBIUS, M5=M5, b=B, c=C, prec=dw.DW_F32)
    latw.load_gauge(U)
    psiw = inputs.gaussian_fermion(DIMS, 1, 1, seed=SEED)
    xw = latw.pack(psiw)
    yw = latw.empty(1)
    tw = latw.tune(dw.DW_OP_DHOP, 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    msw = time_op_flushed(lambda: dw.dw_apply_Dhop(latw.handle, yw.data_ptr(), xw.data_ptr(),
                                                   1, sh), max(10, args.steps // 2), 3, stream,
                          flush)
    moved = 4 * (48 + 48) * V4
    ops_out["wilson_dslash_f32"] = {"ms": msw, "gflops": FLOP_DHOP * V4 / msw / 1e6,
                                    "gbs": moved / msw / 1e6, "frac": moved / msw / 1e6 / peak,
                                    "bytes_per_site": 384, "l2": "flushed before each launch",
                                    "tile": tw}
    del xw, yw, flush
    latw.close()

    # layout conversion (A0): canonical complex128 <-> internal FP32, device to device
    canon = torch.zeros(V5 * 24, dtype=torch.float64, device="cuda")
    canon_bytes = canon.numel() * 8
    ms_pack = time_op(lambda: dw.dw_pack_fermion(lat.handle, y.data_ptr(), dw.DW_F32,
                                                  canon.data_ptr(), 1, sh), args.steps, 3, stream)
    ms_unpack = time_op(lambda: dw.dw_unpack_fermion(lat.handle, canon.data_ptr(), x.data_ptr(),
                                                      dw.DW_F32, 1, sh), args.steps, 3, stream)
    field_bytes = lat.fermion_bytes(1)
    for name, msv in (("pack_f32", ms_pack), ("unpack_f32", ms_unpack)):
        gbs = (canon_bytes + field_bytes) / msv / 1e6
        ops_out[name] = {"ms": msv, "gbs": gbs, "frac": gbs / peak}
    del canon

    # end to end through the host-buffer entry point (pinned host, H2D + D2H inside)
    nbytes = lat.fermion_bytes(1)
    hin = x.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    lat.apply_host(dw.DW_OP_DHOP, hout, hin)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("e2e_timed")
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.apply_host(dw.DW_OP_DHOP, hout, hin)
    torch.cuda.nvtx.range_pop()
    e2e_ms, e2e_rate = aggregate(ws, (time.perf_counter() - t0) / e2e_steps * 1e3, V5)
    e2e_s = e2e_ms * 1e-3
    e2e = {"value": FLOP_DHOP * e2e_rate / 1e9, "unit": "GFlop/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "ms_per_step": e2e_s * 1e3}

    line["e2e"] = e2e
    line["ops"] = ops_out
    line["paper_context"] = paper_context()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(psi, U)
        line["oracle_timings"] = oracle_timings(psi, U)
    del x, y
    lat.close()
    if not args.no_cg:
        line["batched"] = bench_batched(args)
        line["cg"] = bench_cg(args)
        line["cg_eo"] = bench_eo(args)
        if args.cg_full:
            line["cg_full"] = bench_cg(args, DIMS, LS, SEED)
            line["cg_eo_full"] = bench_eo(args, DIMS, LS, SEED, f64=False)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
