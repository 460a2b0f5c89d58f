#!/usr/bin/env python
"""Benchmark of the SDRT residual on GB300: DOF-updates/s of classical RK4 steps.

Workload (default): compressible Euler (5 variables, gamma = 1.4) on the
periodic cube [-5, 5]^3 split into 24^3 x 6 = 82,944 tetrahedra, SDRT degree
p = 3 (20 solution points per element), Rusanov common flux, isentropic vortex
(Ma 0.5, S = 13.5, R = 1.5) times (1 + 1e-3 U(-1, 1)) with NumPy PCG64 seed
20210518, RK4 with dt = 1e-3.  One step = one RK4 step = 4 residual
evaluations, each fused with its stage update.  DOF-updates/s =
nsol * nvar * nelem * 4 / step time (paper App. C's PM metric inverted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
  python bench.py --impl reference      # the FP64 CPU oracle on the same workload

Multi-GPU (torchrun): every rank steps its own replica of the workload
(independent problems, no data-path collective); value = all ranks' DOF
updates / max over ranks of the timed region.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SDRT residual DOF-updates/s on 1 GB300 (FP32/batched vs FP64 at stated L2 err), % roofline"
UNIT = "DOF-updates/s"
WORKLOAD = "euler3d_tet_p3_82944_rk4"
SEED = 20210518
DT = 1e-3
NCELL = 24
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sdrt", choices=["sdrt", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU path and the accuracy check")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--accuracy-steps", type=int, default=20)
    ap.add_argument("--ncell", type=int, default=NCELL, help="cubes per axis (profiling of smaller cases)")
    ap.add_argument("--tc-div", type=int, default=0, choices=[0, 1],
                    help="divergence on the tensor cores (SDRT_OPT_TC_DIVERGENCE)")
    ap.add_argument("--tc-interp", type=int, default=0, choices=[0, 1],
                    help="interpolation on the tensor cores (SDRT_OPT_TENSOR_CORES)")
    return ap.parse_args()


def workload_mesh(ncell=NCELL):
    from inputs import meshes
    return meshes.box_mesh("tet", (ncell,) * 3, [-5.0] * 3, [5.0] * 3)


def initial_field(X, seed):
    from inputs import fields
    u = fields.isentropic_vortex(X, gamma=1.4, mach=0.5)
    return u * (1 + fields.uniform_noise(u.shape, seed, 1e-3))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(nsol, nfe, nfiu, nvar, nfaces, nd, s, nelem):
    """Algorithmic bytes per launch of the two kernels of one RK4 stage
    (padding of the records excluded).

    k_interp_rec : read U (nsol V s); write the external-point states (nfe V s)
                   and the internal-point states (nfiu V s)
    k_flux_rec   : read own and partner external-point states (2 nfe V s), the
                   internal-point states (nfiu V s), the metric
                   ((1 + nd^2 + nfaces (nd+1)) s), the partner permutation
                   (nfe B) and partner face offsets (nfaces * 4 B); stage update
                   averaged over the 4 RK4 stages in state volumes (nsol V s):
                   stage 1 read u0 + 2 writes = 3, stages 2-3 2 reads + 2 writes
                   = 4, stage 4 read + write = 2 -> 13 / 4 = 3.25
    """
    interp = (nsol + nfe + nfiu) * nvar * s
    metric = (1 + nd * nd + nfaces * (nd + 1)) * s
    resid = (2 * nfe + nfiu) * nvar * s + metric + nfe + 4 * nfaces + 3.25 * nsol * nvar * s
    return interp * nelem, resid * nelem


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_sources_sha():
    """Hash of every CUDA source of the library (identifies the kernel build)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2105_08632_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".hpp")):
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """dram bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "k_flux_rec_tet_p3_euler_fp32.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_sources_sha()
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(ncell=16):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    the same element type, degree, physics and initial field on a periodic
    ncell^3 x 6 tetrahedron box, one RK4 step (4 residual evaluations)."""
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from oracle import residual as ores
    mesh = workload_mesh(ncell)
    geom = omesh.build(mesh, 3)
    phys = ophx.Physics("euler", 3, "rusanov", gamma=1.4)
    U = []
    for g in geom.blocks:
        X = g.xsol.reshape(-1, 3)
        v = initial_field(X, SEED).reshape(g.nelem, g.ops.n_sol, 5)
        U.append(np.ascontiguousarray(np.transpose(v, (1, 2, 0))))
    t0 = time.perf_counter()
    ores.rk4_step(geom, phys, U, DT)
    t = time.perf_counter() - t0
    ndof = sum(g.ops.n_sol * 5 * g.nelem for g in geom.blocks)
    return {"value": ndof * 4 / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one RK4 step (4 residuals) of the same tet p=3 Euler workload on a {ncell}^3 x 6 = "
                      f"{6 * ncell ** 3}-element periodic box; NumPy FP64, single-threaded einsum; "
                      f"{t:.2f} s; host affinity {len(os.sched_getaffinity(0))} cores"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(ncell=4)
        if i >= args.warmup:
            steps.append(cb["value"])
    v = float(np.mean(steps))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": "4^3 x 6 = 384 tetrahedra per step (bounded CPU sample)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one RK4 step on a 4^3 x 6 tetrahedron periodic box per bench step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_leg(sdrt, ctx, mesh, stream, flush, U0, ndof, args):
    """The plain FP64 GPU path on the same workload (timed like the main arm,
    fewer steps) and the accuracy of the FP32 path against it: one residual,
    and the state after a few RK4 steps (relative L2 / L-inf over all values;
    'update' errors are relative to the FP64 change of the state)."""
    import torch
    M32 = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp32", gamma=1.4))
    M64 = sdrt.Mesh(ctx, mesh, 3, sdrt.make_physics("euler", 3, "rusanov", "fp64", gamma=1.4))
    dev = flush.device
    h64 = M64.pack([U0])
    U64 = torch.from_numpy(h64).to(dev)
    for i in range(3):
        flush.fill_(float(i))
        M64.rk4_step(U64, DT, 1)
    M64.sync()
    ms = []
    for i in range(args.fp64_steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M64.rk4_step(U64, DT, 1)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    M64.sync()
    ms64 = float(np.mean(ms))
    fp64 = {"value": ndof * 4 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
            "dtype": "f64"}
    # accuracy of the FP32 path against the FP64 path
    a64 = torch.from_numpy(h64).to(dev)
    a32 = torch.from_numpy(M32.pack([U0])).to(dev)
    r64 = torch.zeros_like(a64)
    r32 = torch.zeros_like(a32)
    M64.residual(a64, r64)
    M32.residual(a32, r32)
    M64.rk4_step(a64, DT, args.accuracy_steps)
    M32.rk4_step(a32, DT, args.accuracy_steps)
    M32.sync()
    M64.sync()
    R64, R32 = M64.unpack(r64.cpu().numpy())[0], M32.unpack(r32.cpu().numpy())[0].astype(np.float64)
    S64, S32 = M64.unpack(a64.cpu().numpy())[0], M32.unpack(a32.cpu().numpy())[0].astype(np.float64)
    dR, dS, dU = R32 - R64, S32 - S64, S64 - U0

    def rel(a, b):
        return {"rel_l2": float(np.linalg.norm(a) / np.linalg.norm(b)),
                "rel_linf": float(np.abs(a).max() / np.abs(b).max())}

    accuracy = {"reference": "FP64 GPU path on the same workload",
                "residual": rel(dR, R64),
                f"state_after_{args.accuracy_steps}_steps": rel(dS, S64),
                f"update_after_{args.accuracy_steps}_steps": rel(dS, dU)}
    return fp64, accuracy


def aggregate(total_ms, steps, ndof, dist=None, device="cpu"):
    """Whole-job timing of the replicas: the timed region is the maximum over
    ranks, the throughput counts every rank's DOF updates (4 residual
    evaluations per RK4 step).  Returns (total ms, ms per step, DOF-updates/s)."""
    world = 1
    if dist is not None:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        world = dist.get_world_size()
    ms_per_step = total_ms / steps
    return total_ms, ms_per_step, world * ndof * 4 / (ms_per_step / 1e3)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2105_08632_gb300 import sdrt
    if not os.path.exists(sdrt.LIB_PATH):
        from paper_2105_08632_gb300 import build
        build.build()

    stream = torch.cuda.Stream(local)
    torch.cuda.set_stream(stream)
    ctx = sdrt.Context(local, stream.cuda_stream)
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TC_DIVERGENCE, args.tc_div)
    sdrt.sdrt_set_option(ctx.ptr, sdrt.SDRT_OPT_TENSOR_CORES, args.tc_interp)
    mesh = workload_mesh(args.ncell)
    phys = sdrt.make_physics("euler", 3, "rusanov", args.precision, gamma=1.4)
    M = sdrt.Mesh(ctx, mesh, 3, phys)
    lay = M.layouts[0]
    nelem, nsol, nvar = lay["nelem"], lay["nsol"], lay["nvar"]
    ndof = M.info["ndof"]
    X = M.sol_points()[0].reshape(-1, 3)
    U0 = initial_field(X, SEED + rank).reshape(nelem, nsol, nvar).transpose(1, 2, 0)
    host = M.pack([U0])
    tdtype = torch.float32 if args.precision == "fp32" else torch.float64
    U = torch.from_numpy(host).to(f"cuda:{local}")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")

    for i in range(args.warmup):
        flush.fill_(float(i))
        M.rk4_step(U, DT, 1)
    M.sync()
    sdrt.sdrt_profile_enable(ctx.ptr, True)
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = sdrt.sdrt_launch_count(ctx.ptr)
    prof = {k: [0.0, 0] for k in sdrt.KERNEL_KINDS}
    step_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))                      # evict L2 (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.rk4_step(U, DT, 1)
        e1.record(stream)
        for k, (ms, n) in sdrt.sdrt_profile_collect(ctx.ptr).items():   # synchronises
            prof[k][0] += ms
            prof[k][1] += n
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = sdrt.sdrt_launch_count(ctx.ptr) - launches0
    clocks = sampler.stop()
    sdrt.sdrt_profile_enable(ctx.ptr, False)
    M.sync()
    total_ms, ms_per_step, value = aggregate(float(np.sum(step_ms)), args.steps, ndof, dist, f"cuda:{local}")

    # Roofline of the dominant kernel (the residual / divergence kernel).
    s = 4 if args.precision == "fp32" else 8
    info = sdrt.sdrt_get_etype_info(ctx.ptr, M.etypes[0])
    b_interp, b_resid = algorithmic_bytes(nsol, info["nfe"], info["nfiu"], nvar, info["nfaces"], 3, s, nelem)
    ms_r, n_r = prof["residual"]
    ms_i, n_i = prof["interp_ext"]
    avg_r = ms_r / max(n_r, 1)
    avg_i = ms_i / max(n_i, 1)
    peak, peak_kind = peaks()
    achieved = b_resid / (avg_r / 1e3) / 1e9 if n_r else None
    traffic = ncu_traffic()
    roofline = {"bound": "hbm", "kernel": "k_flux_rec", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "peak_source": ("of measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                else "of fallback"),
                "algorithmic_bytes_per_launch": b_resid, "avg_launch_ms": avg_r,
                "kernel_sources_sha256_16": kernel_sources_sha(),
                "k_interp_rec": {"algorithmic_bytes_per_launch": b_interp, "avg_launch_ms": avg_i,
                                 "achieved_gbs": b_interp / (avg_i / 1e3) / 1e9 if n_i else None},
                "step_share": {"k_flux_rec": ms_r / max(total_ms, 1e-9) if not dist else None,
                               "k_interp_rec": ms_i / max(total_ms, 1e-9) if not dist else None},
                "step_hbm_frac": ((b_resid + b_interp) * 4 / (ms_per_step / 1e3) / 1e9) / peak}

    # End to end through the host-buffer entry point (pinned memory).
    pin_in = torch.from_numpy(host).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    e2e_t = []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        t0 = time.perf_counter()
        M.rk4_step_host(pin_in, pin_out, DT, 1)
        t1 = time.perf_counter()
        if i > 0:
            e2e_t.append(t1 - t0)
    nbytes = host.nbytes
    e2e = None
    if e2e_t:
        e2e = {"value": world * ndof * 4 / float(np.mean(e2e_t)), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "api": "sdrt_rk4_step_host (pinned host buffers, 1 step per call)"}

    fp64, accuracy = None, None
    if rank == 0 and args.precision == "fp32" and not args.no_fp64:
        fp64, accuracy = fp64_leg(sdrt, ctx, mesh, stream, flush, U0, ndof, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        workload = WORKLOAD if args.ncell == NCELL else f"euler3d_tet_p3_{6 * args.ncell ** 3}_rk4"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": {"workload": workload, "elements": nelem, "tc_divergence": args.tc_div,
                           "tc_interpolation": args.tc_interp, "degree": 3, "nsol": nsol, "nvar": nvar,
                           "ndof": ndof, "residuals_per_step": 4, "precision": args.precision,
                           "l2": "flushed between timed steps (256 MiB write, untimed)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fp64_path": fp64, "accuracy": accuracy}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()
