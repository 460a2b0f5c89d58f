#!/usr/bin/env python
"""Benchmark of the SDRT residual on GB300: DOF-updates/s of classical RK4 steps.

Workloads (all periodic, synthetic, seeded; one step = one RK4 step = 4
residual evaluations, each fused with its stage update; DOF-updates/s =
sum over blocks of nsol * nvar * nelem * 4 / step time, the inverse of the
paper's App. C PM metric):

  mixed (default)  the batched configuration: four independent FP32 Euler
                   meshes in one (degrees 1..4; hexahedra / x-extruded prisms
                   and tetrahedra / z-extruded prisms in seeded slab orders,
                   489,664 elements), the isentropic vortex with one seed per
                   mesh, dt = 1e-3
  euler            compressible Euler (5 variables, gamma = 1.4) on [-5, 5]^3
                   split into 24^3 x 6 = 82,944 tetrahedra, degree 3, Rusanov,
                   isentropic vortex (Ma 0.5, S = 13.5, R = 1.5) times
                   (1 + 1e-3 U(-1, 1)), NumPy PCG64 seed 20210518, dt = 1e-3
  tgv              Navier-Stokes Taylor-Green vortex (Re 1600, Ma 0.1,
                   Pr 0.71, LDG beta = 0.5, eta = 0.1) on [0, 2 pi]^3 split into
                   48^3 x 6 = 663,552 tetrahedra of degree 4, dt = 2e-4

The JSON line's value is the selected workload; the other two are measured
with fewer steps and reported under "other_workloads".

  python bench.py [--workload W] [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample

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
WORKLOAD = "euler3d_tet_p3_82944_rk4"     # label of the 3D Euler workload at full size
SEED = 20210518
DT = 1e-3
NCELL = 24
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="sdrt", choices=["sdrt", "reference"])
    ap.add_argument("--workload", default="mixed", choices=["euler", "tgv", "mixed"])
    ap.add_argument("--no-others", action="store_true", help="skip the other two workloads")
    ap.add_argument("--other-steps", type=int, default=100, help="timed steps of the other workloads (TGV: / 10)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU path and the accuracy check")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--accuracy-steps", type=int, default=20)
    ap.add_argument("--ncell", type=int, default=None, help="size parameter (profiling of smaller cases)")
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


# Batched mixed meshes: (structure, degree, cubes per slab side, slab kinds).
# Slab counts give element counts of ~300k, 120k, 50k and 20k at full size.
MIXED_PARTS = [("hex", 1, 40, 100, 44), ("tet", 2, 32, 16, 10), ("hex", 3, 24, 45, 21), ("tet", 4, 16, 11, 6)]


def workload_label(name, ncell=None):
    """The label Workload(name, ncell).label has, without building the mesh."""
    if name == "euler":
        n = ncell or NCELL
        return f"euler3d_tet_p3_{6 * n ** 3}_rk4"
    if name == "tgv":
        n = ncell or 48
        return f"tgv_ns_tet_p4_{6 * n ** 3}_rk4"
    f = ncell / 40.0 if ncell else 1.0
    per = {"hex": 1, "pri_x": 2, "tet": 6, "pri": 2}
    total = 0
    for kind, p, nc, n1, n2 in MIXED_PARTS:
        m = max(12, int(round(nc * f)))
        a, b_ = max(1, int(round(n1 * f))), max(1, int(round(n2 * f)))
        total += m * m * (a * per[kind] + b_ * per["pri_x" if kind == "hex" else "pri"])
    return f"mixed_euler_hex_pri_tet_p1-4_{total}_rk4"


class Workload:
    """Mesh, degrees, physics and initial state of one benchmark workload.
    scale < 1 shrinks the mesh (bounded oracle samples)."""

    def __init__(self, name, ncell=None, rank=0, scale=1.0):
        from inputs import fields, meshes
        self.name = name
        self.nd = 3
        self.block_mesh = None
        self.rank = rank
        if name == "euler":
            n = ncell or NCELL
            if scale != 1.0:
                n = max(2, int(round(n * scale)))
            self.mesh = workload_mesh(n)
            self.degrees = [3] * len(self.mesh["blocks"])
            self.parts = [(self.mesh, self.degrees)]
            self.system, self.riemann, self.kw, self.dt = "euler", "rusanov", {"gamma": 1.4}, DT
            self._init = lambda b, X: initial_field(X, SEED + rank)
        elif name == "tgv":
            n = ncell or 48
            if scale != 1.0:
                n = max(2, int(round(n * scale)))
            self.mesh = meshes.box_mesh("tet", (n,) * 3, [0.0] * 3, [2 * np.pi] * 3)
            self.degrees = [4] * len(self.mesh["blocks"])
            self.parts = [(self.mesh, self.degrees)]
            self.system, self.riemann, self.dt = "ns", "rusanov", 2e-4
            self.kw = {"gamma": 1.4, "mu": 1.0 / 1600.0, "prandtl": 0.71, "beta": 0.5, "eta": 0.1}
            self._init = lambda b, X: fields.taylor_green(X, gamma=1.4, mach=0.1)
        elif name == "mixed":
            f = (ncell / 40.0 if ncell else 1.0) * scale
            parts, self.degrees, self.block_mesh = [], [], []
            for k, (kind, p, nc, n1, n2) in enumerate(MIXED_PARTS):
                m = max(12, int(round(nc * f)))    # coarser cross-sections under-resolve the vortex core
                a, b_ = max(1, int(round(n1 * f))), max(1, int(round(n2 * f)))
                slabs = (["hex"] * a + ["pri_x"] * b_) if kind == "hex" else (["tet"] * a + ["pri"] * b_)
                order = np.random.default_rng(SEED + k).permutation(len(slabs))
                mk = meshes.box_mesh([slabs[i] for i in order], (m, m, len(slabs)), [-5.0] * 3, [5.0] * 3)
                parts.append(mk)
                self.degrees += [p] * len(mk["blocks"])
                self.block_mesh += [k] * len(mk["blocks"])
            self.mesh = meshes.merge_meshes(parts)
            self.parts = [(mk, [p] * len(mk["blocks"])) for mk, (_, p, _, _, _) in zip(parts, MIXED_PARTS)]
            self.system, self.riemann, self.kw, self.dt = "euler", "rusanov", {"gamma": 1.4}, DT
            self._init = lambda b, X: initial_field(X, SEED + 1000 * self.block_mesh[b] + rank)
        else:
            raise ValueError(name)
        self.nelem = sum(len(b["verts"]) for b in self.mesh["blocks"])
        self.nvar = 1 if self.system in ("advection", "advdiff") else self.nd + 2
        shapes = sorted({b["shape"] for b in self.mesh["blocks"]})
        tag = {"euler": f"euler3d_tet_p3_{self.nelem}_rk4", "tgv": f"tgv_ns_tet_p4_{self.nelem}_rk4",
               "mixed": f"mixed_euler_{'_'.join(shapes)}_p1-4_{self.nelem}_rk4"}[name]
        self.label = tag

    def physics(self, sdrt, precision):
        return sdrt.make_physics(self.system, self.nd, self.riemann, precision, **self.kw)

    def state(self, sol_points):
        """Initial state per block, (N_s, V, E), from the solution points (E, N_s, ND)."""
        out = []
        for b, X in enumerate(sol_points):
            E, ns = X.shape[0], X.shape[1]
            u = self._init(b, X.reshape(-1, X.shape[-1])).reshape(E, ns, self.nvar)
            out.append(np.ascontiguousarray(u.transpose(1, 2, 0)))
        return out

    def part_state(self, k, sol_points):
        """Initial state of the blocks of independent mesh k (self.parts[k]),
        the same values as in the merged mesh."""
        b0 = sum(len(m["blocks"]) for m, _ in self.parts[:k])
        out = []
        for j, X in enumerate(sol_points):
            E, ns = X.shape[0], X.shape[1]
            u = self._init(b0 + j, X.reshape(-1, X.shape[-1])).reshape(E, ns, self.nvar)
            out.append(np.ascontiguousarray(u.transpose(1, 2, 0)))
        return out

    def composition(self):
        c = {}
        for b, p in zip(self.mesh["blocks"], self.degrees):
            key = f"{b['shape']}_p{p}"
            c[key] = c.get(key, 0) + len(b["verts"])
        return c


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def record_path(infos, system, riemann):
    """Whether every block runs on the register-blocked record path
    (tetrahedra of degree 3 or 4, Euler / Rusanov or advection)."""
    ok_sys = system == "advection" or (system == "euler" and riemann == "rusanov")
    return ok_sys and all(i["ndim"] == 3 and i["nfaces"] == 4 and i["nsol"] in (20, 35) for i in infos)


def residual_bytes(info, nvar, s, viscous):
    """Algorithmic bytes per element of one residual evaluation (the method's
    own data movement, independent of the kernels): read U, write the own
    external-point states, re-read U for the divergence, read the partner's
    external-point states, write R -- s V (3 N_s + 2 N_fe) -- plus the affine
    geometry (1 / det J, det J J^-1, per face a normal and a scale) and the
    face connectivity (8 B per face).  Viscous systems (LDG):
    s V (4 N_s + 3 N_fe + ND (2 N_s + 2 N_fe)) + geometry + connectivity."""
    ns, nfe, nf, nd = info["nsol"], info["nfe"], info["nfaces"], info["ndim"]
    geom = (1 + nd * nd + nf * (nd + 1)) * s
    conn = 8 * nf
    if viscous:
        return s * nvar * (4 * ns + 3 * nfe + nd * (2 * ns + 2 * nfe)) + geom + conn
    return s * nvar * (3 * ns + 2 * nfe) + geom + conn


def generated_bytes(info, nvar, s):
    """Bytes per element that the operator-specialised kernels move in one RK4
    step: the interpolation reads U and writes the face records; each stage
    reads the stage state, the partners' records, the metric rows and the
    partner map, reads / writes its RK volumes (stage 1: u0 in, uacc and the
    next state out; stages 2-3: u0 and uacc in, uacc and the next state out;
    stage 4: uacc in, U out) and stages 1-3 write the next face records."""
    ns, nfe, nf, nd = info["nsol"], info["nfe"], info["nfaces"], info["ndim"]
    vol, rec = ns * nvar * s, nfe * nvar * s
    side = (1 + nd * nd + nf * (nd + 1)) * s + 4 * nfe
    stage = vol + rec + side
    return {"interp_ext": vol + rec, "residual": 4 * stage + (3 + 4 + 4 + 2) * vol + 3 * rec}


def algorithmic_bytes(info, nelem, nvar, s, record, viscous, fused=False):
    """Implementation bytes of one RK4 step per kernel kind for one block of
    the record / generic kernels (padding excluded).  Stage updates in state
    volumes N_s V s: stage 1 reads u0 and writes uacc and the next state = 3,
    stages 2-3 read u0, uacc and write two = 4, stage 4 reads uacc and writes
    U = 2 -> 13 per step.

    record path   k_interp_*   : read U, write external + internal point states
                  k_flux_rec   : own + partner external states, internal states,
                                 metric, permutation, partner offsets, stage update
                  fused        : one interpolation per step; stages 1-3 keep the
                                 next state on chip (no write of it: 10 volumes
                                 per step) and write its external + internal
                                 point states instead
    generic path  k_interp_ext : read U, write external point states
                  k_grad       : read U, own + partner external states, write the
                                 physical gradients at all flux points (viscous)
                  k_residual   : read U, partner external states (+ own and
                                 partner gradients, internal gradients), metric,
                                 face map, stage update
    """
    ns, nfe, nfiu, nf, nd = info["nsol"], info["nfe"], info["nfiu"], info["nfaces"], info["ndim"]
    V = nvar
    metric = (1 + nd * nd + nf * (nd + 1)) * s
    vol = ns * V * s
    if record:
        points = (ns + nfe + nfiu) * V * s
        flux = (2 * nfe + nfiu) * V * s + metric + nfe + 4 * nf
        if fused:
            return {"interp_ext": points * nelem,
                    "residual": (4 * flux + 10 * vol + 3 * (nfe + nfiu) * V * s) * nelem}
        return {"interp_ext": 4 * points * nelem, "residual": (4 * flux + 13 * vol) * nelem}
    out = {"interp_ext": 4 * (ns + nfe) * V * s * nelem,
           "residual": (4 * ((ns + nfe) * V * s + metric + 4 * nfe) + 13 * vol) * nelem}
    if viscous:
        out["residual"] += 4 * (2 * nd * nfe + nd * nfiu) * V * s * nelem
        out["gradient"] = 4 * ((ns + 2 * nfe) * V * s + nd * (nfe + nfiu) * V * s + metric + 4 * nfe) * nelem
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        return self.parse(out)

    @staticmethod
    def parse(out):
        """Median SM clock, maximum SM clock and the throttle reasons seen active,
        from `nvidia-smi --query-gpu=<Q> --format=csv,noheader,nounits` lines."""
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


# Sources each kernel family is compiled from; a change to any of them makes
# the committed ncu counters of that family stale.
KERNEL_SOURCES = {
    "record": ("device_math.cuh", "flux_rec.cuh", "kargs.hpp", "kernels_fast.cu"),
    "generated": ("device_math.cuh", "flux_rec.cuh", "kargs.hpp", "generic.cuh", "gen_api.hpp", "gen_stage.cuh",
                  "gen/opgen.cpp", "refel.cpp"),
}
# Committed ncu summaries holding the dominant kernel's DRAM bytes per launch.
TRAFFIC_PROFILES = {("record", "euler"): "k_flux_rec_tet_p3_euler_fp32.txt",
                    ("generated", "mixed"): "k_gen_stage_mixed_euler_fp32.txt"}


def kernel_sources_sha(family="record"):
    """Hash of a kernel family's sources (identifies the profiled build)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2105_08632_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[family]:
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(family, workload, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources."""
    name = TRAFFIC_PROFILES.get((family, workload))
    path = os.path.join(ROOT, "profiles", name) if name else None
    if not path or not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256_16") != kernel_sources_sha(family):
        return None
    try:
        return float(vals[f"dram_bytes_per_launch_full_size[{kernel}]"])
    except (KeyError, ValueError):
        return None


_ORACLE_SETUP = {}


def _oracle_rk4_part(job):
    """RK4 steps of one independent mesh of a workload with the FP64 oracle
    (run in a spawned worker or in-process).  Returns (DOF, seconds of the
    steps alone, excluding the set-up)."""
    name, ncell, scale, k, steps = job
    from oracle import mesh as omesh
    from oracle import physics as ophx
    from oracle import residual as ores
    key = (name, ncell, scale, k)
    if key not in _ORACLE_SETUP:                 # set-up once per process (untimed)
        spec = Workload(name, ncell, 0, scale)
        mesh, degrees = spec.parts[k]
        geom = omesh.build(mesh, list(degrees))
        kw = dict(spec.kw)
        oph = ophx.Physics(spec.system, spec.nd, spec.riemann, gamma=kw.get("gamma", 1.4), mu=kw.get("mu", 0.0),
                           Pr=kw.get("prandtl", 0.72), beta=kw.get("beta", 0.5), eta=kw.get("eta", 0.1))
        _ORACLE_SETUP[key] = (spec, geom, oph, spec.part_state(k, [g.xsol for g in geom.blocks]))
    spec, geom, oph, U = _ORACLE_SETUP[key]
    t0 = time.perf_counter()
    for _ in range(steps):
        U = ores.rk4_step(geom, oph, U, spec.dt)
    t = time.perf_counter() - t0
    return sum(g.ops.n_sol * spec.nvar * g.nelem for g in geom.blocks), t


def _noop(_):
    return 0


class OraclePool:
    """Spawned worker processes, one per independent mesh of a workload (the
    oracle itself is single-threaded NumPy; its BLAS is held to one thread)."""

    def __init__(self, nparts):
        import multiprocessing as mp
        self.n = max(1, min(nparts, len(os.sched_getaffinity(0))))
        keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in keep:
            os.environ[k] = "1"
        self.pool = mp.get_context("spawn").Pool(self.n)
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        self.pool.map(_noop, range(self.n))          # workers started and NumPy imported

    def run(self, jobs):
        return self.pool.map(_oracle_rk4_part, jobs)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(name, ncell, scale, steps=1):
    """The FP64 oracle, as it stands, on a bounded sample of the workload (the
    same element types, degrees, physics and initial field on smaller
    meshes): `steps` RK4 steps.  Timed twice: on one core (the independent
    meshes one after the other) and on all the cores the meshes can use (one
    spawned process per independent mesh, running at the same time; the
    time is the slowest process's)."""
    spec = Workload(name, ncell, 0, scale)
    jobs = [(name, ncell, scale, k, steps) for k in range(len(spec.parts))]
    one = [_oracle_rk4_part(j) for j in jobs]
    ndof = sum(d for d, _ in one)
    t1 = sum(t for _, t in one)
    pool = OraclePool(len(jobs))
    par = pool.run(jobs)
    pool.close()
    tp = max(t for _, t in par)
    aff = len(os.sched_getaffinity(0))
    sample = (f"{steps} RK4 step(s) (4 residuals each) of {spec.label} ({spec.nelem} elements, "
              f"{len(jobs)} independent mesh(es)); NumPy FP64, single-threaded per process; "
              f"host affinity {aff} cores")
    return {"value": ndof * 4 * steps / tp, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": sample,
            "seconds": tp,
            "single_core": {"value": ndof * 4 * steps / t1, "unit": UNIT, "cores": 1, "seconds": t1}}


CPU_SCALE = {"euler": 16 / 24, "tgv": 10 / 48, "mixed": 0.35}
REF_SCALE = {"euler": 5 / 24, "tgv": 3 / 48, "mixed": 0.12}
REF_BUDGET_S = 150.0


# Solution points per element (paper App. A, Table "nsolpts_nfpts").
N_SOL = {"tri": lambda p: (p + 1) * (p + 2) // 2, "quad": lambda p: (p + 1) ** 2,
         "tet": lambda p: (p + 1) * (p + 2) * (p + 3) // 6, "pri": lambda p: (p + 1) ** 2 * (p + 2) // 2,
         "hex": lambda p: (p + 1) ** 3}


def full_ndof(name, ncell=None):
    """DOF of a full-size workload from its element counts (no mesh built)."""
    if name == "euler":
        return 6 * (ncell or NCELL) ** 3 * N_SOL["tet"](3) * 5
    if name == "tgv":
        return 6 * (ncell or 48) ** 3 * N_SOL["tet"](4) * 5
    f = ncell / 40.0 if ncell else 1.0
    total = 0
    for kind, p, nc, n1, n2 in MIXED_PARTS:
        m = max(12, int(round(nc * f)))
        a, b_ = max(1, int(round(n1 * f))), max(1, int(round(n2 * f)))
        main = N_SOL["hex"](p) * a if kind == "hex" else N_SOL["tet"](p) * 6 * a
        total += m * m * (main + N_SOL["pri"](p) * 2 * b_) * 5
    return total


def run_reference(args):
    """The oracle as the reference arm: one RK4 step of a bounded sample of the
    workload per bench step (its independent meshes in parallel processes),
    warm-up steps untimed; to keep the run within a few minutes for any
    --steps, timing stops after REF_BUDGET_S seconds and the mean is taken
    over the steps timed so far.  ms_per_step is the sample's own step time;
    the full-size projection at the sampled rate has its own key."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    small = Workload(args.workload, args.ncell, 0, REF_SCALE[args.workload])
    jobs = [(args.workload, args.ncell, REF_SCALE[args.workload], k, 1) for k in range(len(small.parts))]
    pool = OraclePool(len(jobs))
    secs, ndof = [], 0
    t_start = time.perf_counter()
    for i in range(args.warmup + args.steps):
        res = pool.run(jobs)
        ndof = sum(d for d, _ in res)
        if i >= args.warmup:
            secs.append(max(t for _, t in res))
        if secs and time.perf_counter() - t_start > REF_BUDGET_S:
            break
    pool.close()
    step_s = float(np.mean(secs))
    v = ndof * 4 / step_s
    ndof_full = full_ndof(args.workload, args.ncell)
    label = workload_label(args.workload, args.ncell)
    sample = (f"{small.label} ({small.nelem} elements, {len(jobs)} independent mesh(es) in {pool.n} processes), "
              f"one RK4 step per bench step; {len(secs)} of {args.steps} steps timed within the "
              f"{REF_BUDGET_S:.0f} s budget")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": len(secs),
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": label, "sample": sample, "sample_elements": small.nelem, "sample_ndof": ndof,
                       "ms_per_step": "one RK4 step of the sample"},
            "full_size_ms_per_step_extrapolated": ndof_full * 4 / v * 1e3,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.n, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_leg(sdrt, ctx, spec, stream, flush, U0, ndof, args):
    """The plain FP64 GPU path on the same workload (timed like the main arm,
    fewer steps) and the accuracy of the FP32 path against it: one residual,
    and the state after a few RK4 steps (relative L2 / L-inf over all values;
    'update' errors are relative to the FP64 change of the state)."""
    import torch
    M32 = sdrt.Mesh(ctx, spec.mesh, list(spec.degrees), spec.physics(sdrt, "fp32"))
    M64 = sdrt.Mesh(ctx, spec.mesh, list(spec.degrees), spec.physics(sdrt, "fp64"))
    dev = flush.device
    h64 = M64.pack(U0)
    U64 = torch.from_numpy(h64).to(dev)
    for i in range(3):
        flush.fill_(float(i))
        M64.rk4_step(U64, spec.dt, 1)
    M64.sync()
    ms = []
    for i in range(args.fp64_steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M64.rk4_step(U64, spec.dt, 1)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    M64.sync()
    ms64 = float(np.mean(ms))
    fp64 = {"value": ndof * 4 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
            "dtype": "f64"}
    a64 = torch.from_numpy(h64).to(dev)
    a32 = torch.from_numpy(M32.pack(U0)).to(dev)
    r64 = torch.zeros_like(a64)
    r32 = torch.zeros_like(a32)
    M64.residual(a64, r64)
    M32.residual(a32, r32)
    M64.rk4_step(a64, spec.dt, args.accuracy_steps)
    M32.rk4_step(a32, spec.dt, args.accuracy_steps)
    M32.sync()
    M64.sync()
    cat = lambda blocks: np.concatenate([b.astype(np.float64).ravel() for b in blocks])   # noqa: E731
    R64, R32 = cat(M64.unpack(r64.cpu().numpy())), cat(M32.unpack(r32.cpu().numpy()))
    S64, S32 = cat(M64.unpack(a64.cpu().numpy())), cat(M32.unpack(a32.cpu().numpy()))
    dR, dS, dU = R32 - R64, S32 - S64, S64 - cat(U0)

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


KERNEL_NAMES = {"record": {"interp_ext": "k_interp_rec", "residual": "k_flux_rec"},
                "generic": {"interp_ext": "k_interp_ext", "residual": "k_residual", "gradient": "k_grad"}}
BYTE_MODEL = ("algorithmic bytes of one residual evaluation per element: s V (3 N_s + 2 N_fe) (read U, write the own "
              "external-point states, re-read U, read the partner's external-point states, write R) + affine "
              "geometry + 8 B per face of connectivity; LDG viscous: s V (4 N_s + 3 N_fe + ND (2 N_s + 2 N_fe)) + "
              "geometry + connectivity; a stage launch of an element type processes one residual of its elements, an "
              "interpolation launch reads U and writes the external-point states")


def measure(sdrt, ctx, stream, flush, spec, args, steps, warmup, dist, local, world):
    """Time `steps` RK4 steps of a workload (after `warmup`), then the same
    steps again with an event pair around every launch inside the step graph
    for the per-kernel durations and the roofline, then the end-to-end call
    with host buffers."""
    import torch
    dev = f"cuda:{local}"
    M = sdrt.Mesh(ctx, spec.mesh, list(spec.degrees), spec.physics(sdrt, args.precision))
    ndof = M.info["ndof"]
    path = sdrt.PATHS[sdrt.sdrt_get_mesh_info(ctx.ptr, M.id)["path"]]
    U0 = spec.state(M.sol_points())
    host = M.pack(U0)
    U = torch.from_numpy(host).to(dev)
    dt = spec.dt
    infos = [sdrt.sdrt_get_etype_info(ctx.ptr, et) for et in M.etypes]
    if path == "generic":
        M.autotune(U, reps=3)          # tile widths of the generic kernels, per block (untimed)
    tiles = None
    if path == "generic":
        tiles = {f"{b['shape']}_p{p}_{i}": {k: v for k, v in t.items() if k in ("residual", "gradient")}
                 for i, (b, p, t) in enumerate(zip(spec.mesh["blocks"], spec.degrees, M.tiles()))}
    for i in range(warmup):
        flush.fill_(float(i))
        M.rk4_step(U, dt, 1)
    M.sync()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = sdrt.sdrt_launch_count(ctx.ptr)
    events = []
    for i in range(steps):
        flush.fill_(float(i))                      # evict L2 (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.rk4_step(U, dt, 1)
        e1.record(stream)
        events.append((e0, e1))
    torch.cuda.synchronize()
    launches = sdrt.sdrt_launch_count(ctx.ptr) - launches0
    step_ms = [a.elapsed_time(b) for a, b in events]
    total_ms, ms_per_step, value = aggregate(float(np.sum(step_ms)), steps, ndof, dist, dev)

    # Per-kernel durations: the same number of steps again with an event pair
    # around every launch inside the step's graph.  Event-record nodes between
    # the kernels lengthen the step, so `value` comes from the pass above.
    nb = len(M.layouts)
    sdrt.sdrt_profile_enable(ctx.ptr, True)
    flush.fill_(0.0)
    M.rk4_step(U, dt, 1)                           # graph capture with the event nodes (untimed)
    sdrt.sdrt_profile_collect_blocks(ctx.ptr, nb)
    prof = [{k: [0.0, 0] for k in sdrt.KERNEL_KINDS} for _ in range(nb + 1)]
    inst_ms = []
    for i in range(steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.rk4_step(U, dt, 1)
        e1.record(stream)
        for r, row in enumerate(sdrt.sdrt_profile_collect_blocks(ctx.ptr, nb)):   # synchronises
            for k, (ms, n) in row.items():
                prof[r][k][0] += ms
                prof[r][k][1] += n
        inst_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    sdrt.sdrt_profile_enable(ctx.ptr, False)
    M.sync()
    inst_total = float(np.sum(inst_ms))

    # Roofline of the dominant kernel (live CUDA-event durations inside the
    # timed region against the algorithmic bytes of what one launch processes).
    s = 4 if args.precision == "fp32" else 8
    viscous = spec.system in ("advdiff", "ns")
    shapes = [b["shape"] for b in spec.mesh["blocks"]]
    res_b = [residual_bytes(i, spec.nvar, s, viscous) * lay["nelem"] for i, lay in zip(infos, M.layouts)]
    interp_b = [s * spec.nvar * (i["nsol"] + i["nfe"]) * lay["nelem"] for i, lay in zip(infos, M.layouts)]
    fused = False
    entries = {}

    def entry(name, kind_key, ms_k, n_k, alg, impl):
        if n_k == 0:
            return
        avg = ms_k / n_k
        entries[name] = {"launches": n_k, "total_ms": ms_k, "avg_launch_ms": avg, "step_share": ms_k / max(inst_total, 1e-9),
                         "algorithmic_bytes_per_launch": alg, "achieved_gbs": alg / (avg / 1e3) / 1e9,
                         "implementation_bytes_per_launch": impl,
                         "implementation_gbs": impl / (avg / 1e3) / 1e9 if impl else None, "kind": kind_key}

    if path == "generated":
        for b in range(nb):
            tag = f"{shapes[b]}{spec.degrees[b]}"
            gb = generated_bytes(infos[b], spec.nvar, s)
            ne = M.layouts[b]["nelem"]
            ms_i, n_i = prof[b + 1]["interp_ext"]
            ms_r, n_r = prof[b + 1]["residual"]
            entry(f"k_gen_interp<{tag}>", "interp_ext", ms_i, n_i, interp_b[b], gb["interp_ext"] * ne)
            entry(f"k_gen_stage<{tag}>", "residual", ms_r, n_r, res_b[b], gb["residual"] * ne / 4)
        impl_step = sum(sum(generated_bytes(i, spec.nvar, s).values()) * lay["nelem"]
                        for i, lay in zip(infos, M.layouts))
    else:
        rec = path == "record"
        names = dict(KERNEL_NAMES[path])
        if rec and args.precision == "fp32":
            names["interp_ext"] = "k_interp_pipe"   # TMA-fed pipeline (FP32); FP64 keeps k_interp_rec
        if rec and args.tc_div and args.precision == "fp32":
            names["residual"] = "k_flux_tc"
        if rec and args.tc_interp and args.precision == "fp32":
            names["interp_ext"] = "k_interp_tc"
        # One interpolation launch per block and step: the RK4 stages
        # interpolate the next stage's state in their update (SDRT_OPT_FUSED_RK).
        fused = bool(rec and prof[0]["interp_ext"][1] == steps * nb)
        per_step = {}
        for info, lay in zip(infos, M.layouts):
            for k, bb in algorithmic_bytes(info, lay["nelem"], spec.nvar, s, rec, viscous, fused).items():
                per_step[k] = per_step.get(k, 0.0) + bb
        impl_step = sum(per_step.values())
        for k, bb in per_step.items():
            ms_k, n_k = prof[0][k]
            if n_k == 0:
                continue
            per_launch_impl = bb * steps / n_k
            if k == "residual":
                alg = sum(res_b) if rec else sum(res_b)
            elif k == "interp_ext":
                alg = sum(interp_b)
            else:
                alg = per_launch_impl
            entry(names[k], k, ms_k, n_k, alg, per_launch_impl)
    dom = max(entries, key=lambda k: entries[k]["total_ms"])
    dk = entries[dom]
    peak, peak_kind = peaks()
    family = "generated" if path == "generated" else "record"
    traffic = ncu_traffic(family, spec.name, dom) if (not args.ncell and args.precision == "fp32") else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": dk["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": dk["achieved_gbs"] / peak, "traffic": traffic,
                "peak_source": ("of measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                else "of fallback"),
                "byte_model": BYTE_MODEL,
                "algorithmic_bytes_per_launch": dk["algorithmic_bytes_per_launch"],
                "avg_launch_ms": dk["avg_launch_ms"],
                "implementation": {"bytes_per_launch": dk["implementation_bytes_per_launch"],
                                   "achieved": dk["implementation_gbs"],
                                   "frac": dk["implementation_gbs"] / peak if dk["implementation_gbs"] else None,
                                   "model": "bytes the kernels move, RK stage volumes and face records included"},
                "kernel_sources_sha256_16": kernel_sources_sha(family),
                "kernels": entries,
                "timing": "kernel durations from a second pass of the same steps with per-launch events "
                          "inside the graph (element types' kernels one after the other instead of concurrent; "
                          "ms_per_step there: %.4f); value and ms_per_step from the pass without them"
                          % (inst_total / max(steps, 1)),
                "fused_rk_stages": fused,
                "step_hbm_frac": (4 * sum(res_b) / (ms_per_step / 1e3) / 1e9) / peak,
                "step_hbm_frac_implementation": (impl_step / (ms_per_step / 1e3) / 1e9) / peak}

    # End to end through the host-buffer entry point (pinned memory).
    pin_in = torch.from_numpy(host).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    e2e_t = []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        t0 = time.perf_counter()
        M.rk4_step_host(pin_in, pin_out, dt, 1)
        t1 = time.perf_counter()
        if i > 0:
            e2e_t.append(t1 - t0)
    e2e = None
    if e2e_t:
        e2e = {"value": world * ndof * 4 / float(np.mean(e2e_t)), "unit": UNIT, "h2d_bytes_per_step": host.nbytes,
               "d2h_bytes_per_step": host.nbytes, "api": "sdrt_rk4_step_host (pinned host buffers, 1 step per call)"}
    return {"M": M, "U0": U0, "ndof": ndof, "path": path, "value": value, "ms_per_step": ms_per_step,
            "roofline": roofline, "e2e": e2e, "launches": launches, "clocks": clocks, "tiles": tiles}


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
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    spec = Workload(args.workload, args.ncell, rank)
    res = measure(sdrt, ctx, stream, flush, spec, args, args.steps, args.warmup, dist, local, world)

    fp64, accuracy = None, None
    if rank == 0 and args.precision == "fp32" and not args.no_fp64:
        fp64, accuracy = fp64_leg(sdrt, ctx, spec, stream, flush, res["U0"], res["ndof"], args)

    others = None
    if not args.no_others and not args.ncell:
        others = {}
        for name in ("mixed", "euler", "tgv"):
            if name == args.workload:
                continue
            osteps = max(3, args.other_steps // (10 if name == "tgv" else 1))
            o = measure(sdrt, ctx, stream, flush, Workload(name, None, rank), args, osteps, 3, dist, local, world)
            r = o["roofline"]
            others[workload_label(name)] = {
                "value": o["value"], "unit": UNIT, "ms_per_step": o["ms_per_step"], "steps": osteps,
                "path": o["path"], "gpu_launches": o["launches"], "clocks": o["clocks"],
                "e2e": o["e2e"],
                "roofline": {k: r[k] for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic",
                                               "algorithmic_bytes_per_launch", "avg_launch_ms", "step_hbm_frac",
                                               "step_hbm_frac_implementation")},
                "roofline_implementation": r["implementation"]}
            del o

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.ncell, CPU_SCALE[args.workload])

    if rank == 0:
        workload = workload_label(args.workload, args.ncell)
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
                "data": "synthetic",
                "config": {"workload": workload, "elements": spec.nelem, "composition": spec.composition(),
                           "system": spec.system, "riemann": spec.riemann, "nvar": spec.nvar, "ndof": res["ndof"],
                           "dt": spec.dt, "residuals_per_step": 4, "precision": args.precision,
                           "path": res["path"], "tiles": res["tiles"],
                           "tc_divergence": args.tc_div, "tc_interpolation": args.tc_interp,
                           "l2": "flushed between timed steps (256 MiB write, untimed)",
                           "parallelism": f"replicas x{world}"},
                "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"], "gpu_launches": res["launches"],
                "clocks": res["clocks"], "fp64_path": fp64, "accuracy": accuracy, "other_workloads": others}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()
