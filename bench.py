#!/usr/bin/env python
"""Benchmark: time-steps/s over all cases at certified relative residual 1e-8 (one JSON line).

Default workload (--config large): the large single mesh -- a 256x256x128 hex box (h = 1/64, a 4 x 4 x 2
domain) split into 50,331,648 linear tets (8,520,321 nodes, 25,560,963 DOF), five seeded log-normal layers
plus a half-ellipsoid low-velocity basin (mu x 0.3) at the surface, bottom fixed, 8 cases sharing the mesh
(Ricker point sources at seeded interior nodes, f0 ~ U[2, 8]), Newmark dt = 0.004 with Rayleigh damping
(0.01, 0.001).  The solver is the FP32-inner / FP64-refined block-Jacobi PCG with the EBE product, started
from the data-driven predictor (s = 16 stored steps, regions of 1024 nodes).  --config medium runs the
64x64x32 box (786,432 tets) with 16 cases and s = 32 instead.

A "step" advances all cases by one time step: predictor, right-hand side, certified solve, Newmark update.
The simulation is first run for --spinup steps (default 250: the paper times steps 250-500), then --warmup
untimed steps, then --steps timed steps.

Under torchrun (N > 1) every rank runs its own replica of the workload (different case seeds) on its own
GPU; value = all ranks' case-steps / the slowest rank's time ("replicas only": cases are independent).

--impl reference times the FP64 CPU oracle (scipy CSR, Algorithm 1, the regional MGS predictor) on the
host cores: one process per case on a bounded sub-box of the same recipe (all cores), its case-steps/s
scaled to the full mesh by the DOF ratio (labelled as extrapolated).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-steps/s over all cases at rel. residual 1e-8; EBE matvec HBM GB/s vs peak"
UNIT = "case-steps/s"
FLOP_PER_ELEM_CASE = 190.0     # factorised tet4 apply + consistent mass + fused p^T A p (FMA = 2 flops)
# FP64 split product (M p and K p separately): 157 flops (FMA = 2) in 115 FP64 instructions per element and case
FLOP_PER_ELEM_CASE_SPLIT = 157.0
DP_INSTR_PER_ELEM_CASE_SPLIT = 115.0


_T0 = time.perf_counter()


def log(msg):
    """Progress note on stderr (the JSON result is the only stdout line)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--spinup", type=int, default=250)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--predictor", default="dd", choices=["dd", "ab4"])
    ap.add_argument("--config", default="large", choices=["large", "medium"],
                    help="large: 256x256x128 box, 5 layers + basin, 8 cases, s = 16; medium: 64x64x32 box, "
                         "3 layers, 16 cases, s = 32")
    ap.add_argument("--cases", type=int, default=None)
    ap.add_argument("--source", default="ricker", choices=["ricker", "impulses"],
                    help="ricker: one Ricker point force per case; impulses: random impulses at surface points "
                         "(the paper's random inputs)")
    ap.add_argument("--impulse-points", type=int, default=None,
                    help="impulse points per case (default: 7%% of the surface nodes)")
    ap.add_argument("--impulse-steps", type=int, default=100, help="impulses fall in steps 1 .. this")
    ap.add_argument("--absorbing", action="store_true", help="absorbing (dashpot) boundaries on the four sides")
    ap.add_argument("--cpu-predictor", action="store_true",
                    help="the paper's heterogeneous scheme: data-driven correction on the host CPU, two case sets "
                         "alternating, s balanced against the solve time")
    ap.add_argument("--dims", default=None)
    ap.add_argument("--s-max", type=int, default=None)
    ap.add_argument("--region-nodes", type=int, default=1024)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--comparator-steps", type=int, default=None)
    ap.add_argument("--comparator-spinup", type=int, default=None)
    ap.add_argument("--cpu-dims", default=None,
                    help="hex dims of the oracle's sample (a sub-box of the same recipe; default: 32,32,16 for "
                         "large, the full mesh for medium)")
    ap.add_argument("--cpu-spinup", type=int, default=40, help="oracle steps from rest before its timed sample")
    ap.add_argument("--cpu-steps", type=int, default=20, help="timed oracle steps per case")
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes (0: min(cores, cases))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="eager launches instead of the captured step graph")
    ap.add_argument("--cert", type=int, default=3,
                    help="certification product: 0 EBE FP64, 1 EBE double-float, 2 assembled FP64, "
                         "3 assembled double-float")
    ap.add_argument("--snapshot-format", type=int, default=2,
                    help="predictor snapshot storage: 0 FP64, 1 FP32, 2 double-float, 3 FP32 + BF16 residual")
    ap.add_argument("--inner-product", default=None, choices=["fp32", "tc"],
                    help="inner CG products: FP32 element kernels, or FP16 hex element matrices on the tensor cores "
                         "(default: tc for the large box's 8 cases, fp32 for the medium box's 16, the faster one "
                         "for each)")
    ap.add_argument("--inner-margin", type=float, default=None,
                    help="FP32-inner solves aim at this fraction of the tolerance (default: the library's)")
    ap.add_argument("--no-guard", action="store_true",
                    help="keep every data-driven correction (no guess guard: fem_opts.pred_guard = 0)")
    ap.add_argument("--check-every", type=int, default=8,
                    help="inner CG iterations per convergence check (graph: launches per WHILE-loop body)")
    ap.add_argument("--profile-steps", type=int, default=40,
                    help="steps after the timed region timed per kernel class with CUDA events (eager)")
    ap.add_argument("--kernel", default=None, choices=["ebe", "ebe10", "pcg10", "split", "predictor", "mlp"],
                    help="time one kernel alone (EBE product) instead of the full step")
    ap.add_argument("--kernel-precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--variant", type=int, default=0,
                    help="EBE variant: 0 auto, 1 generic, 2 tiled hex, 3 staged tiles, 4 case-major staged tiles, "
                         "5/6 packed staged tiles (two / one block per SM)")
    ap.add_argument("--hex-per-tile", type=int, default=0)
    ap.add_argument("--element", default="tet4", choices=["tet4", "tet10"],
                    help="tet10: the time-stepping solver on the medium box's tets as 10-node tets (its own line)")
    ap.add_argument("--uneven", action="store_true",
                    help="batched uneven meshes: --meshes cases on meshes of different sizes fused into one system")
    ap.add_argument("--meshes", type=int, default=64)
    ap.add_argument("--no-fuse", action="store_true", help="(--uneven) step one group per mesh instead")
    ap.add_argument("--learned", action="store_true",
                    help="learned-proposal measurement: collect, train, evaluate on held-out cases")
    ap.add_argument("--train-cases", type=int, default=200)
    ap.add_argument("--eval-cases", type=int, default=32)
    ap.add_argument("--case-steps", type=int, default=500, help="steps per case (learned-proposal mode)")
    ap.add_argument("--updates", type=int, default=3000)
    ap.add_argument("--loss", default="residual", choices=["residual", "coef"],
                    help="learned proposal: residual-space loss ||Y (c + d) - e||^2 / ||e||^2 per region, or the "
                         "squared error of the coefficient correction")
    ap.add_argument("--dt", type=float, default=None, help="time step (default: the configuration's)")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--collect-from", type=int, default=0,
                    help="learned proposal: collect training samples from this step on (0: every step)")
    ap.add_argument("--batch", type=int, default=4096)
    a = ap.parse_args(argv)
    if a.learned or a.uneven or a.kernel in ("ebe10", "pcg10") or a.element == "tet10":
        a.config = "medium"          # these modes run on medium-size meshes
    large = a.config == "large"
    if a.cases is None:
        a.cases = 8 if large else 16
    if a.dims is None:
        a.dims = "256,256,128" if large else "64,64,32"
    if a.inner_product is None:
        a.inner_product = "tc" if large and a.element == "tet4" and a.precision == "mixed" else "fp32"
    if a.s_max is None:     # (10-node tets: s = 32 overfits on the medium box, one case's guess 7x worse than AB4)
        a.s_max = 16 if large or a.element == "tet10" else 32
    if a.comparator_steps is None:     # (large: the plain FP64 comparators need minutes; run them on request)
        a.comparator_steps = 0 if large else 4
    if a.comparator_spinup is None:
        a.comparator_spinup = 10 if large else 30
    if a.cpu_dims is None:
        a.cpu_dims = "32,32,16" if large else a.dims
    return a


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_first_case(rank, cases):
    """Cases are sharded by rank: rank k steps the recipe's cases k * cases .. (k + 1) * cases - 1."""
    return rank * cases


def max_over_ranks(x, ws, device):
    """The largest value of x over the job's ranks (the slowest rank's time); x itself for one rank."""
    if ws == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


def job_value(ws, cases_per_rank, steps, t_max_ms):
    """Whole-job case-steps per second: all ranks' case-steps over the slowest rank's time."""
    return ws * cases_per_rank * steps / (t_max_ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def ncu_traffic(kernel_tag, sources):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of one kernel, from the committed
    ncu summary profiles/<kernel_tag>.md, or None when that summary is missing or the kernel's source files
    changed since it was taken (the summary records their sha256)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", kernel_tag + ".md")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    traffic, digest = None, None
    for line in open(path):
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1])
        elif line.startswith("source_sha256:"):
            digest = line.split(":", 1)[1].strip()
    return traffic if digest == h.hexdigest() else None


EBE_SOURCES = ["paper_2409_20380_gb300/csrc/k_ebe.cu", "paper_2409_20380_gb300/csrc/fem_internal.cuh"]
BCSR_SOURCES = ["paper_2409_20380_gb300/csrc/k_bcsr.cu"]


def kuhn_grid_nnz(Hx, Hy, Hz):
    """Node-pair blocks of the assembled operator of a Kuhn-split Hx x Hy x Hz hex grid: every node with itself
    and both directions of every element edge -- the grid's axis edges, one diagonal per hex face and one
    body diagonal per hex (equal to the pattern the library assembles; checked against np.unique of the
    element node pairs on small grids)."""
    n = (Hx + 1) * (Hy + 1) * (Hz + 1)
    axis = Hx * (Hy + 1) * (Hz + 1) + (Hx + 1) * Hy * (Hz + 1) + (Hx + 1) * (Hy + 1) * Hz
    faces = Hx * Hy * (Hz + 1) + Hx * (Hy + 1) * Hz + (Hx + 1) * Hy * Hz
    return n + 2 * (axis + faces + Hx * Hy * Hz)


def make_mesh(config, dims):
    from paper_2409_20380_gb300 import workload as wl
    Hx, Hy, Hz = (int(v) for v in dims.split(","))
    if config == "large":
        return wl.config4_mesh(Hx, Hy, Hz), wl.config4_time_params()
    return wl.config2_mesh(Hx, Hy, Hz), wl.config2_time_params()


def make_sources(config, mesh, n_cases, first_case=0):
    from paper_2409_20380_gb300 import workload as wl
    if config == "large":
        return wl.config4_sources(mesh, n_cases, first_case=first_case)
    return wl.config2_sources(mesh, n_cases, first_case=first_case)


def workload(args, rank):
    from paper_2409_20380_gb300 import workload as wl
    mesh, tp = make_mesh(args.config, args.dims)
    if args.source == "impulses":
        npts = args.impulse_points or max(1, int(0.07 * wl.surface_nodes(mesh).size))
        cfg = 4 if args.config == "large" else 2
        first = rank_first_case(rank, args.cases)
        srcs = [wl.random_impulses(mesh, wl.rng_for(cfg, 0, first + c, 4), npts, args.impulse_steps)
                for c in range(args.cases)]
    else:
        srcs = make_sources(args.config, mesh, args.cases, first_case=rank_first_case(rank, args.cases))
    return mesh, srcs, tp, wl.region_map(mesh, args.region_nodes)


def margin_kw(args):
    """fem_opts overrides of the inner solves (their aim, their CG product) and of the guess guard given on
    the command line."""
    kw = {} if args.inner_margin is None else {"inner_margin": args.inner_margin}
    if args.inner_product == "tc":
        kw["inner_product"] = 1
    if args.no_guard:
        kw["pred_guard"] = 0
    return kw


def add_case(fem, bt, h, s):
    if hasattr(s, "steps"):
        return fem.fem_case_add_impulses(bt, h, s)
    return fem.fem_case_add(bt, h, s)


def _oracle_case(config, dims, case, predictor, s_max, region_nodes, spinup, steps, barrier, out, source="ricker",
                 absorbing=False, impulse_steps=100):
    """One case of the oracle sample, in its own (spawned) process: the FP64 oracle as it stands on the
    sample mesh, `spinup` steps from rest, then `steps` timed steps after every process is ready."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2409_20380_gb300 import workload as wl
    mesh, tp = make_mesh(config, dims)
    if source == "impulses":
        npts = max(1, int(0.07 * wl.surface_nodes(mesh).size))
        src = wl.random_impulses(mesh, wl.rng_for(4 if config == "large" else 2, 0, case, 4), npts, impulse_steps)
    else:
        src = make_sources(config, mesh, case + 1)[case]
    sysm, A = oracle.build_system(mesh, tp, absorbing_faces=wl.side_faces(mesh) if absorbing else None)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    sim = oracle.CaseSimulator(sysm, A, Binv, src, predictor=predictor, s_max=s_max,
                               region_of_node=wl.region_map(mesh, region_nodes))
    for _ in range(spinup):
        sim.step()
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    its = 0
    for _ in range(steps):
        its += sim.step().iters
    t1 = time.perf_counter()
    out.put((case, t0, t1, its))


def oracle_sample(args, n_procs, spinup, steps):
    """Runs the oracle on n_procs cases at once (one spawned process per case, single-threaded each) on the
    --cpu-dims sample mesh; returns case-steps/s measured there and scaled to the full mesh by the DOF ratio."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    barrier = ctx.Barrier(n_procs) if n_procs > 1 else None
    pred = "dd" if args.predictor == "dd" else "ab4"
    procs = [ctx.Process(target=_oracle_case, args=(args.config, args.cpu_dims, c, pred, args.s_max,
                                                    args.region_nodes, spinup, steps, barrier, out, args.source,
                                                    args.absorbing, args.impulse_steps))
             for c in range(n_procs)]
    for p in procs:
        p.start()
    res = [out.get() for _ in procs]
    for p in procs:
        p.join()
    t0 = min(r[1] for r in res)
    t1 = max(r[2] for r in res)
    its = sum(r[3] for r in res)
    sub = [int(v) for v in args.cpu_dims.split(",")]
    full = [int(v) for v in args.dims.split(",")]
    n_sub = 3 * (sub[0] + 1) * (sub[1] + 1) * (sub[2] + 1)
    n_full = 3 * (full[0] + 1) * (full[1] + 1) * (full[2] + 1)
    v_sub = n_procs * steps / (t1 - t0)
    return {"value_sample": v_sub, "value_full": v_sub * n_sub / n_full, "dof_sample": n_sub, "dof_full": n_full,
            "seconds": t1 - t0, "cg_iters_per_case_step": its / (n_procs * steps), "procs": n_procs}


def cpu_baseline(args):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: --cpu-dims sub-box of the same
    recipe (the same mesh for medium), steps cpu_spinup+1 .. cpu_spinup+cpu_steps from rest; timed on one
    core alone and then with one process per case on min(cores, cases) cores."""
    n_all = args.cpu_procs or max(1, min(os.cpu_count() or 1, args.cases))
    one = oracle_sample(args, 1, args.cpu_spinup, args.cpu_steps)
    allc = oracle_sample(args, n_all, args.cpu_spinup, args.cpu_steps) if n_all > 1 else one
    extrap = args.cpu_dims != args.dims
    w0, w1 = args.cpu_spinup + 1, args.cpu_spinup + args.cpu_steps
    sample = (f"oracle (scipy CSR FP64 Algorithm 1 + regional MGS, single-threaded per process) on "
              f"{'a ' + args.cpu_dims.replace(',', 'x') + ' hex sub-box of the same recipe' if extrap else 'the same mesh'}"
              f" ({allc['dof_sample']} DOF), cases 0-{n_all - 1} of its sources, steps {w0}-{w1} from rest, "
              f"{allc['cg_iters_per_case_step']:.2f} CG iterations per case-step; "
              + (f"case-steps/s scaled to the full mesh by the DOF ratio {allc['dof_sample']}/{allc['dof_full']} "
                 f"(extrapolated)" if extrap else "measured on the full mesh"))
    return {"value": allc["value_full"], "unit": UNIT, "cores": n_all, "kind": "oracle", "sample": sample,
            "extrapolated": extrap, "value_on_sample": allc["value_sample"], "seconds": allc["seconds"],
            "cg_iters_per_case_step": allc["cg_iters_per_case_step"],
            "single_core": {"value": one["value_full"], "value_on_sample": one["value_sample"], "cores": 1,
                            "seconds": one["seconds"], "cg_iters_per_case_step": one["cg_iters_per_case_step"]}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n_all = args.cpu_procs or max(1, min(os.cpu_count() or 1, args.cases))
    r = oracle_sample(args, n_all, args.cpu_spinup + args.warmup, args.steps)
    value = r["value_full"]
    extrap = args.cpu_dims != args.dims
    sample = (f"one process per case ({n_all} cases, one core each) on "
              f"{'a ' + args.cpu_dims.replace(',', 'x') + ' hex sub-box of the same recipe' if extrap else 'the same mesh'}"
              f" ({r['dof_sample']} DOF); {args.cpu_spinup} spin-up + {args.warmup} warm-up steps from rest, then "
              f"{args.steps} timed steps of every case ({r['cg_iters_per_case_step']:.2f} CG iterations per "
              f"case-step)" + (f"; case-steps/s scaled to the full mesh by the DOF ratio "
                               f"{r['dof_sample']}/{r['dof_full']} (extrapolated)" if extrap else ""))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_all, "kind": "oracle", "sample": sample,
                         "extrapolated": extrap, "value_on_sample": r["value_sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def config_dict(args, mesh=None):
    if mesh is None:     # sizes of the Kuhn-split hex box without building it
        Hx, Hy, Hz = (int(v) for v in args.dims.split(","))
        mesh = argparse.Namespace(n_elems=6 * Hx * Hy * Hz, n_nodes=(Hx + 1) * (Hy + 1) * (Hz + 1))
    solver = ("FP32-inner/FP64-refined" if args.precision == "mixed" else "FP64") + " block-Jacobi EBE-PCG to rel. residual 1e-8"
    pred = "data-driven predictor s=%d" % args.s_max if args.predictor == "dd" else "AB4 predictor"
    if args.cpu_predictor:
        pred = ("data-driven predictor on the host CPU (two case sets alternating, s balanced against the solve "
                "time, at most %d)" % args.s_max)
    src = ("random surface impulses" if args.source == "impulses" else "Ricker point sources") + \
        (", absorbing sides" if args.absorbing else "")
    if args.config == "large":
        name = (f"large: {args.dims.replace(',', 'x')} hex box (h=1/64) split into {mesh.n_elems} tets "
                f"({mesh.n_nodes} nodes), 5 layers + low-velocity basin, {args.cases} cases on one mesh ({src}), "
                f"{solver}, {pred}")
    else:
        name = (f"medium: {args.dims.replace(',', 'x')} hex box split into {mesh.n_elems} tets "
                f"({mesh.n_nodes} nodes), {args.cases} cases on one mesh ({src}), {solver}, {pred}")
    return {"workload": name, "mesh_hex": args.dims, "n_elems": mesh.n_elems, "n_nodes": mesh.n_nodes,
            "cases_per_gpu": args.cases, "precision": args.precision, "predictor": args.predictor,
            "s_max": args.s_max, "cert_product": args.cert, "region_nodes": args.region_nodes, "tol": 1e-8,
            "inner_margin": args.inner_margin if args.inner_margin is not None else 0.5,
            "inner_product": ("FP16 hex element matrices on the tensor cores in passes whose reduction targets "
                              "are 1e-3 or coarser, FP32 element kernels otherwise") if args.inner_product == "tc"
                             else "FP32 element kernels",
            "guess_guard": args.predictor == "dd" and not args.no_guard,
            "spinup_steps": args.spinup, "source": args.source, "absorbing_sides": args.absorbing,
            "cpu_predictor": args.cpu_predictor,
            "l2": "inputs larger than L2: each step streams the cases' state and the snapshot ring (>1 GB)",
            "parallelism": "replicas"}


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    log("building the workload")
    mesh, srcs, tp, regions = workload(args, rank)
    log(f"mesh: {mesh.n_elems} tets, {mesh.n_nodes} nodes")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER if args.precision == "mixed" else fem.FEM_FP64,
                                predictor=fem.FEM_PRED_DD if args.predictor == "dd" else fem.FEM_PRED_AB4,
                                s_max=args.s_max, snapshot_format=args.snapshot_format, tol=1e-8, cert_df=args.cert,
                                use_graph=0 if args.no_graph else 1, check_every=args.check_every,
                                cpu_predictor=1 if args.cpu_predictor else 0, **margin_kw(args))
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_set_regions(h, regions)
    if args.absorbing:
        fem.fem_mesh_set_absorbing(h, wl.side_faces(mesh))
    if args.variant or args.hex_per_tile:
        fem.fem_mesh_tune(h, args.variant, args.hex_per_tile)
    bt = fem.fem_batch_create(opts)
    nc = len(srcs)
    for s in srcs:
        add_case(fem, bt, h, s)
    log("library mesh and batch created")
    fem.fem_step(bt, args.spinup, nc)
    free_b, total_b = torch.cuda.mem_get_info()
    log(f"{args.spinup} spin-up steps done; device memory in use {(total_b - free_b) / 1e9:.1f} of {total_b / 1e9:.1f} GB")
    fem.fem_step(bt, args.warmup, nc)
    # ---- timed region: device-resident, CUDA events on the batch stream ----
    dropped0 = sum(fem.fem_case_stats(bt, c)["fallbacks"] for c in range(nc))
    sampler = ClockSampler(local)
    fem.fem_batch_profile(bt, 2)        # count launches only: the step graph stays a graph
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()        # ncu --profile-from-start off captures the timed region only
    ev0.record(stream)
    st, iters, relres = fem.fem_step(bt, args.steps, nc)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier()
    clocks = sampler.stop()
    log(f"timed region: {args.steps} steps")
    launches = fem.fem_batch_profile(bt, 0)["kernel_launches"]
    dropped = sum(fem.fem_case_stats(bt, c)["fallbacks"] for c in range(nc)) - dropped0
    ms = ev0.elapsed_time(ev1)
    # per-kernel-class device times: CUDA events around each launch over the next --profile-steps steps
    # (eager launches of the same kernels; events cannot sit inside the graph's conditional loops)
    # The inner loop issues its launches in chunks of check_every iterations; those after the slowest case
    # has converged return at once.  Launches that did work: per step, the slowest case's inner iterations
    # (one refinement pass per step here) plus the product of the predictor's correction.
    fem.fem_batch_profile(bt, 1)
    working32 = 0
    for _ in range(max(1, args.profile_steps)):
        _, it_k, _ = fem.fem_step(bt, 1, nc)
        working32 += int(it_k.max()) + (1 if args.predictor == "dd" else 0)
    prof = fem.fem_batch_profile(bt, 0)
    t_max = max_over_ranks(ms, ws, "cuda")
    value = job_value(ws, nc, args.steps, t_max)
    # ---- end to end through the public API: H2D loads, step, D2H displacements ----
    N = mesh.n_nodes
    step0 = fem.fem_batch_steps(bt)
    ne = args.e2e_steps
    ricker = args.source == "ricker"
    loads = torch.zeros((ne + 2, nc, 3), dtype=torch.float64).pin_memory()
    for k in range(ne + 2):
        tk = (step0 + 1 + k) * tp.dt
        for c, s in enumerate(srcs):
            if ricker:
                loads[k, c] = torch.from_numpy(wl.ricker_load(s, tk))
    # each step's loads come from pinned host memory and its displacement fields go to alternating pinned
    # host buffers; steps are queued without host waits, the copy of step k runs on the batch's copy stream
    # while step k+1 computes, and fem_batch_sync (which also checks every step's status) ends the region
    u_host = [torch.empty(nc * N * 3, dtype=torch.float64).pin_memory() for _ in range(2)]
    for k in range(2):
        if ricker:
            fem.fem_batch_set_loads(bt, loads[k])
        fem.fem_step(bt, 1, nc)
        fem.fem_batch_get_field_async(bt, fem.FEM_FIELD_U, u_host[k % 2])
    fem.fem_batch_sync(bt)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(2, ne + 2):
        if ricker:
            fem.fem_batch_set_loads(bt, loads[k])
        fem.fem_step_async(bt, 1)
        fem.fem_batch_get_field_async(bt, fem.FEM_FIELD_U, u_host[k % 2])
    fem.fem_batch_sync(bt)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, ws, "cuda")
    log("end-to-end region done")
    e2e = {"value": job_value(ws, nc, ne, 1e3 * e2e_s), "unit": UNIT, "h2d_bytes_per_step": nc * 3 * 8 if ricker else 0,
           "d2h_bytes_per_step": nc * N * 3 * 8, "steps": ne}
    # ---- plain FP64 PCG with Adams-Bashforth on the same state: with the EBE product (the comparator) and
    # with the assembled 3x3-block product (the CRS-style form the paper compares the EBE with) ----
    comparator = crs_comparator = None
    if not args.no_comparator and args.comparator_steps > 0:
        runs = {}
        for name, variant in (("ebe", 0), ("crs", 8)):
            fem.fem_mesh_tune(h, variant, 0)
            cmp_opts = fem.fem_opts_default(precision=fem.FEM_FP64, predictor=fem.FEM_PRED_AB4, tol=1e-8)
            bt2 = fem.fem_batch_create(cmp_opts)
            for s in srcs:
                add_case(fem, bt2, h, s)
            # same physics from rest is not the same state; run the comparator on the steps right after a
            # short spin-up so its iteration counts are those of a developed wavefield
            fem.fem_step(bt2, args.comparator_spinup, nc)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st2, it2, rr2 = fem.fem_step(bt2, args.comparator_steps, nc)
            e1.record(stream)
            torch.cuda.synchronize()
            runs[name] = (e0.elapsed_time(e1), float(it2.sum()) / (nc * args.comparator_steps))
            fem.fem_batch_destroy(bt2)
        fem.fem_mesh_tune(h, args.variant, args.hex_per_tile)
        steps_w = "steps %d-%d" % (args.comparator_spinup + 1, args.comparator_spinup + args.comparator_steps)
        comparator = {"value": nc * args.comparator_steps / (runs["ebe"][0] / 1e3), "unit": UNIT,
                      "what": "plain FP64 EBE-PCG + Adams-Bashforth, same GPU, " + steps_w,
                      "cg_iters_per_case_step": runs["ebe"][1]}
        crs_comparator = {"value": nc * args.comparator_steps / (runs["crs"][0] / 1e3), "unit": UNIT,
                          "what": "plain FP64 PCG with the assembled 3x3-block (CRS-style) product + "
                                  "Adams-Bashforth, same GPU, " + steps_w,
                          "cg_iters_per_case_step": runs["crs"][1]}
    if rank != 0:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    # ---- rooflines: the FP32 EBE product of the inner solve and the certification product; the one with
    # the larger measured time per step is the dominant kernel ----
    hbm_peak, peak_kind, sm_max = peaks()
    E = mesh.n_elems
    rpad = 1 << (nc - 1).bit_length()
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    alu32 = n_sm * 128 * 2 * sm_max * 1e6 / 1e12      # FP32: SMs x 128 lanes x FMA x max clock
    alu64 = n_sm * 2 * 2 * sm_max * 1e6 / 1e12        # FP64: SMs x 2 DFMA/clk x 2 flops x max clock
    inner = None
    if prof["ebe32_launches"] > 0:
        avg32 = prof["ebe32_ms"] / max(1, min(working32, prof["ebe32_launches"]))
        bytes32 = E * (16 + 12 * 4) + rpad * N * 3 * (4 + 4)
        fl = FLOP_PER_ELEM_CASE * E * rpad
        gbs = bytes32 / (avg32 * 1e-3) / 1e9
        inner = {"bound": "alu", "achieved": fl / (avg32 * 1e-3) / 1e12, "peak": alu32, "unit": "TFLOP/s",
                 "frac": fl / (avg32 * 1e-3) / 1e12 / alu32,
                 "peak_kind": "derived: %d SMs x 128 FP32 lanes x 2 flops x max SM clock" % n_sm,
                 "traffic": ncu_traffic("ebe_packed_f32_%s%d" % (args.config, rpad), EBE_SOURCES) if not args.variant else None,
                 "kernel": ("k_ebe_hex_staged<float,1,0,1> (FP32 EBE product A p of the inner PCG, TMA-staged "
                            "hex tiles, two cases per thread; %d cases)" % rpad),
                 "avg_launch_ms": avg32, "launches": working32, "launches_issued": prof["ebe32_launches"],
                 "launch_note": "launches that did work (the slowest case's inner iterations + the correction's "
                                "product per step); avg_launch_ms = all launches' time over them",
                 "alg_bytes_per_launch": bytes32,
                 "alg_flops_per_launch": fl, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak, "hbm_peak": hbm_peak,
                 "hbm_peak_kind": peak_kind, "ms_per_step": prof["ebe32_ms"] / max(prof["steps"], 1)}
    if args.inner_product == "tc" and prof.get("ebe16_launches", 0) > 0:
        # the inner CG products on the tensor cores: per hex a 784-byte FP16 matrix record and its corner
        # table (16 bytes), p read and q written in FP32; four mma.sync a hex and 8 cases
        H = E // 6
        working16 = max(1, working32 - (args.profile_steps if args.predictor == "dd" else 0))
        avg16 = prof["ebe16_ms"] / max(1, min(working16, prof["ebe16_launches"]))
        bytes16 = H * (784 + 16) + rpad * N * 3 * (4 + 4)
        fl16 = H * (rpad // 8) * 2 * (16 * 8 * 16 + 16 * 8 * 8) * 2
        gbs = bytes16 / (avg16 * 1e-3) / 1e9
        inner = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                 "peak_kind": peak_kind,
                 "traffic": ncu_traffic("ebe_tc_f16_%s%d" % (args.config, rpad), EBE_SOURCES),
                 "kernel": ("k_ebe_hex_tc<true> (inner PCG product A p with FP16 hex element matrices on the tensor "
                            "cores (mma.sync), FP32 vectors; %d cases)" % rpad),
                 "avg_launch_ms": avg16, "launches": working16, "launches_issued": prof["ebe16_launches"],
                 "launch_note": "launches that did work (the slowest case's inner iterations per step)",
                 "alg_bytes_per_launch": bytes16, "alg_tensor_flops_per_launch": fl16,
                 "tensor_tflops": fl16 / (avg16 * 1e-3) / 1e12,
                 "ms_per_step": prof["ebe16_ms"] / max(prof["steps"], 1),
                 "correction_product_ms_per_step": prof["ebe32_ms"] / max(prof["steps"], 1)}
    cert = None
    if prof["ebe64_launches"] > 0:
        avg = prof["ebe64_ms"] / prof["ebe64_launches"]
        if args.cert in (2, 3):
            nnz = kuhn_grid_nnz(*mesh.dims)
            bytes_c = nnz * (4 + 80) + N * 4 + rpad * N * 3 * (8 + 8 + 8 + (16 if args.cert == 3 else 0))
            if args.cert == 3:     # per block and case: 12 double-float FMAs of 14 FP32 flops each
                fl = 12 * 14 * nnz * rpad
                roof = {"bound": "alu", "peak": alu32, "peak_kind": "derived: FP32 lanes x max SM clock"}
                kname = ("k_bcsr_split_df2 (certification product M p, K p: assembled 3x3 blocks, double-float, "
                         "two cases a thread)" if rpad >= 2 else
                         "k_bcsr_split_df (certification product M p, K p: assembled 3x3 blocks, double-float)")
            else:
                fl = 12 * 2 * nnz * rpad
                roof = {"bound": "alu", "peak": alu64, "peak_kind": "derived: %d SMs x 2 DFMA/clk x max SM clock" % n_sm}
                kname = "k_bcsr_split_f64 (certification product M p, K p: assembled 3x3 blocks, FP64)"
            roof.update({"nnz_blocks": nnz})
        else:
            fl = FLOP_PER_ELEM_CASE_SPLIT * E * rpad
            bytes_c = E * (16 + 12 * 8) + rpad * N * 3 * (8 + 8 + 8)
            roof = {"bound": "alu", "peak": alu64, "peak_kind": "derived: %d SMs x 2 DFMA/clk x max SM clock" % n_sm}
            kname = "k_ebe_split%s (certification product M p, K p, element by element)" % ("_df" if args.cert == 1 else "")
        achieved = fl / (avg * 1e-3) / 1e12
        gbs = bytes_c / (avg * 1e-3) / 1e9
        roof.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / roof["peak"],
                     "traffic": (ncu_traffic("ebe_split_f64_%s%d" % (args.config, rpad), EBE_SOURCES) if args.cert == 0 else
                                 ncu_traffic("bcsr_split_df_%s%d" % (args.config, rpad), BCSR_SOURCES) if args.cert == 3 else None),
                     "kernel": kname + ", %d cases" % rpad, "avg_launch_ms": avg, "launches": prof["ebe64_launches"],
                     "alg_bytes_per_launch": bytes_c, "alg_flops_per_launch": fl, "hbm_gbs": gbs,
                     "hbm_frac": gbs / hbm_peak, "hbm_peak": hbm_peak,
                     "ms_per_step": prof["ebe64_ms"] / max(prof["steps"], 1)})
        cert = roof
    if inner is not None and (cert is None or inner["ms_per_step"] >= cert["ms_per_step"]):
        roof, other = inner, cert
    else:
        roof, other = cert, inner
    log("comparators and rooflines done")
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(args)
        log("oracle baseline done")
    balance = None
    if args.cpu_predictor:
        balance = [fem.fem_batch_predictor_balance(bt, c) for c in (0, 1)]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": config_dict(args, mesh), "roofline": roof, "roofline_second": other, "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks,
        "step_graph": not args.no_graph,
        "kernel_timing": f"CUDA events around each launch over the {prof['steps']} steps after the timed region "
                         f"(eager launches of the same kernels)",
        "cg_iters_per_case_step": float(iters.sum()) / (nc * args.steps),
        "max_certified_relres": float(relres.max()), "status": int(st),
        "guess_guard_dropped": dropped,
        "phase_ms_per_step": {k: prof[k] / max(prof["steps"], 1) for k in
                              ("predict_ms", "rhs_ms", "solve_ms", "update_ms")},
        "kernel_ms_per_step": {"ebe32": prof["ebe32_ms"] / max(prof["steps"], 1),
                               "ebe64": prof["ebe64_ms"] / max(prof["steps"], 1),
                               "cg_vec": prof["cg_vec_ms"] / max(prof["steps"], 1),
                               "ebe16": prof["ebe16_ms"] / max(prof["steps"], 1)},
        "kernel_launches_per_step": {"ebe32": prof["ebe32_launches"] / max(prof["steps"], 1),
                                     "ebe16": prof["ebe16_launches"] / max(prof["steps"], 1),
                                     "ebe64": prof["ebe64_launches"] / max(prof["steps"], 1),
                                     "cg_vec": prof["cg_vec_launches"] / max(prof["steps"], 1),
                                     "all": prof["kernel_launches"] / max(prof["steps"], 1)},
        "host_predictor_balance": balance,
        "fp64_plain_comparator": comparator,
        "fp64_crs_comparator": crs_comparator,
    }
    print(json.dumps(out), flush=True)
    fem.fem_batch_destroy(bt)
    fem.fem_mesh_destroy(h)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_kernel(args):
    """Times the EBE product alone (CUDA events, inputs resident) on the --dims mesh with --cases cases."""
    import numpy as np
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    mesh, tp = make_mesh(args.config, args.dims)
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_tune(h, args.variant, args.hex_per_tile)
    r = args.cases
    dt = torch.float32 if args.kernel_precision == "fp32" else torch.float64
    g = torch.Generator(device="cuda").manual_seed(0)
    p = torch.randn(mesh.n_nodes * 3 * r, device="cuda", dtype=dt, generator=g)
    p.view(mesh.n_nodes, 3, r)[torch.from_numpy(mesh.fixed_dof.reshape(-1, 3).astype(bool)).cuda()] = 0
    q = torch.empty_like(p)
    ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    for _ in range(args.warmup):
        fem.fem_ebe_apply(h, p, q, r, cM, cK, ptq)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fem.fem_ebe_apply(h, p, q, r, cM, cK, ptq)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    w = 4 if args.kernel_precision == "fp32" else 8
    E, N = mesh.n_elems, mesh.n_nodes
    bytes_launch = E * (16 + 12 * w) + r * N * 3 * 2 * w
    if args.variant == 9 and args.kernel_precision == "fp32":   # FP16 hex records and corner tables
        bytes_launch = (E // 6) * (784 + 16) + r * N * 3 * 2 * w
    info = fem.fem_mesh_info(h)
    print(json.dumps({"kernel": "ebe", "precision": args.kernel_precision, "dims": args.dims, "cases": r,
                      "variant": args.variant, "hex_per_tile": args.hex_per_tile, "mesh_info": info,
                      "ms_per_launch": ms, "alg_gbs": bytes_launch / (ms * 1e-3) / 1e9,
                      "alg_tflops": FLOP_PER_ELEM_CASE * E * r / (ms * 1e-3) / 1e12,
                      "note": "includes the q zero-fill and the Dirichlet mask pass of fem_ebe_apply"}), flush=True)
    fem.fem_mesh_destroy(h)


# Tet10 product as executed: per Gauss point the corner-weighted sums W_a (84 flops), G = sum W_a g_a^T (63),
# the stress (21), T_a = sigma g_a (60), the nodal forces (78) and the point's coefficients (12): 318; four
# points, plus the consistent mass through its corner and edge sums (~100 a component, 300): ~1.57 kflop per
# element and case (FMA = 2)
FLOP_PER_TET10_CASE = 4 * 318 + 300


def run_kernel10(args):
    """Times the tet10 EBE product alone (CUDA events, inputs resident) on the --dims mesh turned into 10-node
    tets (edge midpoints), --cases cases."""
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    Hx, Hy, Hz = (int(v) for v in args.dims.split(","))
    mesh = wl.tet10_mesh(wl.config2_mesh(Hx, Hy, Hz))
    tp = wl.config2_time_params()
    h = fem.fem_mesh10_create(mesh)
    r = args.cases
    dt = torch.float32 if args.kernel_precision == "fp32" else torch.float64
    g = torch.Generator(device="cuda").manual_seed(0)
    p = torch.randn(mesh.n_nodes * 3 * r, device="cuda", dtype=dt, generator=g)
    p.view(mesh.n_nodes, 3, r)[torch.from_numpy(mesh.fixed_dof.reshape(-1, 3).astype(bool)).cuda()] = 0
    q = torch.empty_like(p)
    ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    for _ in range(args.warmup):
        fem.fem_ebe10_apply(h, p, q, r, cM, cK, ptq)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fem.fem_ebe10_apply(h, p, q, r, cM, cK, ptq)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    w = 4 if args.kernel_precision == "fp32" else 8
    E, N = mesh.n_elems, mesh.n_nodes
    bytes_launch = E * (40 + 12 * w) + r * N * 3 * 2 * w
    print(json.dumps({"kernel": "ebe10", "precision": args.kernel_precision, "dims": args.dims, "cases": r,
                      "n_elems": E, "n_nodes": N, "ms_per_launch": ms,
                      "alg_gbs": bytes_launch / (ms * 1e-3) / 1e9,
                      "alg_tflops": FLOP_PER_TET10_CASE * E * r / (ms * 1e-3) / 1e12,
                      "flop_per_elem_case": FLOP_PER_TET10_CASE,
                      "note": "one thread per (element, case), global atomics; includes the q zero-fill and "
                              "the Dirichlet mask pass"}), flush=True)
    fem.fem_mesh10_destroy(h)


def run_pcg10(args):
    """Plain FP64 PCG with the tet10 EBE product on the --dims grid as tet10, --cases cases, from a zero guess
    against a right-hand side M v (v random on the free DOFs): time and iterations of one solve."""
    import numpy as np
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    Hx, Hy, Hz = (int(v) for v in args.dims.split(","))
    mesh = wl.tet10_mesh(wl.config2_mesh(Hx, Hy, Hz))
    tp = wl.config2_time_params()
    h = fem.fem_mesh10_create(mesh)
    r = args.cases
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    g = torch.Generator(device="cuda").manual_seed(1)
    v = torch.randn(mesh.n_nodes * 3 * r, device="cuda", dtype=torch.float64, generator=g)
    v.view(mesh.n_nodes, 3, r)[torch.from_numpy(mesh.fixed_dof.reshape(-1, 3).astype(bool)).cuda()] = 0
    b = torch.empty_like(v)
    fem.fem_ebe10_apply(h, v, b, r, 1.0, 0.0)          # b = M v: a smooth, mass-weighted load
    x = torch.zeros_like(b)
    prec = fem.FEM_FP64 if args.kernel_precision == "fp64" else fem.FEM_FP32_INNER
    fem.pcg10_solve(h, b, x, r, cM, cK, tol=1e-8, precision=prec)     # warm-up (allocations, first launches)
    x.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    iters, relres = fem.pcg10_solve(h, b, x, r, cM, cK, tol=1e-8, precision=prec)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"kernel": "pcg10", "precision": "fp64" if prec == fem.FEM_FP64 else "fp32-inner/fp64",
                      "dims": args.dims, "cases": r,
                      "n_elems": mesh.n_elems, "n_nodes": mesh.n_nodes, "ms_per_solve": ms,
                      "iters": [int(i) for i in iters], "max_relres": float(np.max(relres)),
                      "ms_per_iteration": ms / max(1, int(np.max(iters))),
                      "note": "block-Jacobi PCG, tet10 EBE product, zero guess, certified tol 1e-8 (FP64 residual)"}),
          flush=True)
    fem.fem_mesh10_destroy(h)


def run_learned(args):
    """Learned proposal on the medium mesh: samples from --train-cases cases x --case-steps steps, Adam on
    the GPU, then --eval-cases held-out cases with and without the network (same certified tolerance)."""
    import numpy as np
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    Hx, Hy, Hz = (int(v) for v in args.dims.split(","))
    mesh = wl.config2_mesh(Hx, Hy, Hz)
    tp = wl.config2_time_params()
    if args.dt:
        tp.dt = args.dt
    regions = wl.region_map(mesh, args.region_nodes)
    R = int(regions.max()) + 1
    train_src, held_src = wl.config5_sources(mesh, args.train_cases, args.eval_cases)
    residual = args.loss == "residual"
    tw = fem.FEM_MLP_RES if residual else 32
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_set_regions(h, regions)
    K = args.case_steps
    # both arms step eagerly (the proposal is not captured in the step graph) and without the guess guard
    # (steps that take a proposal skip it): the same mode for both
    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=args.s_max,
                                tol=1e-8, snapshot_format=args.snapshot_format, cert_df=args.cert, use_graph=0,
                                pred_guard=0)

    counts = [0, 0]

    def run(srcs, net=None, xs=None, ts=None, window=(250, 500)):
        """Cases in batches of --cases; returns (rows collected, case-steps/s over the window, iterations,
        log initial residuals over the window)."""
        rows, t_win, cs_win, its, logs = 0, 0.0, 0, 0, []
        counts[:] = [0, 0]
        for g0 in range(0, len(srcs), args.cases):
            grp = srcs[g0:g0 + args.cases]
            bt = fem.fem_batch_create(opts)
            for s_ in grp:
                fem.fem_case_add(bt, h, s_)
            if net is not None:
                fem.fem_batch_set_mlp(bt, net)
            nc = len(grp)
            w0, w1 = min(window[0], K), min(window[1], K)
            done = 0
            if xs is not None:
                done = min(args.collect_from, w0)
                fem.fem_step(bt, done, nc)
                (fem.fem_batch_collect_residual if residual else fem.fem_batch_collect)(bt, xs[rows:], ts[rows:])
            fem.fem_step(bt, w0 - done, nc)
            for k in range(w0, w1):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st, it, rr = fem.fem_step(bt, 1, nc)
                e1.record(stream)
                torch.cuda.synchronize()
                t_win += e0.elapsed_time(e1) / 1e3
                cs_win += nc
                its += int(it.sum())
                for c in range(nc):
                    logs.append(math.log(max(fem.fem_case_stats(bt, c)["init_relres"], 1e-30)))
            if K > w1:
                fem.fem_step(bt, K - w1, nc)
            if xs is not None:
                rows += fem.fem_batch_collected(bt)[0]
            if net is not None:
                tk, rj = fem.fem_batch_proposal_counts(bt)
                counts[0] += tk
                counts[1] += rj
            fem.fem_batch_destroy(bt)
        return rows, (cs_win / t_win if t_win > 0 else None), its, logs

    cap = len(train_src) * K * R
    xs = torch.empty((cap, 64), device="cuda")
    ts = torch.empty((cap, tw), device="cuda")
    t0 = time.perf_counter()
    rows, _, _, _ = run(train_src, xs=xs, ts=ts, window=(K, K))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    th0 = wl.mlp_init_weights(0).astype(np.float32)
    if residual:      # zero output layer: the untrained network proposes no correction (the plain predictor)
        th0[-(32 * 256 + 32):] = 0.0
    net = fem.fem_mlp_create(th0)
    g = torch.Generator(device="cuda").manual_seed(0)
    order = torch.randint(0, rows, (args.updates, args.batch), device="cuda", generator=g, dtype=torch.int32)
    t0 = time.perf_counter()
    losses = (fem.fem_mlp_train_residual if residual else fem.fem_mlp_train)(net, xs[:rows], ts[:rows], order,
                                                                              lr=args.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # loss of the zero correction (the plain predictor): mean of ||w||^2, or of the squared targets
    train_var = float((ts[:rows, -32:] ** 2).sum(dim=1).mean()) if residual else float((ts[:rows] ** 2).mean())
    del xs, ts
    hcap = len(held_src) * K * R
    hx = torch.empty((hcap, 64), device="cuda")
    ht = torch.empty((hcap, tw), device="cuda")
    hrows, v_dd, it_dd, log_dd = run(held_src, xs=hx, ts=ht)
    held_loss, n_l = 0.0, 0
    for a in range(0, hrows, 65536):
        b = min(hrows, a + 65536)
        held_loss += (fem.fem_mlp_loss_grad_residual if residual else fem.fem_mlp_loss_grad)(net, hx[a:b], ht[a:b]) * (b - a)
        n_l += b - a
    held_loss /= max(n_l, 1)
    held_var = float((ht[:hrows, -32:] ** 2).sum(dim=1).mean()) if residual else float((ht[:hrows] ** 2).mean())
    del hx, ht
    _, v_ml, it_ml, log_ml = run(held_src, net=net)
    print(json.dumps({
        "metric": "learned proposal: held-out time-steps/s and CG iterations at rel. residual 1e-8",
        "unit": UNIT, "value": v_ml, "plain_dd_value": v_dd,
        "config": {"workload": f"medium {args.dims.replace(',', 'x')} mesh, {len(train_src)} training + "
                               f"{len(held_src)} held-out cases x {K} steps, window steps 251-{min(500, K)}, "
                               f"s={args.s_max}, regions of {args.region_nodes} nodes ({R}), dt={tp.dt}",
                   "updates": args.updates, "batch": args.batch, "loss": args.loss, "lr": args.lr,
                   "step_mode": "eager (both arms)"},
        "samples": rows, "sample_gen_s": t_gen, "train_s": t_train,
        "train_loss_first": float(losses[0]), "train_loss_last": float(np.mean(losses[-50:])),
        "train_target_mean_sq": train_var, "heldout_loss": held_loss, "heldout_target_mean_sq": held_var,
        "heldout_r2": 1.0 - held_loss / held_var if held_var > 0 else None,
        "loss_note": ("residual space: mean over samples of ||W d - w||^2 = relative error of the corrected guess "
                      "above the least-squares floor; *_target_mean_sq is that of the plain predictor (d = 0)")
                     if residual else "coefficient space: mean squared error of c* - c",
        "cg_iters_per_case_step": {"plain_dd": it_dd / max(len(log_dd), 1), "learned": it_ml / max(len(log_ml), 1)},
        "proposal_taken_rejected": list(counts),
        "geo_mean_init_relres": {"plain_dd": math.exp(np.mean(log_dd)), "learned": math.exp(np.mean(log_ml))},
    }), flush=True)
    fem.fem_mlp_destroy(net)
    fem.fem_mesh_destroy(h)


def run_uneven(args):
    """Batched uneven cases: --meshes meshes with hex dims Hx, Hy ~ U{24..64}, Hz ~ U{24..48} (h = 1/64,
    three seeded layers), one point source each, FP32-inner / FP64-certified PCG with the data-driven
    predictor; all cases fused into one system (one launch sequence per step) unless --no-fuse."""
    import numpy as np
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    tp = wl.config2_time_params()
    dims = wl.config3_dims(args.meshes)
    handles, n_el, n_nd = [], 0, 0
    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=args.s_max,
                                tol=1e-8, snapshot_format=args.snapshot_format, fuse_meshes=0 if args.no_fuse else 1,
                                cert_df=args.cert, use_graph=0 if args.no_graph else 1, **margin_kw(args))
    bt = fem.fem_batch_create(opts)
    for i, d in enumerate(dims):
        m = wl.config3_mesh(i, d)
        h = fem.fem_mesh_create(m, tp)
        fem.fem_mesh_set_regions(h, wl.region_map(m, args.region_nodes))
        fem.fem_case_add(bt, h, wl.random_source(m, wl.rng_for(3, i, 0, 2)))
        handles.append(h)
        n_el += m.n_elems
        n_nd += m.n_nodes
    nc = len(dims)
    fem.fem_step(bt, args.spinup, nc)
    fem.fem_step(bt, args.warmup, nc)
    sampler = ClockSampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    torch.cuda.synchronize()
    ev0.record(stream)
    st, iters, relres = fem.fem_step(bt, args.steps, nc)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    print(json.dumps({
        "metric": "batched uneven cases: time-steps/s over all cases at rel. residual 1e-8", "unit": UNIT,
        "value": nc * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps, "steps": args.steps,
        "warmup": args.warmup, "spinup_steps": args.spinup, "n_gpus": 1, "higher_is_better": True,
        "config": {"workload": f"{nc} meshes, hex dims U{{24..64}}^2 x U{{24..48}}, h = 1/64, {n_el} tets and "
                               f"{n_nd} nodes in total, one case each, "
                               f"{'fused into one system' if not args.no_fuse else 'one group per mesh'}, "
                               f"FP32-inner/FP64-refined PCG, data-driven predictor s={args.s_max}",
                   "fused": not args.no_fuse, "dims": dims},
        "cg_iters_per_case_step": float(iters.sum()) / (nc * args.steps),
        "max_certified_relres": float(relres.max()), "status": int(st), "clocks": clocks,
    }), flush=True)
    fem.fem_batch_destroy(bt)
    for h in handles:
        fem.fem_mesh_destroy(h)


def run_step10(args):
    """The time-stepping solver on 10-node tets (--element tet10): the --dims box of the medium recipe with
    its tets as quadratic tets (all nodes renumbered in Morton order of their position), --cases cases with
    the recipe's point sources, FP32-inner / FP64-certified block-Jacobi PCG with the tet10 element kernel,
    the data-driven predictor (or AB4) on regions of --region-nodes nodes; graph steps after --spinup steps,
    CUDA events over --steps steps.  The product alone is timed after the steps (FP32, all cases, 10
    launches)."""
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    mesh, tp = make_mesh("medium", args.dims)
    m10, new_id = wl.tet10_mesh_ordered(mesh)
    srcs = make_sources("medium", mesh, args.cases)
    for s in srcs:
        s.node = int(new_id[s.node])
    log(f"tet10 mesh: {m10.n_elems} elements, {m10.n_nodes} nodes")
    h = fem.fem_mesh_create_tet10(m10, tp)
    fem.fem_mesh_tune(h, 8 if args.variant == 8 else 0, 0)   # the element kernel, or the assembled blocks
    fem.fem_mesh_set_regions(h, wl.region_map10(m10, mesh.h, args.region_nodes))
    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER if args.precision == "mixed" else fem.FEM_FP64,
                                predictor=fem.FEM_PRED_DD if args.predictor == "dd" else fem.FEM_PRED_AB4,
                                s_max=args.s_max, tol=1e-8, snapshot_format=args.snapshot_format,
                                cert_df=args.cert, use_graph=0 if args.no_graph else 1, **margin_kw(args))
    bt = fem.fem_batch_create(opts)
    nc = len(srcs)
    for s in srcs:
        fem.fem_case_add(bt, h, s)
    fem.fem_step(bt, args.spinup, nc)
    fem.fem_step(bt, args.warmup, nc)
    sampler = ClockSampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    torch.cuda.synchronize()
    ev0.record(stream)
    st, iters, relres = fem.fem_step(bt, args.steps, nc)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    # per-phase and per-kernel-class device times over --profile-steps eager steps after the timed region
    fem.fem_batch_profile(bt, 1)
    fem.fem_step(bt, max(1, args.profile_steps), nc)
    prof = fem.fem_batch_profile(bt, 0)
    npf = max(prof.get("steps", 1), 1)
    prof_ms = {k: v / npf for k, v in prof.items() if k.endswith("_ms") or k.endswith("_launches")}
    last = [fem.fem_case_stats(bt, c) for c in range(nc)]
    fem.fem_batch_destroy(bt)
    r = nc
    g = torch.Generator(device="cuda").manual_seed(0)
    p = torch.randn(m10.n_nodes * 3 * r, device="cuda", generator=g).float()
    q = torch.empty_like(p)
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    for _ in range(3):
        fem.fem_ebe_apply(h, p, q, r, cM, cK)
    ev0.record(stream)
    for _ in range(10):
        fem.fem_ebe_apply(h, p, q, r, cM, cK)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_prod = ev0.elapsed_time(ev1) / 10
    print(json.dumps({
        "metric": "time-steps/s over all cases at rel. residual 1e-8 (10-node tets)", "unit": UNIT,
        "value": nc * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps, "steps": args.steps,
        "warmup": args.warmup, "spinup_steps": args.spinup, "n_gpus": 1, "higher_is_better": True,
        "config": {"workload": f"{args.dims} hex box of the medium recipe as 10-node tets: {m10.n_elems} elements, "
                               f"{m10.n_nodes} nodes, {nc} cases on one mesh, "
                               f"{'FP32-inner/FP64-refined' if args.precision == 'mixed' else 'FP64'} block-Jacobi "
                               f"EBE-PCG, {'data-driven predictor s=%d' % args.s_max if args.predictor == 'dd' else 'AB4'}",
                   "element": "tet10", "graph": not args.no_graph,
                   "product": "assembled 3x3 blocks" if args.variant == 8 else "tet10 element kernel"},
        "cg_iters_per_case_step": float(iters.sum()) / (nc * args.steps),
        "max_certified_relres": float(relres.max()), "status": int(st), "clocks": clocks,
        "tet10_product_ms": ms_prod, "profile_ms_per_step": prof_ms,
        "last_step": {"iters": [x["iters"] for x in last], "outer": [x["outer"] for x in last],
                      "init_relres": [x["init_relres"] for x in last]},
        "tet10_product_note": "FP32 element kernel, q = A p for all cases, p^T q not fused, incl. zero fill and mask",
    }), flush=True)
    fem.fem_mesh_destroy(h)


def run_mlp(args):
    """Times the learned proposal's network alone (--kernel mlp): Adam updates of batch --batch on the
    residual-space loss, 100 updates a step, and the forward pass over one step's (region, case) rows of the
    medium workload (137 regions x 16 cases).  Random samples, inputs resident; CUDA events.  A dense
    64-256-256-32 network costs 2 x 90112 flops a row forward and 2 x 163840 backward (no input gradient of
    the first layer)."""
    import numpy as np
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    net = fem.fem_mlp_create(wl.mlp_init_weights(0).astype(np.float32))
    g = torch.Generator(device="cuda").manual_seed(0)
    n, upd = 65536, 100
    xs = torch.randn((n, fem.FEM_MLP_IN), device="cuda", generator=g)
    ss = 0.1 * torch.randn((n, fem.FEM_MLP_RES), device="cuda", generator=g)
    order = torch.randint(0, n, (upd, args.batch), device="cuda", generator=g, dtype=torch.int32)
    for _ in range(args.warmup):
        fem.fem_mlp_train_residual(net, xs, ss, order, with_loss=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fem.fem_mlp_train_residual(net, xs, ss, order, with_loss=False)
    e1.record()
    torch.cuda.synchronize()
    ms_upd = e0.elapsed_time(e1) / (args.steps * upd)
    rows = 137 * 16
    out = torch.empty((rows, fem.FEM_MLP_OUT), device="cuda")
    for _ in range(args.warmup):
        fem.fem_mlp_forward(net, xs[:rows], out)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps * 10):
        fem.fem_mlp_forward(net, xs[:rows], out)
    e1.record()
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1) / (args.steps * 10)
    fl_upd = 2.0 * args.batch * (90112 + 163840)
    print(json.dumps({"kernel": "mlp", "batch": args.batch, "ms_per_update": ms_upd,
                      "update_tflops": fl_upd / ms_upd / 1e9, "forward_rows": rows, "ms_per_forward": ms_fwd,
                      "forward_tflops": 2.0 * rows * 90112 / ms_fwd / 1e9,
                      "note": "update = forward, residual-space loss, backward, Adam (BF16 mma.sync GEMMs)"}),
          flush=True)
    fem.fem_mlp_destroy(net)


def run_split(args):
    """Times the certification product alone (fem_mesh_split_product, form --cert) on the --dims mesh with
    --cases cases (CUDA events, inputs resident)."""
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    mesh, tp = make_mesh(args.config, args.dims)
    h = fem.fem_mesh_create(mesh, tp)
    r = args.cases
    g = torch.Generator(device="cuda").manual_seed(0)
    p = torch.randn(mesh.n_nodes * 3 * r, device="cuda", dtype=torch.float64, generator=g)
    qM, qK = torch.empty_like(p), torch.empty_like(p)
    for _ in range(args.warmup):
        fem.fem_mesh_split_product(h, args.cert, p, qM, qK, r)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fem.fem_mesh_split_product(h, args.cert, p, qM, qK, r)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"kernel": "split", "form": args.cert, "dims": args.dims, "cases": r,
                      "ms_per_launch": e0.elapsed_time(e1) / args.steps,
                      "note": "includes the input split to double-float pairs (form 3) and the temporary copy"}),
          flush=True)
    fem.fem_mesh_destroy(h)


def run_predictor_kernels(args):
    """Times the predictor's ring passes alone on the --dims mesh with --cases cases and s = --s-max, after
    --spinup steps fill the snapshot ring: predictor_fit (one Gram row per stored snapshot: s+1 launches of
    the dot kernel) and predictor_predict (Adams-Bashforth, the Gram solves and the combination)."""
    import torch
    from paper_2409_20380_gb300 import build, fem
    from paper_2409_20380_gb300 import workload as wl
    build.build()
    fem.lib()
    torch.cuda.set_device(0)
    mesh, tp = make_mesh(args.config, args.dims)
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_set_regions(h, wl.region_map(mesh, args.region_nodes))
    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=args.s_max,
                                snapshot_format=args.snapshot_format, tol=1e-8, cert_df=args.cert)
    bt = fem.fem_batch_create(opts)
    nc = args.cases
    for c in range(nc):
        fem.fem_case_add(bt, h, wl.random_source(mesh, wl.rng_for(2 if args.config == "medium" else 4, 0, c, 0)))
    fem.fem_step(bt, max(args.spinup, args.s_max + 2), nc)
    guess = torch.empty(mesh.n_nodes * 3, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        fem.predictor_fit(bt, 0)
        fem.predictor_predict(bt, 0, guess)
    torch.cuda.synchronize()
    out = {"kernel": "predictor", "dims": args.dims, "cases": nc, "s_max": args.s_max,
           "snapshot_format": args.snapshot_format}
    for name, fn in (("fit", lambda: fem.predictor_fit(bt, 0)), ("predict", lambda: fem.predictor_predict(bt, 0, guess))):
        t0 = time.perf_counter()
        for _ in range(args.steps):
            fn()
        torch.cuda.synchronize()
        out[name + "_ms"] = (time.perf_counter() - t0) * 1e3 / args.steps
    out["dots_ms_per_row"] = out["fit_ms"] / (args.s_max + 1)
    out["note"] = "host-timed calls (each synchronises); fit = s+1 dot-kernel launches"
    print(json.dumps(out), flush=True)
    fem.fem_batch_destroy(bt)
    fem.fem_mesh_destroy(h)


def main():
    args = parse()
    if args.element == "tet10":
        run_step10(args)
        return
    if args.uneven:
        run_uneven(args)
        return
    if args.learned:
        run_learned(args)
        return
    if args.kernel == "ebe10":
        run_kernel10(args)
        return
    if args.kernel == "pcg10":
        run_pcg10(args)
        return
    if args.kernel == "ebe":
        run_kernel(args)
        return
    if args.kernel == "split":
        run_split(args)
        return
    if args.kernel == "mlp":
        run_mlp(args)
        return
    if args.kernel == "predictor":
        run_predictor_kernels(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
