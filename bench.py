#!/usr/bin/env python
"""Throughput of the layered-grating multi-inclusion solver on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsolve|reference]

Workload (the paper's headline size, M = 1000 inclusions): one period d = 1, three layers with
interfaces y = +-0.5 + 0.05 cos(2 pi x) (N = 256 nodes each), k = (40, 60, 80), plane wave at
theta = -pi/5; 1000 seeded non-overlapping disks of radius 0.008 (gap 0.004), index 2 (kp = 80),
multipole order p = 12 (25 000 unknowns); GMRES to 1e-11; FP64 throughout.

The empty-grating block A depends on the grating and the angle only; it is assembled and factored
(pivoted QR + Jacobi SVD) once, timed and reported separately (`grating_factor_ms`, and
`value_incl_grating_factor` charges it to every step).  One step = one new seeded geometry of 1000
disks through the C-ABI: scattering diagonal S and coupling matrices B, C, right-hand side, GMRES on
the preconditioned Schur system (translation + low-rank correction per iteration), Bragg
amplitudes.  `value` is solves/s of the plain FP64 form over K timed steps (CUDA events, max over
ranks); `variants.mixed_c64_ir` times the complex64-translation + FP64-refinement form the same
way; both are checked against the oracle's stored amplitudes (seed-1 geometry).  `e2e` repeats
the steps through the public API from host inputs (set_inclusions copies the disks from host
memory) to host Bragg amplitudes, wall clock.  N > 1 runs independent replicas, distinct
geometries per rank (weak scaling, no data-path collective).

--impl reference times the oracle (the FP64 CPU restatement under oracle/) on this machine's host
cores on a bounded sample of the same workload, scaled to solves/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/sec at 1e-9 Bragg error: plain FP64 vs mixed/batched/warm-start"
WORKLOAD = ("headline: M=1000 disks r=0.008 gap 0.004 index 2 (kp=80), p=12 (25000 unknowns), "
            "3-layer grating y=+-0.5+0.05cos(2pi x), N=256, k=(40,60,80), theta=-pi/5, "
            "A 1904x1689, GMRES tol 1e-11, FP64")
GOLDEN = os.path.join(ROOT, "tests", "golden", "headline_bragg.txt")
# measured HBM copy bandwidth and bf16 GEMM throughput of this machine's GPUs; the recipe's fallback
# (one earlier GB300 measurement) when the file is absent
try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        PEAKS = dict(json.load(_f), source="measured")
except (OSError, ValueError):
    PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}
# DRAM bytes per (target, source image) pair of the table-driven FP64 translation, from the ncu
# capture of k_translate_f64_tab at M = 500 (599.58 MB over 3 * 500^2 - 500 pairs); the pair table
# (49 complex128 per pair) is 784 B of it.  Update with a new capture whenever that kernel changes.
TAB_DRAM_BYTES_PER_PAIR = 599.577344e6 / (3 * 500 ** 2 - 500)
# complex64 pair table: 4p + 1 = 49 complex64 coefficients per pair image (p = 12)
TAB32_BYTES_PER_PAIR = 49 * 8


def load_golden(path=GOLDEN):
    """{(side, order): amplitude} of a stored oracle solution (tests/golden)."""
    ref = {}
    for ln in open(path):
        if not ln.startswith("#"):
            s_, n_, re_, im_ = ln.split()
            ref[(s_, int(n_))] = complex(float(re_), float(im_))
    return ref


def bragg_errors(br, path=GOLDEN):
    """(norm-wise, element-wise maximum) relative errors of Bragg amplitudes against a stored oracle
    solution over the propagating orders; (None, None) if the orders differ."""
    import numpy as np
    ref = load_golden(path)
    got = {("c", int(n)): v for n, v in zip(br["n_top"], br["c"])}
    got.update({("d", int(n)): v for n, v in zip(br["n_bot"], br["d"])})
    if set(got) != set(ref):
        return None, None
    keys = sorted(ref)
    a = np.array([got[k] for k in keys])
    b = np.array([ref[k] for k in keys])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b)), float(np.max(np.abs(a - b) / np.abs(b)))


def geometry_seeds(rank: int, n_geo: int) -> list:
    """Seeds of the geometries rank `rank` solves: distinct across ranks (replicas do independent
    work; nothing is exchanged on the data path)."""
    return [1000 * (rank + 1) + s for s in range(n_geo)]


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """The job's time for a quantity every rank measured: the maximum over the ranks."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, elapsed_max: float) -> float:
    """Whole-job solves/s: every rank solves `steps` geometries; the job ends with the slowest."""
    return world * steps / elapsed_max


def run_study(device: int) -> dict:
    """Disk analogues of the paper's experiments (Sec. 6).  Example 1: homogeneous background
    k = (10, 10, 10) against layered k = (10, 8, 10), M = 100, 500, 1000 disks with k_p = 30, p = 10,
    theta = -arccos(1 - 2 pi / 10) + 0.1 (near a Wood anomaly, not on it).  Example 3: M = 100 disks
    (some crossing the walls), k1 = k3 = 5, k_p = 8, k2 = 1, 10, 20, 30.  FP64 GMRES to 1e-11 (restart
    500), time per solve (device events) and the flux error; the grating factorisation per
    configuration is reported separately."""
    import torch
    import workloads as W
    from paper_1412_7466_gb300 import GratingSolver

    def one(g, theta, dk):
        gs = GratingSolver(device)
        gs.set_layers(g)
        gs.set_incidence([theta])
        gs.set_inclusions(dk)
        st = torch.cuda.current_stream()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(st)
        gs.factor()
        e[1].record(st)
        gs.solve(tol=1e-11, maxit=4000, restart=500)
        br = gs.bragg()
        e[2].record(st)
        torch.cuda.synchronize()
        its, rr = gs.stats()
        gs.close()
        return {"iters": its, "relres": rr, "flux_err": br["flux_err"], "factor_ms": e[0].elapsed_time(e[1]),
                "solve_ms": e[1].elapsed_time(e[2])}

    base = W.grating("small")
    theta1 = -math.acos(1.0 - 2.0 * math.pi / 10.0) + 0.1
    ex1 = []
    for M, r in ((100, 0.025), (500, 0.012), (1000, 0.008)):
        for name, k in (("homogeneous", (10.0, 10.0, 10.0)), ("layered", (10.0, 8.0, 10.0))):
            g = dict(base)
            g["k"] = k
            dk = W.disks(M, r, r / 2, 3.0, 10.0, seed=M, p=10)    # k_p = 30 = 3 k1
            ex1.append(dict(one(g, theta1, dk), M=M, r=r, background=name, k=list(k)))
    ex3 = []
    dk3 = W.disks(100, 0.025, 0.0125, 1.6, 5.0, seed=3, p=10)     # k_p = 8 = 1.6 k1
    for k2 in (1.0, 10.0, 20.0, 30.0):
        g = dict(base)
        g["k"] = (5.0, k2, 5.0)
        ex3.append(dict(one(g, -math.pi / 5, dk3), k2=k2))
    return {"study": "paper experiment analogues with disks", "example1": ex1, "example3": ex3,
            "paper_example1": "no obvious difference in iterations between homogeneous and layered",
            "paper_table3_iters": {"1": 13, "10": 15, "20": 43, "30": 83}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsolve", choices=["gsolve", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-complete", action="store_true",
                    help="also time one complete oracle solve of the headline workload (minutes of CPU)")
    ap.add_argument("--oracle-small-once", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-warm", action="store_true")
    ap.add_argument("--warm-train", type=int, default=24, help="warm start: training sweep points")
    ap.add_argument("--warm-eval", type=int, default=6, help="warm start: held-out sweep points")
    ap.add_argument("--warm-geometry", choices=["headline", "mixed4000"], default="headline",
                    help="warm start: the swept geometry (mixed4000: M = 4000 disks of radius 0.004; its "
                         "held-out points are then solved in the mixed form, FP64 GMRES taking ~40 s each)")
    ap.add_argument("--no-big", action="store_true")
    ap.add_argument("--no-tc", action="store_true")
    ap.add_argument("--no-field", action="store_true")
    ap.add_argument("--no-angles", action="store_true")
    ap.add_argument("--angles", type=int, default=16,
                    help="multi-angle variant: incidence angles of the headline geometry solved in lockstep")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--one-solve", choices=["fp64", "c64"], default=None,
                    help="profiler capture: one warm-up solve of the headline workload, then one solve "
                         "bracketed by cudaProfilerStart/Stop (ncu --profile-from-start off)")
    ap.add_argument("--study", action="store_true",
                    help="disk analogues of the paper's Example 1 (homogeneous vs layered, M = 100/500/1000) "
                         "and Example 3 (k2 = 1, 10, 20, 30): GMRES iterations, time, flux; one JSON line")
    ap.add_argument("--kernel-only", action="store_true",
                    help="factor once, then run warmup + steps calls of one kernel family only, for ncu "
                         "captures: GS_BENCH_PRECISION = fp64 (translation, default), c64 (complex64 "
                         "translation), c64op (the mixed solve's inner operator), batch, tc; GS_BENCH_M "
                         "sets a smaller M")
    return ap.parse_args()


# ---- clocks -----------------------------------------------------------------------------------

CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), float(p[3]), p[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "reasons": reasons, "samples": len(rows)}


# ---- oracle timings (CPU baseline / reference arm) ------------------------------------------------

ORACLE_SLICES = 20   # the reference arm's step is one twentieth of a headline solve's per-geometry work


def oracle_iterations():
    with open(GOLDEN) as f:
        head = f.readline()
    return int(head.split("GMRES its")[1].split(",")[0])


def oracle_small_complete(seed=1):
    """Seconds of one complete oracle solve of the 10-disk workload (M = 10, p = 10, k = (10, 15,
    20)): assembly of A, LAPACK SVD, S, B_phys, C, the dense preconditioned Schur matrix and its LU
    solve, Bragg amplitudes."""
    import workloads as W
    from oracle import solver as S
    cfg = W.config("small", seed=seed)
    t0 = time.perf_counter()
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    beta, _, _ = S.solve_dense(prob)
    prob.recover(beta)
    return time.perf_counter() - t0


def oracle_small_one_core():
    """The complete small solve in a fresh interpreter limited to one thread (BLAS and OpenMP)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-small-once"], env=env,
                       capture_output=True, text=True, timeout=600)
    try:
        return float(r.stdout.strip().splitlines()[-1])
    except (ValueError, IndexError):
        return None


class OracleHeadline:
    """The oracle on the headline workload, in slices of its per-geometry work.

    The GPU step (a new geometry on the factored grating) is coupling + rhs + GMRES + Bragg; for
    the oracle that is B_phys and C for the 1000 disks (per-disk loops) and ~its + 2 operator
    applications (C direct-sum translation over all pairs and images, plus the low-rank GEMVs with
    B_phys, U^*, V, C).  One slice = B_phys and C for 50 of the disks plus (its + 2) / 20 operator
    applications, so a complete solve is 20 slices.  The applications use a factorisation of the
    right shapes (U = the column-scaled A, V = I, zero B_phys and C: the dense GEMVs cost the same
    for any values) so that building the real B_phys and C of all 1000 disks is not needed first;
    the GMRES orthogonalisation (~1 % of the oracle's solve) is left out.  The grating's assembly
    and SVD are timed once, like the GPU's grating factorisation."""

    def __init__(self, cfg):
        import numpy as np
        from oracle import inclusions as I
        from oracle import layers as L
        from oracle import solver as S
        self.I, self.np = I, np
        g, theta, dk = cfg["grating"], cfg["theta"], cfg["disks"]
        self.dk = dk
        t0 = time.perf_counter()
        self.eg = L.build_empty_grating(g, theta)
        t1 = time.perf_counter()
        D = L.jcolumn_scale(self.eg)
        As = self.eg.A * D[None, :]
        np.linalg.svd(As, full_matrices=False)
        t2 = time.perf_counter()
        self.t_assemble, self.t_svd = t1 - t0, t2 - t1
        M, nc = dk["xy"].shape[0], 2 * dk["p"] + 1
        pinv = L.PInv(U=As, s=np.ones(As.shape[1]), Vh=np.eye(As.shape[1], dtype=complex), colscale=D,
                      eps=g["eps_pinv"])
        self.prob = S.Problem(eg=self.eg, pinv=pinv, disks=dk, s=I.scattering_diagonal(dk, g["k"][1]),
                              B=np.zeros((M * nc, As.shape[1]), dtype=complex),
                              C=np.zeros((As.shape[0], M * nc), dtype=complex), timings={})
        self.x = np.random.default_rng(0).standard_normal(M * nc) + 0j
        self.n_apply = oracle_iterations() + 2
        self.per = M // ORACLE_SLICES

    def slice(self, q):
        """Seconds of slice q: B_phys and C for disks [50 k, 50 k + 50), k = q mod 20, and that
        slice's share of the operator applications (the 20 shares add up to all of them)."""
        np = self.np
        k = q % ORACLE_SLICES
        lo = k * self.per
        sub = {key: (v[lo:lo + self.per] if isinstance(v, np.ndarray) else v) for key, v in self.dk.items()}
        napp = self.n_apply * (k + 1) // ORACLE_SLICES - self.n_apply * k // ORACLE_SLICES
        t0 = time.perf_counter()
        self.I.coupling_B(self.eg, sub)
        self.I.coupling_C(self.eg, sub)
        for _ in range(napp):
            self.prob.apply(self.x)
        return time.perf_counter() - t0

    def describe(self, t_slice):
        return (f"oracle (numpy/scipy FP64 + C/OpenMP direct-sum translation) on the headline workload, "
                f"timed in slices of one solve's per-geometry work: one slice = B_phys and C for 50 of the "
                f"1000 disks + {self.n_apply}/20 full-size operator applications ({self.n_apply} = the "
                f"oracle's own GMRES iterations + 2); 20 slices = one solve; {t_slice:.2f} s per slice; "
                f"grating assembly {self.t_assemble:.1f} s and SVD {self.t_svd:.1f} s timed once, outside "
                f"the solve (as on the GPU)")


def oracle_headline_complete(cfg):
    """Seconds of one complete oracle solve of the headline workload: assembly, SVD, S, B_phys, C,
    matrix-free GMRES(200) to the workload's tolerance, Bragg amplitudes."""
    from oracle import solver as S
    t0 = time.perf_counter()
    prob = S.setup(cfg["grating"], cfg["theta"], cfg["disks"])
    t1 = time.perf_counter()
    beta, its, hist, _ = S.solve_gmres(prob, tol=cfg["tol"], restart=200, maxit=3000)
    prob.recover(beta)
    t2 = time.perf_counter()
    return {"seconds": t2 - t0, "setup_s": t1 - t0, "gmres_s": t2 - t1, "gmres_iters": its,
            "factor_s": prob.timings["factor"], "assemble_s": prob.timings["assemble"],
            "couple_s": prob.timings["couple"]}


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ---- main -----------------------------------------------------------------------------------------

def main():
    args = parse()
    if args.oracle_small_once:
        print(oracle_small_complete())
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import workloads as W

    if args.impl == "reference":
        if rank != 0:
            return
        cfg = W.config("headline", seed=1)
        from oracle import m2l
        m2l.build()
        oh = OracleHeadline(cfg)
        for s_ in range(args.warmup):
            oh.slice(s_)
        ts = [oh.slice(args.warmup + s_) for s_ in range(args.steps)]
        t_slice = statistics.mean(ts)
        v = 1.0 / (ORACLE_SLICES * t_slice)        # one slice = 1/20 of a solve
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_slice, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD, "step": "one twentieth of a solve's per-geometry work (see sample)"},
               "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores(), "kind": "oracle",
                                "sample": oh.describe(t_slice)},
               "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    import numpy as np
    import torch
    from paper_1412_7466_gb300 import GS_C64, GS_FP64, GS_MIXED_BF16, GS_PROBE_F32X2, GS_TC_BF16, GratingSolver

    if args.study:
        if rank == 0:
            print(json.dumps(run_study(local)))
        return

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    cfg0 = W.config("headline", seed=1)
    if args.one_solve:
        prec = GS_C64 if args.one_solve == "c64" else GS_FP64
        gs = GratingSolver(local)
        gs.set_layers(cfg0["grating"])
        gs.set_incidence([cfg0["theta"]])
        gs.set_inclusions(cfg0["disks"])
        gs.factor()
        gs.solve(tol=cfg0["tol"], maxit=4000, restart=500, precision=prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        t0 = time.perf_counter()
        gs.solve(tol=cfg0["tol"], maxit=4000, restart=500, precision=prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        torch.cuda.profiler.stop()
        its, rr = gs.stats()
        print(json.dumps({"one_solve": args.one_solve, "workload": WORKLOAD, "solve_ms": 1e3 * (t1 - t0),
                          "iterations": its, "relres": rr, "refinement_sweeps": gs.refinement_sweeps(0)}))
        gs.close()
        return
    if args.kernel_only and os.environ.get("GS_BENCH_M"):
        # smaller case of the same kernel for profiler captures (same grating, disk size and order)
        cfg0["disks"] = W.disks(int(os.environ["GS_BENCH_M"]), 0.008, 0.004, 2.0, cfg0["grating"]["k"][0],
                                seed=1, p=12)
    g, theta, tol = cfg0["grating"], cfg0["theta"], cfg0["tol"]
    gs = GratingSolver(local)
    gs.set_layers(g)
    gs.set_incidence([theta])
    gs.set_inclusions(cfg0["disks"])
    M, p = cfg0["disks"]["xy"].shape[0], cfg0["disks"]["p"]
    nc = 2 * p + 1
    stream = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # per-angle factorisation of the empty grating (assemble A, pivoted QR + Jacobi SVD): once
    e = [ev() for _ in range(3)]
    e[0].record(stream)
    gs.factor()                       # grating + coupling of the first geometry
    e[1].record(stream)
    gs.factor()                       # coupling only (grating factorisation kept)
    e[2].record(stream)
    torch.cuda.synchronize()
    couple_ms = e[1].elapsed_time(e[2])
    grating_ms = e[0].elapsed_time(e[1]) - couple_ms
    factor_stats = gs.factor_stats(0)

    if args.kernel_only and os.environ.get("GS_BENCH_PRECISION") == "batch":
        # batched complex64 translation: the bench's eight uneven-M geometries at the Wood angle
        bgeos = [gg for gg in W.batched_geometries(n_geom=64, seed=4) if gg["xy"].shape[0] <= 1200][:8]
        gb = GratingSolver(local)
        gb.set_layers(g)
        gb.set_incidence([W.wood_angle(g["k"][0], g["d"])])
        gb.set_inclusions_batch(bgeos)
        gb.factor_batch()
        xb = torch.randn(sum(gb.batch_sizes), dtype=torch.complex128, device="cuda")
        for _ in range(args.warmup + args.steps):
            gb.apply_batch(xb, precision=GS_C64)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": True, "batched_applies": args.warmup + args.steps,
                          "geometries_M": [int(x["xy"].shape[0]) for x in bgeos]}))
        gb.close()
        gs.close()
        return

    if args.kernel_only and os.environ.get("GS_BENCH_PRECISION") == "tc":
        # tensor-core multi-right-hand-side translation, R = 256 angles
        R = 256
        ths = W.batched_angles(k1=g["k"][0], n=R)
        alphas = np.exp(1j * g["k"][0] * np.cos(ths) * g["d"])
        betas = torch.randn(R, M * nc, dtype=torch.complex128, device="cuda")
        for _ in range(args.warmup + args.steps):
            gs.translate_multi(alphas, betas)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": True, "translate_multi_launches": args.warmup + args.steps, "R": R}))
        gs.close()
        return

    if args.kernel_only and os.environ.get("GS_BENCH_PRECISION") == "c64op":
        # the mixed solve's inner operator (complex64 translation, double-float C x, complex64 B)
        x = torch.randn(M * nc, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        for _ in range(args.warmup + args.steps):
            gs.apply(x, precision=GS_C64, out=y)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": True, "c64_operator_applies": args.warmup + args.steps}))
        gs.close()
        return

    if args.kernel_only:
        beta = torch.randn(M * nc, dtype=torch.complex128, device="cuda")
        out = torch.empty_like(beta)
        prec = GS_C64 if os.environ.get("GS_BENCH_PRECISION", "fp64") == "c64" else GS_FP64
        for _ in range(args.warmup + args.steps):
            gs.translate(beta, out=out, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": True, "translate_launches": args.warmup + args.steps, "precision": prec}))
        gs.close()
        return

    # seeded geometries, one per step (distinct per rank); host arrays prepared before timing
    n_geo = args.warmup + args.steps
    geos = [W.config("headline", seed=sd)["disks"] for sd in geometry_seeds(rank, n_geo)]

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def run(precision, gather_profile):
        """K timed steps (after W warm-up steps), each a new geometry: coupling, solve, Bragg.
        Device time summed over steps with CUDA events; set_inclusions (host->device copy of the
        disk arrays, 32 KB) happens between the events."""
        for s in range(args.warmup):
            gs.set_inclusions(geos[s])
            gs.factor()
            gs.solve(tol=tol, maxit=4000, restart=500, precision=precision)
            gs.bragg()
        barrier()
        if gather_profile:
            gs.profile(True)
        l0 = gs.launch_count()
        tot = 0.0
        its = []
        with ClockSampler(local) as clk:
            for s in range(args.warmup, n_geo):
                gs.set_inclusions(geos[s])
                a, b = ev(), ev()
                a.record(stream)
                gs.factor()
                gs.solve(tol=tol, maxit=4000, restart=500, precision=precision)
                br = gs.bragg()
                b.record(stream)
                b.synchronize()
                tot += a.elapsed_time(b) / 1e3
                its.append(gs.stats()[0])
        l1 = gs.launch_count()
        prof = {}
        if gather_profile:
            prof = {"fp64": gs.profile_read(GS_FP64), "c64": gs.profile_read(GS_C64)}
            gs.profile(False)
        tot = max_over_ranks(tot, dist, "cuda")
        return {"elapsed": tot, "launches": int(l1 - l0), "iters": its, "clocks": clk.summary(), "prof": prof}

    def e2e(precision):
        barrier()
        t0 = time.perf_counter()
        for s in range(args.warmup, n_geo):
            gs.set_inclusions(geos[s])
            gs.factor()
            gs.solve(tol=tol, maxit=4000, restart=500, precision=precision)
            br = gs.bragg()
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        return el, br

    def golden_error(precision):
        """Bragg amplitudes of the seed-1 geometry against the oracle's stored values: (norm-wise,
        element-wise) relative errors, or (None, None) if the propagating orders differ."""
        gs.set_inclusions(cfg0["disks"])
        gs.factor()
        gs.solve(tol=tol, maxit=4000, restart=500, precision=precision)
        br = gs.bragg()
        return bragg_errors(br), br

    res = {}
    for name, prec in (("fp64", GS_FP64), ("mixed_c64_ir", GS_C64)):
        r = run(prec, gather_profile=True)
        el_e2e, br = e2e(prec)
        (err, err_el), brg = golden_error(prec)
        res[name] = {"r": r, "e2e": el_e2e, "err": err, "err_el": err_el, "flux": brg["flux_err"],
                     "outer": gs.refinement_sweeps(), "n_cd": len(br["c"]) + len(br["d"])}
    # pre-refinement error of the mixed form: one complex64 inner solve from zero, no FP64 correction
    pre_err = None
    try:
        gs.set_inclusions(cfg0["disks"])
        gs.factor()
        gs.solve(tol=tol, maxit=4000, restart=500, precision=GS_C64, allow_unconverged=True, max_sweeps=1)
        pre_err = bragg_errors(gs.bragg())[0]
    except Exception:
        pass

    # tensor-core multi-right-hand-side translation: the headline geometry at R = 256 incidence
    # angles (the batched workload's angle list) in one product, bfloat16 operands, FP32 accumulation
    tcres = None
    if not args.no_tc:
        gs.set_inclusions(cfg0["disks"])
        gs.factor()
        R = 256
        ths = W.batched_angles(k1=g["k"][0], n=R)
        alphas = np.exp(1j * g["k"][0] * np.cos(ths) * g["d"])
        rngt = np.random.default_rng(12)
        wt = np.tile(0.3 ** np.abs(np.arange(-p, p + 1)), M)
        betas = torch.from_numpy((rngt.standard_normal((R, M * nc)) + 1j * rngt.standard_normal((R, M * nc))) * wt
                                 ).to("cuda")
        a_, b_ = ev(), ev()
        a_.record(stream)
        out_tc = gs.translate_multi(alphas, betas)   # first call builds the operator
        b_.record(stream)
        torch.cuda.synchronize()
        first_ms = a_.elapsed_time(b_)
        for _ in range(2):
            gs.translate_multi(alphas, betas)
        n_tc = 5
        gs.profile(True)
        a_, b_ = ev(), ev()
        a_.record(stream)
        for _ in range(n_tc):
            out_tc = gs.translate_multi(alphas, betas)
        b_.record(stream)
        torch.cuda.synchronize()
        call_ms = a_.elapsed_time(b_) / n_tc
        ntc, ms_tc = gs.profile_read(GS_TC_BF16)
        gs.profile(False)
        gemm_ms = ms_tc / max(ntc, 1)
        errs = []
        for r in (0, R // 2, R - 1):
            gs.set_incidence([float(ths[r])])
            gs.factor()
            ref = gs.translate(betas[r])
            errs.append(float(torch.linalg.norm(out_tc[r] - ref) / torch.linalg.norm(ref)))
        gs.set_incidence([theta])
        flops_alg = 8.0 * nc * nc * (3.0 * M * M - M) * R
        rows, cols = 2 * M * nc, 6 * M * nc
        rows_p, cols_p = -(-rows // 128) * 128, -(-cols // 64) * 64
        a_bytes = 2.0 * rows_p * cols_p
        tcres = {"R": R, "unit": "pair-translations/s",
                 "value": (3 * M * M - M) * R / (call_ms * 1e-3),
                 "call_ms": call_ms, "gemm_ms": gemm_ms, "first_call_ms_incl_operator_build": first_ms,
                 "rel_err_vs_fp64_translate": errs,
                 "roofline": {"bound": "hbm", "kernel": "k_tc_gemm (tcgen05, bf16 in, fp32 accumulate)",
                              "achieved": a_bytes / (gemm_ms * 1e-3) / 1e9, "peak": PEAKS.get("hbm_gbs"),
                              "unit": "GB/s", "frac": a_bytes / (gemm_ms * 1e-3) / 1e9 / PEAKS.get("hbm_gbs", 1.0),
                              "peak_source": PEAKS["source"] + " copy bandwidth",
                              "traffic": None, "bytes_per_launch": a_bytes},
                 "tensor": {"achieved_tflops_algorithmic": flops_alg / (gemm_ms * 1e-3) / 1e12,
                            "achieved_tflops_issued": 2.0 * rows_p * cols_p * R / (gemm_ms * 1e-3) / 1e12,
                            "peak": PEAKS.get("bf16_tflops"),
                            "peak_source": PEAKS["source"] + " cuBLAS bf16 burst"},
                 "operator_gb": a_bytes / 1e9,
                 "note": "operator [T_-1 T_0 T_1] in real 2x2 form, bfloat16, built once per geometry; "
                         "the product streams it once for all R right-hand sides"}

    # field plot of the headline solution: the total field on a 512 x 256 grid of the middle layer
    fres = None
    if not args.no_field:
        gs.set_inclusions(cfg0["disks"])
        gs.factor()
        gs.solve(tol=tol, maxit=4000, restart=500)
        xs, ys = np.meshgrid(np.linspace(-0.5, 0.5, 512), np.linspace(-1.2, 1.2, 512))
        pts = torch.from_numpy(np.stack([xs.ravel(), ys.ravel()], axis=1)).to("cuda")
        gs.field(pts)
        a_, b_ = ev(), ev()
        a_.record(stream)
        uf = gs.field(pts)
        b_.record(stream)
        torch.cuda.synchronize()
        fms = a_.elapsed_time(b_)
        fres = {"points": int(pts.shape[0]), "ms": fms, "unit": "points/s", "value": pts.shape[0] / (fms * 1e-3),
                "nan_points": int(torch.isnan(uf.real).sum().item()),
                "max_abs": float(torch.nan_to_num(uf.abs(), nan=0.0).max().item()),
                "grid": "512 x 512 over one period, y in [-1.2, 1.2]: all three layers and the Rayleigh-Bloch "
                        "regions beyond +-y0",
                "per_point": "middle layer: 2 interfaces x 3 copies x N = 256 nodes, a 181-term J-expansion, "
                             "3000 inclusion images x (2p+1) orders; top/bottom: 1 interface x 3 copies x 256 "
                             "nodes and a 181-term J-expansion; beyond +-y0: 61 Rayleigh-Bloch orders (FP64)"}

    # the mixed-precision workload at its own size: M = 4000 disks of radius 0.004 on the same
    # grating and angle (100 000 unknowns); one warm-up geometry, one timed geometry
    bigres = None
    if not args.no_big:
        gbig = [W.config("mixed4000", seed=sd)["disks"] for sd in (1, 2)]
        gs.set_inclusions(gbig[0])
        gs.factor()
        gs.solve(tol=tol, maxit=8000, restart=500, precision=GS_C64)
        gs.bragg()
        barrier()
        gs.set_inclusions(gbig[1])
        a_, b_ = ev(), ev()
        a_.record(stream)
        gs.factor()
        gs.solve(tol=tol, maxit=8000, restart=500, precision=GS_C64)
        brb = gs.bragg()
        b_.record(stream)
        b_.synchronize()
        tb = a_.elapsed_time(b_) / 1e3
        bigres = {"value": 1.0 / tb, "unit": "solves/s", "dtype": "c64 translation + f64 refinement",
                  "M": 4000, "unknowns": 4000 * nc, "inner_iters": gs.stats()[0],
                  "refinement_sweeps": gs.refinement_sweeps(), "relres": gs.stats()[1],
                  "flux_err": brb["flux_err"],
                  "step": "set_inclusions + factor (S, B, C, pair table) + mixed solve to 1e-11 + Bragg; "
                          "Bragg agreement with the FP64 solve at this size: tests/test_gpu_mixed4000.py"}

    # batched form: geometries of uneven size from the batched workload generator, one grating
    # factorisation at the k1 = 40 Wood-anomaly angle, solved together (one persistent translation
    # per product, lockstep GMRES from a CUDA graph) against the same geometries one at a time
    bres = None
    if not args.no_batch:
        bgeos = [gg for gg in W.batched_geometries(n_geom=64, seed=4) if gg["xy"].shape[0] <= 1200][:8]
        theta_w = W.wood_angle(g["k"][0], g["d"])
        gb = GratingSolver(local)
        gb.set_layers(g)
        gb.set_incidence([theta_w])
        gb.set_inclusions(bgeos[0])
        gb.factor()                                   # grating factorisation at the Wood angle, once

        def batched_step():
            gb.set_inclusions_batch(bgeos)
            gb.factor_batch()
            gb.solve_batch(tol=tol, maxit=4000, restart=500, precision=GS_C64)
            return [gb.bragg_batch(q) for q in range(len(bgeos))]

        def sequential_step():
            out_ = []
            for dk in bgeos:
                gb.set_inclusions(dk)
                gb.factor()
                gb.solve(tol=tol, maxit=4000, restart=500, precision=GS_C64)
                out_.append(gb.bragg())
            return out_

        timings = {}
        for name, fn in (("batched", batched_step), ("sequential", sequential_step)):
            fn()
            barrier()
            a_, b_ = ev(), ev()
            a_.record(stream)
            for _ in range(args.steps):
                brs = fn()
            b_.record(stream)
            torch.cuda.synchronize()
            timings[name] = a_.elapsed_time(b_) / 1e3
            if name == "batched":
                bat_brs = brs
                b_iters = [gb.batch_stats(q)[0] for q in range(len(bgeos))]
            else:
                seq_brs = brs
        diff = max(float(np.linalg.norm(np.r_[x["c"], x["d"]] - np.r_[y["c"], y["d"]]) /
                         np.linalg.norm(np.r_[y["c"], y["d"]])) for x, y in zip(bat_brs, seq_brs))
        nG = len(bgeos)
        bres = {"value": nG * args.steps / timings["batched"], "unit": "solves/s",
                "dtype": "c64 translation + f64 refinement",
                "sequential_value": nG * args.steps / timings["sequential"],
                "geometries_M": [int(gg["xy"].shape[0]) for gg in bgeos],
                "pair_images_per_product": int(sum(3 * gg["xy"].shape[0] ** 2 for gg in bgeos)),
                "theta": theta_w, "inner_iters": b_iters, "tuning": list(gb.batch_tuning()),
                "max_bragg_rel_diff_batched_vs_sequential": diff,
                "max_flux_err": max(x["flux_err"] for x in bat_brs),
                "step": "set_inclusions_batch + factor_batch (S, B, C of every geometry, autotune) + "
                        "solve_batch + Bragg of every geometry; grating factorised once at the Wood angle"}
        gb.close()

    # many incidence angles of one geometry (the batched workload's angle list, every 256/R-th
    # angle, with the k1 = 40 Wood angle): all R in lockstep (three-part bf16 tensor-core inner translation,
    # per-angle low rank, FP64 refinement) against the same R angles solved one by one in the mixed
    # form on the same factored context
    angres = None
    if not args.no_angles and args.angles > 0:
        R = args.angles
        allth = W.batched_angles(k1=g["k"][0], n=256)
        th_w = W.wood_angle(g["k"][0], g["d"])
        idx = sorted(set(np.linspace(0, 255, R).round().astype(int).tolist()))
        ths = [float(allth[i]) for i in idx]
        if not any(abs(t - th_w) < 1e-12 for t in ths):
            ths[len(ths) // 2] = th_w
        ga = GratingSolver(local)
        ga.set_layers(g)
        ga.set_incidence(ths)
        ga.set_inclusions(cfg0["disks"])
        a_, b_ = ev(), ev()
        a_.record(stream)
        ga.factor()
        b_.record(stream)
        torch.cuda.synchronize()
        fac_ms = a_.elapsed_time(b_)
        ga.solve_angles(tol=tol, maxit=8000, restart=500, precision=GS_MIXED_BF16)   # warm-up (operators, graph)
        barrier()
        l0 = ga.launch_count()
        a_, b_ = ev(), ev()
        a_.record(stream)
        ga.solve_angles(tol=tol, maxit=8000, restart=500, precision=GS_MIXED_BF16)
        brs_l = [ga.bragg(angle=q) for q in range(len(ths))]
        b_.record(stream)
        torch.cuda.synchronize()
        t_lock = a_.elapsed_time(b_) / 1e3
        launches_l = ga.launch_count() - l0
        st_l = [ga.stats(angle=q) for q in range(len(ths))]
        sw_l = [ga.refinement_sweeps(q) for q in range(len(ths))]
        a_, b_ = ev(), ev()
        a_.record(stream)
        brs_s = []
        for q in range(len(ths)):
            ga.solve(angle=q, tol=tol, maxit=8000, restart=500, precision=GS_C64)
            brs_s.append(ga.bragg(angle=q))
        b_.record(stream)
        torch.cuda.synchronize()
        t_seq = a_.elapsed_time(b_) / 1e3
        its_s = [ga.stats(angle=q)[0] for q in range(len(ths))]
        # the same lockstep with each angle translated from the complex64 table
        ga.solve_angles(tol=tol, maxit=8000, restart=500, precision=GS_C64)   # warm-up (its graph)
        a_, b_ = ev(), ev()
        a_.record(stream)
        ga.solve_angles(tol=tol, maxit=8000, restart=500, precision=GS_C64)
        brs_t = [ga.bragg(angle=q) for q in range(len(ths))]
        b_.record(stream)
        torch.cuda.synchronize()
        t_tab = a_.elapsed_time(b_) / 1e3
        its_t = [ga.stats(angle=q)[0] for q in range(len(ths))]
        sw_t = [ga.refinement_sweeps(q) for q in range(len(ths))]
        diff = max(float(np.linalg.norm(np.r_[x["c"], x["d"]] - np.r_[y["c"], y["d"]]) /
                         np.linalg.norm(np.r_[y["c"], y["d"]])) for x, y in zip(brs_l + brs_t, brs_s + brs_s))
        ga.close()
        angres = {"value": len(ths) / t_tab, "unit": "solves/s",
                  "dtype": "c64 translation (complex64 table, per angle) + f64 refinement, angles in lockstep",
                  "R": len(ths), "sequential_mixed_value": len(ths) / t_seq,
                  "inner_iters_c64": its_t, "refinement_sweeps_c64": sw_t,
                  "tensor_core_lockstep_value": len(ths) / t_lock,
                  "tensor_core_dtype": "three-part bf16 tensor-core translation of all angles + f64 refinement",
                  "thetas": ths, "wood_angle": th_w, "grating_factor_ms_all_angles": fac_ms,
                  "inner_iters_tensor_core": [x[0] for x in st_l], "refinement_sweeps_tensor_core": sw_l,
                  "relres_tensor_core": [x[1] for x in st_l], "sequential_inner_iters": its_s,
                  "max_bragg_rel_diff_lockstep_vs_sequential": diff,
                  "max_flux_err": max(x["flux_err"] for x in brs_l + brs_t),
                  "gpu_launches_tensor_core": int(launches_l),
                  "step": "solve_angles (all R angles: rhs, lockstep inner GMRES, FP64 residuals per angle) + Bragg "
                          "of every angle, timed for each inner translation, and the same R angles solved one by one "
                          "(solve, GS_C64); the R grating factorisations and the coupling are outside the timed "
                          "region (grating_factor_ms_all_angles)"}

    # the 10-disk workload (M = 10, p = 10, k = (10, 15, 20), 128 nodes per interface, tol 1e-12):
    # latency-bound; one new seeded geometry per step on the factored grating, against the oracle's
    # complete solve of the same workload on the host (cpu_baseline.complete_solve_small)
    smallres = None
    if not args.no_small:
        cs = W.config("small", seed=1)
        gsm = GratingSolver(local)
        gsm.set_layers(cs["grating"])
        gsm.set_incidence([cs["theta"]])
        gsm.set_inclusions(cs["disks"])
        a_, b_ = ev(), ev()
        a_.record(stream)
        gsm.factor()
        b_.record(stream)
        torch.cuda.synchronize()
        fac_small = a_.elapsed_time(b_)
        sgeos = [W.config("small", seed=100 + s_)["disks"] for s_ in range(args.warmup + args.steps)]
        for s_ in range(args.warmup):
            gsm.set_inclusions(sgeos[s_])
            gsm.factor()
            gsm.solve(tol=cs["tol"], maxit=500)
            gsm.bragg()
        barrier()
        a_, b_ = ev(), ev()
        a_.record(stream)
        for s_ in range(args.warmup, args.warmup + args.steps):
            gsm.set_inclusions(sgeos[s_])
            gsm.factor()
            gsm.solve(tol=cs["tol"], maxit=500)
            brsm = gsm.bragg()
        b_.record(stream)
        torch.cuda.synchronize()
        t_small = a_.elapsed_time(b_) / 1e3
        its_small = gsm.stats()[0]
        gsm.close()
        smallres = {"value": args.steps / t_small, "unit": "solves/s", "dtype": "f64",
                    "ms_per_solve": 1e3 * t_small / args.steps, "grating_factor_ms": fac_small,
                    "gmres_iters_last": its_small, "flux_err_last": brsm["flux_err"],
                    "value_incl_grating_factor": 1.0 / (t_small / args.steps + fac_small / 1e3),
                    "workload": "M=10 disks r=0.04 index 2, p=10, k=(10,15,20), N=128, theta=-pi/5, tol 1e-12",
                    "step": "set_inclusions + factor (S, B, C, pair table) + FP64 GMRES + Bragg on the factored grating"}

    # learned warm start: the headline geometry under a (phi, k_top) design sweep; the network is
    # trained by the library's kernels on the solutions of the first sweep points, then each
    # held-out point is solved (FP64 GMRES) from the zero start and from the network's start
    wres = None
    if not args.no_warm:
        from paper_1412_7466_gb300.warmstart import SweepTrainer
        n_tr, n_ev = args.warm_train, args.warm_eval
        pts = W.sweep_points(n_tr + n_ev, seed=5)
        big_w = args.warm_geometry == "mixed4000"
        geo = W.config("mixed4000", seed=1)["disks"] if big_w else cfg0["disks"]
        Mw = geo["xy"].shape[0]
        eval_prec = GS_C64 if big_w else GS_FP64
        gw = GratingSolver(local)
        tr = SweepTrainer(gw, p)
        k_lo, k_hi = 35.0, 45.0

        def load_point(phi, kt):
            dk = dict(geo)
            dk["kp"] = np.full(Mw, 2.0 * kt)              # index 2 relative to k_top
            gw.set_layers(W.scaled_grating("headline", kt))
            gw.set_incidence([-math.pi / 2 + phi])
            gw.set_inclusions(dk)
            gw.factor()

        t0 = time.perf_counter()
        for q in range(n_tr):
            load_point(*pts[q])
            gw.solve(tol=1e-9, maxit=4000, restart=500, precision=GS_C64)
            if q == 0:
                tr.begin(W.mlp_init(p, 11), (-math.pi / 2 - math.pi / 3, -math.pi / 2 + math.pi / 3), (k_lo, k_hi))
            tr.add()
        t1 = time.perf_counter()
        hist = tr.fit(2000, 3e-3, 1e-4)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        tz = tw = 0.0
        it_z, it_w, rel0, bdiff = [], [], [], []
        for q in range(n_tr, n_tr + n_ev):
            load_point(*pts[q])
            a_, b_ = ev(), ev()
            a_.record(stream)
            gw.solve(tol=tol, maxit=8000, restart=500, precision=eval_prec)
            brz = gw.bragg()
            b_.record(stream)
            b_.synchronize()
            tz += a_.elapsed_time(b_) / 1e3
            it_z.append(gw.stats()[0])
            a_, b_ = ev(), ev()
            a_.record(stream)
            b0, r0, used = gw.warm_start()
            gw.solve(tol=tol, maxit=8000, restart=500, precision=eval_prec, beta0=b0)
            brw = gw.bragg()
            b_.record(stream)
            b_.synchronize()
            tw += a_.elapsed_time(b_) / 1e3
            it_w.append(gw.stats()[0])
            rel0.append(r0 if used else 1.0)
            bdiff.append(float(np.linalg.norm(np.r_[brw["c"], brw["d"]] - np.r_[brz["c"], brz["d"]]) /
                               np.linalg.norm(np.r_[brz["c"], brz["d"]])))
        gw.close()
        wres = {"value": n_ev / tw, "unit": "solves/s",
                "dtype": ("c64 translation + f64 refinement" if big_w else "f64") + " (network bf16/fp32)",
                "zero_start_value": n_ev / tz,
                "gmres_iters_zero_start": it_z, "gmres_iters_warm_start": it_w,
                "initial_relres_warm_start": rel0,
                "max_bragg_rel_diff_warm_vs_zero": max(bdiff),
                "train_solves": n_tr, "eval_solves": n_ev, "train_epochs": len(hist),
                "train_loss_first_last": [hist[0], hist[-1]],
                "collect_s": t1 - t0, "train_s": t2 - t1,
                "sweep": (("M=4000 geometry (r=0.004" if big_w else "headline geometry (M=1000, r=0.008")
                          + ", p=12), k=(1,1.5,2) k_top, kp=2 k_top, "
                          f"(phi, k_top) iid in [-pi/3, pi/3] x [35, 45] (seed 5); first {n_tr} points train "
                          f"(complex64 + FP64 refinement to 1e-9), next {n_ev} evaluate ("
                          + ("mixed complex64 + FP64 refinement" if big_w else "FP64 GMRES") + " to 1e-11)"),
                "step": "warm_start (features, network, start, FP64 residual check) + solve + Bragg; "
                        "the grating factorisation per sweep point is outside the timed region"}

    peak64 = gs.probe_fma(GS_FP64)
    peak32_scalar = gs.probe_fma(GS_C64)
    peak32 = gs.probe_fma(GS_PROBE_F32X2)   # the complex64 kernel issues packed two-wide FP32 FMAs
    gs.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    flops_per_launch = 8.0 * nc * nc * (3.0 * M * M - M)
    r64 = res["fp64"]["r"]
    n64, ms64 = r64["prof"]["fp64"]
    avg64 = ms64 / max(n64, 1)
    ach64 = flops_per_launch / (avg64 * 1e-3) / 1e12
    rmx = res["mixed_c64_ir"]["r"]
    nmx32, ms_mx32 = rmx["prof"]["c64"]
    nmx64, ms_mx64 = rmx["prof"]["fp64"]
    avg32 = ms_mx32 / max(nmx32, 1)
    ach32 = flops_per_launch / (avg32 * 1e-3) / 1e12
    value = job_throughput(world, args.steps, r64["elapsed"])
    value_mx = job_throughput(world, args.steps, rmx["elapsed"])
    d2h = res["fp64"]["n_cd"] * (16 + 4) + 8

    def variant(name, vv, rr, dtype):
        x = res[name]
        return {"value": vv, "unit": "solves/s", "dtype": dtype, "ms_per_step": 1e3 * rr["elapsed"] / args.steps,
                "gmres_iters_per_step": rr["iters"], "bragg_rel_err_vs_oracle": x["err"],
                "bragg_max_elementwise_rel_err_vs_oracle": x["err_el"], "flux_err": x["flux"],
                "refinement_sweeps": x["outer"], "gpu_launches": rr["launches"], "clocks": rr["clocks"],
                "e2e": {"value": job_throughput(world, args.steps, x["e2e"]), "unit": "solves/s",
                        "h2d_bytes_per_step": M * 4 * 8, "d2h_bytes_per_step": d2h}}

    per_step_grating = grating_ms / 1e3
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * r64["elapsed"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": world, "parallelism": f"replicas{world}",
                   "step": "one new seeded geometry per step on the factored grating: coupling S, B, C "
                           "(a4), rhs, GMRES (translation + low-rank), Bragg amplitudes",
                   "l2": "inputs larger than L2: B (482 MB) and C (506 MB) are rebuilt and streamed every step"},
        "gmres_iters": r64["iters"], "bragg_rel_err_vs_oracle": res["fp64"]["err"],
        "bragg_max_elementwise_rel_err_vs_oracle": res["fp64"]["err_el"], "flux_err": res["fp64"]["flux"],
        "grating_factor_ms": grating_ms, "grating_factor_phases": factor_stats, "coupling_ms": couple_ms,
        "value_incl_grating_factor": 1.0 / (r64["elapsed"] / args.steps + per_step_grating),
        "pair_translations_per_s": (3 * M * M - M) * n64 / (ms64 * 1e-3) if ms64 > 0 else None,
        "roofline": {"bound": "alu", "kernel": "k_translate_f64_tab<12>", "achieved": ach64, "peak": peak64,
                     "unit": "TFLOP/s", "frac": ach64 / peak64,
                     "peak_source": "measured: FP64 FMA-chain probe (gs_probe_fma) in this process",
                     "traffic": TAB_DRAM_BYTES_PER_PAIR * (3 * M * M - M),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_translate_f64_tab "
                                       "at M=500 (599.6 MB), scaled per launch by the pair count",
                     "flops_per_launch": flops_per_launch, "avg_launch_ms": avg64,
                     "launches_timed": n64},
        "clocks": r64["clocks"],
        "gpu_launches": r64["launches"],
        "e2e": {"value": job_throughput(world, args.steps, res["fp64"]["e2e"]), "unit": "solves/s",
                "h2d_bytes_per_step": M * 4 * 8, "d2h_bytes_per_step": d2h},
        "variants": {
            "plain_fp64": variant("fp64", value, r64, "f64"),
            "mixed_c64_ir": dict(variant("mixed_c64_ir", value_mx, rmx, "c64 translation + f64 refinement"),
                                 pre_refinement_bragg_rel_err=pre_err,
                                 roofline={"bound": "alu", "kernel": "k_translate_c64_tab<12>", "achieved": ach32,
                                           "peak": peak32, "unit": "TFLOP/s", "frac": ach32 / peak32,
                                           "peak_source": "measured: packed FP32 (fma.rn.f32x2) FMA-chain probe "
                                                          "(gs_probe_fma); scalar FFMA probe "
                                                          f"{peak32_scalar:.1f} TFLOP/s",
                                           "flops_per_launch": flops_per_launch,
                                           # the complex64 table streams from HBM at the same time
                                           "hbm": {"bytes_per_launch": TAB32_BYTES_PER_PAIR * (3 * M * M),
                                                   "achieved_gbs": TAB32_BYTES_PER_PAIR * (3 * M * M)
                                                   / (avg32 * 1e-3) / 1e9,
                                                   "frac": TAB32_BYTES_PER_PAIR * (3 * M * M) / (avg32 * 1e-3)
                                                   / 1e9 / PEAKS.get("hbm_gbs", 1.0),
                                                   "peak": PEAKS.get("hbm_gbs"),
                                                   "unit": "GB/s"},
                                           "avg_launch_ms": avg32, "launches_timed": nmx32,
                                           "fp64_residual_launches": nmx64,
                                           "fp64_residual_ms": ms_mx64}),
            "mixed_c64_ir_M4000": bigres,
            "field_grid_fp64": fres,
            "translate_multi_tc_bf16": tcres,
            "batched_c64_ir": bres,
            "warm_start_fp64": wres,
            "angles_lockstep_c64_ir": angres,
            "small_fp64": smallres,
        },
    }
    if world == 1 and not args.no_cpu_baseline:
        from oracle import m2l
        m2l.build()
        oh = OracleHeadline(cfg0)
        t_slice = oh.slice(0)
        v = 1.0 / (ORACLE_SLICES * t_slice)
        t_small = oracle_small_complete()
        t_small1 = oracle_small_one_core()
        out["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": cores(), "kind": "oracle",
                               "sample": oh.describe(t_slice),
                               "complete_solve_small": {
                                   "workload": "M=10 disks r=0.04, p=10, k=(10,15,20), N=128, theta=-pi/5",
                                   "what": "complete solve: assembly, SVD, S, B_phys, C, dense Schur matrix + LU, Bragg",
                                   "seconds_all_cores": t_small, "seconds_one_core": t_small1,
                                   "solves_per_s_all_cores": 1.0 / t_small,
                                   "solves_per_s_one_core": (1.0 / t_small1) if t_small1 else None}}
        if args.cpu_complete:
            out["cpu_baseline"]["complete_solve_headline"] = oracle_headline_complete(cfg0)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
