#!/usr/bin/env python
"""Throughput benchmark of GPU DDPS: solves per second at true relative
residual ||f - A x||_inf / ||f||_inf <= 1e-10.

Workload (default): 3-D 7-point convection-diffusion on a 64^3 grid, one
convection constant per axis ~ U[0, 50] (seeded), 16 z-slab blocks of 3-5
planes, f = A x_true with x_true ~ U[-1, 1] (seed 0).  One step = one whole
DDPS pass over one system: ddps_factor (Fig. 2 steps 1-5: split, block LU,
spikes, G^) + ddps_solve (Fig. 2 step 6: outer BiCGStab with the Fig. 3
preconditioner).  The symbolic analysis depends only on the sparsity
pattern; it runs once before the timed region and is reported as
``analyze_ms``.

Forms: ``mixed`` = FP32 block factors and spike solves with the spike
products on the tensor cores (bf16x3 operands, fp32 accumulation), G^ stored
in FP16 (products accumulate in FP32), FP32 inner vectors, FP64 outer Krylov
(the headline); ``mixed_simt`` = the
same with FP32 SIMT spike products; ``fp64`` = plain FP64 DDPS.

Under torchrun every rank solves its own copy of the workload (the systems
are independent; no collective on the data path) and ``value`` counts the
solves of all ranks over the slowest rank's time.
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
sys.path.insert(0, ROOT)
# The CPU oracle legs run on one host thread: BLAS pools are sized from these
# variables when numpy first loads (nothing on the GPU path uses host BLAS).
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")


class _one_thread:
    """Holds the host BLAS pools to one thread where threadpoolctl is
    installed; otherwise the variables above already did."""

    def __enter__(self):
        try:
            from threadpoolctl import threadpool_limits
            self._lim = threadpool_limits(1)
        except ImportError:
            self._lim = None
        return self

    def __exit__(self, *exc):
        if self._lim is not None:
            self._lim.restore_original_limits()
        return False

METRIC = "solves/s at rel. residual 1e-10, mixed/batched/learned vs plain FP64 DDPS on GB300"
UNIT = "solves/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cd3d_64_slabs16",
                    choices=["cd3d_64_slabs16", "cd2d_64_p4", "cd3d_48_slabs8", "cd2d_batch256",
                             "randband_1m", "cd3d_48_seq"])
    ap.add_argument("--form", choices=["mixed", "mixed_simt", "fp64", "implicit", "direct", "ilu"],
                    default="mixed",
                    help="mixed: the paper's method with FP32 factors, tensor-core spikes and "
                         "FP16 G^; implicit: the variant that applies G^ by block solves "
                         "instead of forming the spikes")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="steps of the plain-FP64 comparison run (0 skips it; default 3, "
                         "0 for randband_1m whose FP64 factor takes over a minute)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads' sub-results (256-system batch, 1M random "
                         "band, 48^3 learned sequence) and the FP32-G^ and solve-only lines")
    ap.add_argument("--drop-sweep", action="store_true",
                    help="instead of the bench line: the Sec. 3 column rule on the random-band "
                         "workload for several delta (outer/inner iterations, |c|, solves/s)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# workload and solver settings
# ----------------------------------------------------------------------------

def make_workload(name):
    """Returns (problem, sys_block_ptr or None, number of systems, drop rule or None)."""
    import types

    import numpy as np

    import workloads as W
    if name == "cd3d_64_slabs16":
        return W.cfg2(), None, 1, None
    if name == "cd2d_64_p4":
        return W.cfg1(), None, 1, None
    if name in ("cd3d_48_slabs8", "cd3d_48_seq"):
        return W.cfg5(1), None, 1, None
    if name == "randband_1m":
        return W.cfg4(), None, 1, ("abs", 1e-4)
    if name == "cd2d_batch256":
        from paper_1008_1700_gb300.solver import stack_systems
        probs = W.cfg3()
        rp, ci, v, bp, sbp, srp = stack_systems([(p.rowptr, p.colind, p.values, p.block_ptr)
                                                 for p in probs])
        P = types.SimpleNamespace(n=int(srp[-1]), nnz=int(rp[-1]), rowptr=rp, colind=ci, values=v,
                                  block_ptr=bp, p=len(bp) - 1,
                                  f=np.concatenate([q.f for q in probs]),
                                  x_true=np.concatenate([q.x_true for q in probs]), systems=probs)
        return P, sbp, len(probs), None
    raise ValueError(name)


def form_options(form):
    from paper_1008_1700_gb300 import native as N
    base = dict(tol_out=1e-10, maxit_out=1000, tol_in=1e-4, maxit_in=100)
    if form == "mixed":
        # FP32 block factors and spike solves, spike products and the block-LU
        # updates of large fronts on the tensor cores (bf16x3 operands, fp32
        # accumulation), FP16 G^ storage with FP32
        # accumulation, FP32 inner vectors, FP64 outer
        base.update(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16X3, ghat_prec=N.DDPS_FP16,
                    inner_prec=N.DDPS_FP32, update_prec=N.DDPS_BF16X3)
    elif form == "direct":
        # the mixed form with 6.3 solved directly (block LU of the block-tridiagonal
        # G^ of a chain of slabs) instead of by the inner BiCGStab
        base.update(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_BF16X3, ghat_prec=N.DDPS_FP16,
                    inner_prec=N.DDPS_FP32, update_prec=N.DDPS_BF16X3,
                    reduced_solver=N.DDPS_REDUCED_DIRECT)
    elif form == "ilu":
        # Sec. 3's approximate block factors: ILU(0) in FP32, SIMT spike solves,
        # FP16 G^, FP32 inner vectors, FP64 outer
        base.update(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_FP32, ghat_prec=N.DDPS_FP16,
                    inner_prec=N.DDPS_FP32, factor_kind=N.DDPS_FACTOR_ILU0)
    elif form == "implicit":
        # variant (departs from Fig. 2 step 4): no spikes, G^ v = v + (D~^-1 R~ v)(c)
        base.update(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_FP32, ghat_prec=N.DDPS_FP32,
                    inner_prec=N.DDPS_FP32, ghat_mode=N.DDPS_GHAT_IMPLICIT)
    elif form == "mixed_simt":
        base.update(factor_prec=N.DDPS_FP32, spike_prec=N.DDPS_FP32, ghat_prec=N.DDPS_FP32,
                    inner_prec=N.DDPS_FP32)
    else:
        base.update(factor_prec=N.DDPS_FP64, spike_prec=N.DDPS_FP64, ghat_prec=N.DDPS_FP64,
                    inner_prec=N.DDPS_FP64)
    return base


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "sm_max_mhz": float(pk.get("sm_max_mhz", 2070.0)),
                "bf16_tflops": float(pk.get("bf16_tflops", 1900.0)),
                "bf16_tflops_sustained": float(pk.get("bf16_tflops_sustained", 1700.0)),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# algorithmic work per kernel class (bytes for memory-bound, flops for ALU-bound)
# ----------------------------------------------------------------------------

# DRAM bytes per algorithmic byte of a launch, from one ncu capture of the
# kernel (dram__bytes_read.sum + dram__bytes_write.sum over the algorithmic
# bytes of that launch; profiles/ncu_ghat_matvec_tiled_cd3d_48.md): a launch's
# traffic is this ratio times its algorithmic bytes.  Classes without a
# capture of their current kernel report null.
TRAFFIC_RATIO = {"ghat_matvec": (1.012, "ncu --set full, k_ghat_matvec_tiled<__half,float>, "
                                        "cd3d_48_slabs8 (279.6 MB per 276.3 MB), scaled by bytes")}


def algorithmic_work(sizes, P, form, steps, prof):
    """Per class: (kind, total algorithmic amount over the timed region)."""
    sf = 8 if form == "fp64" else 4
    sg = 8 if form == "fp64" else (2 if form in ("mixed", "direct", "ilu") else 4)  # G^ storage
    si = sf
    n, nnz, m = sizes["n"], sizes["nnz"], sizes["m"]
    out = {}
    # per factor: Fig. 2 steps 2 and 4
    out["front_lu"] = ("flops", sizes["factor_flops"] * steps)
    out["spike_fwd"] = ("flops", sizes["spike_flops"] / 2 * steps)
    out["spike_bwd"] = ("flops", sizes["spike_flops"] / 2 * steps)
    # values and map read, front entries written, pivot thresholds (one pass over A)
    out["assemble"] = ("bytes", (nnz * (8 + 8 + sf) + nnz * 20 + n * 8) * steps)
    out["ghat_extract"] = ("bytes", sizes["ghat_entries"] * (sf + sg) * steps)
    # per call of the solve phase
    calls = {k: v[1] for k, v in prof.items()}
    out["block_solve"] = ("bytes", (sizes["factor_lu_entries"] * sf + n * 16) * calls["block_solve"])
    if form == "implicit":
        # R~ product, one block solve (factors once, permuted in/out) and the gathered add
        out["ghat_matvec"] = ("bytes", (sizes["nnz_rt"] * 12 + n * 8 + sizes["factor_lu_entries"] * sf +
                                        n * 16 + m * (2 * si + 8)) * calls["ghat_matvec"])
    else:
        out["ghat_matvec"] = ("bytes", (sizes["ghat_entries"] * sg + 2 * m * si) * calls["ghat_matvec"])
    out["spmv"] = ("bytes", (nnz * 12 + (n + 1) * 4 + n * 16) * calls["spmv"])
    out["direct_factor"] = ("flops", sizes.get("direct_flops", 0.0) * steps)
    out["direct_solve"] = ("bytes", (sizes.get("direct_bytes", 0) + m * 24) * calls.get("direct_solve", 0))
    return out


# ----------------------------------------------------------------------------
# CPU oracle sample (bench's CPU-baseline leg and the reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(P, nblocks=2, ncols=256, counts=None):
    """Times the oracle, as it stands, on a bounded sample of one DDPS solve
    of the workload and scales each measured piece to the whole solve.

    Measured on the sample (one thread: BLAS is held to one thread, SuperLU
    is single-threaded):
      * Fig. 2 step 1 and 5 (split, c) on the whole matrix;
      * step 2 (LU) of `nblocks` blocks, scaled by the number of blocks;
      * step 4 (spikes) of `ncols` columns of those blocks, scaled by the
        blocks' coupling-column counts;
      * step 6 pieces: one block solve of each sampled block (scaled to all
        blocks), one product of each sampled block's G^ rows with a vector
        (scaled by the G^ entries), one product with A;
    and combined with the iteration counts of a whole solve (`counts`:
    outer products with A, Fig. 3 applications, inner iterations).
    Returns (seconds per solve, wall seconds of the sample, description)."""
    import numpy as np

    from oracle.ddps_oracle import csr, factor_blocks, interface_columns, split_block_rows

    counts = counts or DEFAULT_ORACLE_COUNTS
    with _one_thread():
        t0 = time.perf_counter()
        A = csr(P.n, P.rowptr, P.colind, P.values)
        D, R = split_block_rows(A, P.block_ptr)
        c = interface_columns(R)
        t_split = time.perf_counter() - t0
        bp = P.block_ptr
        lu_t, sp_t, bs_t, mv_t = [], [], [], []
        pick = np.linspace(0, P.p - 1, min(nblocks, P.p)).round().astype(int)
        g_entries_tot = 0
        for i in range(P.p):
            Ri = R[bp[i]:bp[i + 1], :]
            rows_c = np.count_nonzero((c >= bp[i]) & (c < bp[i + 1]))
            g_entries_tot += rows_c * len(np.unique(Ri.indices))
        g_entries_samp = 0
        for i in pick:
            t1 = time.perf_counter()
            lu = factor_blocks([D[i]])[0]
            lu_t.append(time.perf_counter() - t1)
            Ri = R[bp[i]:bp[i + 1], :]
            ci = np.unique(Ri.indices)
            k = min(ncols, len(ci))
            if k:
                t2 = time.perf_counter()
                cols = Ri.tocsc()[:, ci[:k]].toarray()
                G = lu.solve(cols)
                sp_t.append((time.perf_counter() - t2) * len(ci) / k)
                rows_c = c[(c >= bp[i]) & (c < bp[i + 1])] - bp[i]
                Gh = G[rows_c, :]
                v = np.ones(k)
                t3 = time.perf_counter()
                for _ in range(3):
                    Gh @ v
                mv_t.append((time.perf_counter() - t3) / 3 * len(ci) / k)
                g_entries_samp += len(rows_c) * len(ci)
            y = np.ones(bp[i + 1] - bp[i])
            t4 = time.perf_counter()
            lu.solve(y)
            bs_t.append(time.perf_counter() - t4)
        xv = np.ones(P.n)
        t5 = time.perf_counter()
        for _ in range(3):
            A @ xv
        t_spmv = (time.perf_counter() - t5) / 3
        wall = time.perf_counter() - t0
    scale_b = P.p / len(pick)
    t_factor = t_split + sum(lu_t) * scale_b + sum(sp_t) * scale_b
    t_block_solve = sum(bs_t) * scale_b
    t_ghat = (sum(mv_t) * g_entries_tot / g_entries_samp) if g_entries_samp else 0.0
    t_solve = (counts["spmv"] * t_spmv + 2 * counts["applies"] * t_block_solve +
               2 * counts["inner"] * t_ghat)
    desc = ("oracle (numpy/scipy, one thread) timed on a sample: split and c of the whole "
            "matrix, LU and %d spike columns of %d of the %d blocks, one block solve and one "
            "G^-row product of those blocks, one product with A; scaled to the whole solve "
            "(factor %.1f s, solve %.1f s per solve) with the iteration counts of a whole "
            "oracle solve (%d products with A, %d Fig. 3 applications, %d inner iterations); "
            "sample wall %.1f s" % (ncols, len(pick), P.p, t_factor, t_solve, counts["spmv"],
                                    counts["applies"], counts["inner"], wall))
    return t_factor + t_solve, wall, desc


# Iteration counts of one whole oracle solve (eps_in 1e-4, tol 1e-10) of the
# 64^3 slab workload, measured once (1.5 outer iterations = 3 Fig. 3
# applications with 15, 12 and 10.5 inner iterations; products with A: 2 per
# outer iteration plus the true-residual checks).
DEFAULT_ORACLE_COUNTS = {"spmv": 5, "applies": 3, "inner": 38}


def oracle_batch_sample(systems, count=3):
    """Whole oracle solves (Fig. 2 and 3, eps_in 1e-4, tol 1e-10) of the first
    `count` systems of a batch, scaled to the batch by the number of unknowns."""
    from oracle.ddps_oracle import DDPSOracle
    with _one_thread():
        t0 = time.perf_counter()
        nsamp = 0
        for p in systems[:count]:
            DDPSOracle(p.n, p.rowptr, p.colind, p.values, p.block_ptr).solve(p.f, tol=1e-10,
                                                                              eps_in=1e-4)
            nsamp += p.n
        wall = time.perf_counter() - t0
    ntot = sum(p.n for p in systems)
    est = wall * ntot / nsamp
    return est, wall, ("whole oracle solves (Fig. 2 and 3, one thread) of %d of the %d systems "
                       "(%.1f s wall), scaled by unknowns to the batch" % (count, len(systems), wall))


def cpu_baseline_entry(P, nsys, workload):
    if nsys > 1:
        est, wall, sample = oracle_batch_sample(P.systems)
    else:
        nb, nc = (1, 256) if workload == "randband_1m" else (4, 1024)
        est, wall, sample = oracle_sample(P, nblocks=nb, ncols=nc)
    return {"value": nsys / est, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}


# ----------------------------------------------------------------------------
# replicas: one rank per GPU, no data-path collective; the step time is the
# slowest rank's and the value counts every rank's systems
# ----------------------------------------------------------------------------

def max_over_ranks_of(v, dist=None, device="cuda"):
    """Largest value of v over the ranks of the process group (v itself
    without one)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ms_max, world, units_per_rank, steps):
    """Units per second of the whole job: every rank's units over the slowest
    rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


# ----------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ----------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    P, sbp, nsys, drop = make_workload(args.workload)
    nb, nc = (1, 32) if args.workload == "randband_1m" else (1, 128)

    def sample():
        if nsys > 1:
            return oracle_batch_sample(P.systems, count=1)
        return oracle_sample(P, nblocks=nb, ncols=nc)

    for _ in range(args.warmup):
        sample()
    ests, walls, desc = [], [], ""
    for _ in range(args.steps):
        e, w, desc = sample()
        ests.append(e)
        walls.append(w)
    sec = statistics.mean(ests)
    value = nsys / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # each step is one bounded sample of a solve; its wall time is the step time
        "ms_per_step": statistics.mean(walls) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "systems_per_step": nsys, "n": P.n, "nnz": P.nnz,
                   "blocks": P.p, "parallelism": "host cores"},
        "seconds_per_solve_scaled": sec,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def timed(stream, fn, steps):
    """CUDA-event milliseconds of `steps` calls of fn on `stream` (synchronised on
    both sides); returns (ms, list of fn's results)."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def kernel_table(prof, work, ms_total, peaks):
    """Per kernel class: time, launch groups, share of the profiled steps and
    achieved rate (plus the fraction of the HBM peak for memory-bound ones)."""
    kern = {}
    for cls, (kms, cnt) in prof.items():
        if cnt == 0:
            continue
        kind, amount = work.get(cls, ("bytes", 0.0))
        rate = amount / (kms / 1e3) if kms > 0 else 0.0
        e = {"ms": round(kms, 3), "groups": cnt, "share": round(kms / ms_total, 4),
             "achieved": round(rate / (1e9 if kind == "bytes" else 1e12), 3),
             "unit": "GB/s" if kind == "bytes" else "TFLOP/s"}
        if kind == "bytes":
            e["frac_hbm"] = round(e["achieved"] / peaks["hbm_gbs"], 4)
        kern[cls] = e
    return kern


def measure_workload(name, form, steps, warmup, stream, extra_opts=None, solve_only=False,
                     profile=False):
    """Factor + solve steps of one workload in one form (profiling off):
    solves/s and accuracy; used for the sub-results of the bench line."""
    import numpy as np
    import torch

    from paper_1008_1700_gb300 import Solver, native as N

    P, sbp, nsys, drop = make_workload(name)
    opts = form_options(form)
    if drop is not None:
        opts.update(drop_mode=N.DDPS_DROP_ABS, drop_tol=drop[1])
    if extra_opts:
        opts.update(extra_opts)
    t0 = time.perf_counter()
    S = Solver(P.rowptr, P.colind, P.block_ptr, sbp, P.values if drop else None, **opts)
    analyze_ms = (time.perf_counter() - t0) * 1e3
    vals = torch.tensor(P.values, device="cuda")
    f = torch.tensor(P.f, device="cuda")
    x = torch.empty_like(f)

    def step():
        S.factor(vals)
        return S.solve(f, x)[1]

    for _ in range(warmup):
        step()
    ms, infos = timed(stream, step, steps)
    xh = x.cpu().numpy()
    out = {"value": nsys * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "systems_per_step": nsys, "form": form, "n": P.n,
           "blocks": P.p, "m_interface": S.m, "analyze_ms": round(analyze_ms, 1),
           "relres_inf": max(i["relres_inf"] for i in infos),
           "converged": all(i["status"] == "DDPS_OK" for i in infos),
           "outer_iterations": infos[-1]["outer_iterations"],
           "inner_iterations": infos[-1]["inner_iterations"]}
    if P.x_true is not None:
        out["rel_err_vs_xtrue"] = float(np.linalg.norm(xh - P.x_true) / np.linalg.norm(P.x_true))
    if solve_only:
        nr = 4
        F4 = torch.stack([f * (1.0 + 0.25 * j) for j in range(nr)]).contiguous()
        X4 = torch.empty_like(F4)
        S.solve(F4, X4)
        sms, sinf = timed(stream, lambda: S.solve(F4, X4)[1], 2)
        out["solve_only"] = {"value": 2 * nr * nsys / (sms / 1e3), "unit": UNIT,
                             "ms_per_solve": sms / (2 * nr), "nrhs_per_call": nr,
                             "relres_inf": max(i["relres_inf"] for i in sinf)}
        # per-class split of one factor + solve
        S.set_profiling((1 << len(N.PROF_CLASSES)) - 1)
        S.profile(reset=True)
        step()
        prof = S.profile(reset=True)
        S.set_profiling(0)
        out["classes_ms"] = {k: round(v[0], 3) for k, v in prof.items() if v[1]}
    if profile:
        # one profiled factor + solve: per-class time, rate and fraction of the HBM peak
        S.set_profiling((1 << len(N.PROF_CLASSES)) - 1)
        S.profile(reset=True)
        pms, _ = timed(stream, step, 1)
        prof = S.profile(reset=True)
        S.set_profiling(0)
        out["kernels"] = kernel_table(prof, algorithmic_work(S.sizes, P, form, 1, prof), pms,
                                      load_peaks())
    S.close()
    del vals, f, x
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1008_1700_gb300 import Solver, native as N

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        return max_over_ranks_of(v, dist, "cuda")

    P, sbp, nsys, drop = make_workload(args.workload)
    opts = form_options(args.form)
    if drop is not None:
        opts.update(drop_mode=N.DDPS_DROP_ABS, drop_tol=drop[1])
    t0 = time.perf_counter()
    S = Solver(P.rowptr, P.colind, P.block_ptr, sbp, P.values if drop else None, **opts)
    analyze_ms = (time.perf_counter() - t0) * 1e3
    sizes = S.sizes
    vals = torch.tensor(P.values, device="cuda")
    f = torch.tensor(P.f, device="cuda")
    x = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    def step():
        S.factor(vals)
        _, info = S.solve(f, x)
        return info

    for _ in range(args.warmup):
        step()

    # timed region: profiling off, inputs resident in HBM (G^ and the fronts
    # are larger than L2, so every product streams them from HBM)
    launches0 = S.launch_count()
    clocks = ClockSampler(local)
    barrier()
    ms, infos = timed(stream, step, args.steps)
    barrier()
    clk = clocks.stop()
    launches = S.launch_count() - launches0
    ms_max = max_over_ranks(ms)
    value = whole_job_rate(ms_max, world, nsys, args.steps)

    # accuracy of the last step against the known solution and the residual
    xh = x.cpu().numpy()
    err_xtrue = (float(np.linalg.norm(xh - P.x_true) / np.linalg.norm(P.x_true))
                 if P.x_true is not None else None)
    relres = max(i["relres_inf"] for i in infos)
    converged = all(i["status"] == "DDPS_OK" for i in infos)

    # per-class split from a separate pass of the same steps with every
    # kernel class bracketed by CUDA events on the launching stream
    psteps = min(args.steps, 5)
    S.set_profiling((1 << len(N.PROF_CLASSES)) - 1)
    S.profile(reset=True)
    pms, _ = timed(stream, step, psteps)
    prof = S.profile(reset=True)
    S.set_profiling(0)
    peaks = load_peaks()
    work = algorithmic_work(sizes, P, args.form, psteps, prof)
    kern = kernel_table(prof, work, pms, peaks)
    dom = max(kern, key=lambda k: kern[k]["ms"])
    dk = kern[dom]
    sm_mhz = peaks["sm_max_mhz"]
    if dk["unit"] == "GB/s":
        peak = peaks["hbm_gbs"]
        bound = "hbm"
        peak_note = f"{peaks['source']} HBM copy bandwidth"
    elif args.form in ("mixed", "direct") and dom in ("spike_fwd", "spike_bwd", "front_lu"):
        # bf16 tensor-core products (3 passes per algorithmic product): sustained bf16 peak
        peak = peaks["bf16_tflops_sustained"]
        bound = "tensor"
        peak_note = (f"{peaks['source']} sustained dense bf16 (cuBLAS); achieved counts the "
                     "algorithmic flops once, the tensor cores run 3 bf16 passes" +
                     ("; the LU's block updates run there, its panels and triangular "
                      "inverses on the SIMT cores" if dom == "front_lu" else ""))
    else:
        # FP32 (mixed) or FP64 (plain) SIMT: 152 SMs x lanes x 2 flops x max SM clock
        lanes = 2 if args.form == "fp64" else 128
        peak = 152 * lanes * 2 * sm_mhz * 1e6 / 1e12
        bound = "alu"
        peak_note = ("FP64: 152 SMs x 2 FMA/clk x 2 x %.0f MHz" % sm_mhz if args.form == "fp64"
                     else "FP32 SIMT: 152 SMs x 128 lanes x 2 x %.0f MHz" % sm_mhz)
    traffic, traffic_note = None, None
    if dk["unit"] == "GB/s" and dom in TRAFFIC_RATIO and args.form == "mixed":
        ratio, traffic_note = TRAFFIC_RATIO[dom]
        per_launch = work[dom][1] / max(prof[dom][1], 1)
        traffic = int(ratio * per_launch)
    roof = {"kernel": dom, "bound": bound, "achieved": dk["achieved"], "peak": round(peak, 2),
            "unit": dk["unit"], "frac": round(dk["achieved"] / peak, 4), "traffic": traffic,
            "traffic_source": traffic_note, "peak_source": peak_note,
            "timing": "CUDA events per kernel class on the launching stream, over a pass of "
                      "%d steps after the timed region (the timed region runs unprofiled)" % psteps}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.form == "fp64" else ("bf16x3+f16+f32+f64" if args.form in ("mixed", "direct") else "f32+f64"),
        "variant": ("implicit G^: block solves instead of stored spikes (departs from Fig. 2 "
                    "step 4)" if args.form == "implicit" else
                    "6.3 solved directly: block LU of the block-tridiagonal G^ of the slab chain"
                    if args.form == "direct" else None),
        "data": "synthetic",
        "config": {"workload": args.workload, "systems_per_step": nsys, "n": P.n, "nnz": P.nnz,
                   "blocks": P.p,
                   "m_interface": sizes["m"], "ghat_entries": sizes["ghat_entries"],
                   "form": args.form, "parallelism": f"replicas{world}",
                   "l2": ("working set (fronts %.2f GB) larger than L2" %
                          (sizes["factor_entries"] * 4 / 1e9) if args.form == "implicit" else
                          "working set (G^ %.1f GB) larger than L2" %
                          (sizes["ghat_entries"] * (8 if args.form == "fp64" else
                                                    (2 if args.form in ("mixed", "direct")
                                                     else 4)) / 1e9)),
                   "tol_out": opts["tol_out"], "tol_in": opts["tol_in"]},
        "analyze_ms": round(analyze_ms, 1),
        "accuracy": {"relres_inf": relres, "rel_err_vs_xtrue": err_xtrue, "converged": converged,
                     "outer_iterations": infos[-1]["outer_iterations"],
                     "inner_iterations": infos[-1]["inner_iterations"]},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
        "kernels": kern,
        "hbm_targets": {k: kern[k].get("frac_hbm") for k in ("block_solve", "spmv", "ghat_matvec")
                        if k in kern},
    }

    # e2e through the C ABI with host buffers (pinned): ddps_factor_host copies
    # the values, ddps_solve_host copies f in and x out, all inside the timed region
    if not args.no_e2e:
        vals_h = torch.tensor(P.values).pin_memory()
        f_h = torch.tensor(P.f).pin_memory()
        x_h = torch.empty_like(f_h).pin_memory()

        def e2e_step():
            N.ddps_factor_host(S.h, vals_h)
            N.ddps_solve_host(S.h, f_h, x_h)

        e2e_step()
        barrier()
        ems, _ = timed(stream, e2e_step, args.steps)
        barrier()
        ems = max_over_ranks(ems)
        line["e2e"] = {"value": whole_job_rate(ems, world, nsys, args.steps), "unit": UNIT,
                       "h2d_bytes_per_step": int(P.nnz * 8 + P.n * 8),
                       "d2h_bytes_per_step": int(P.n * 8),
                       "path": "ddps_factor_host + ddps_solve_host (pinned host buffers)"}

    extras = not args.no_extras and world == 1
    if extras and args.form == "mixed":
        # solve-only throughput with the factors kept (repeated right-hand sides,
        # the factor phase needs none: Sec. 3); 4 right-hand sides per call
        nr = 4
        F4 = torch.tensor(np.stack([P.f * (1.0 + 0.25 * j) for j in range(nr)]), device="cuda")
        X4 = torch.empty_like(F4)
        S.factor(vals)
        S.solve(F4, X4)
        sms, sinf = timed(stream, lambda: S.solve(F4, X4)[1], 2)
        line["solve_only"] = {"value": 2 * nr * nsys / (sms / 1e3), "unit": UNIT,
                              "ms_per_solve": sms / (2 * nr), "nrhs_per_call": nr,
                              "relres_inf": max(i["relres_inf"] for i in sinf)}
        del F4, X4

    # plain FP64 DDPS on the same GPU and workload (the comparison the metric names)
    if args.form != "fp64" and args.fp64_steps > 0:
        o64 = form_options("fp64")
        if drop is not None:
            o64.update(drop_mode=N.DDPS_DROP_ABS, drop_tol=drop[1])
        S64 = Solver(P.rowptr, P.colind, P.block_ptr, sbp, P.values if drop else None, **o64)
        x64 = torch.empty_like(f)

        def step64():
            S64.factor(vals)
            return S64.solve(f, x64)[1]

        step64()
        fms, i64 = timed(stream, step64, args.fp64_steps)
        fms = max_over_ranks(fms)
        v64 = whole_job_rate(fms, world, nsys, args.fp64_steps)
        line["plain_fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": fms / args.fp64_steps,
                              "steps": args.fp64_steps,
                              "relres_inf": max(i["relres_inf"] for i in i64),
                              "outer_iterations": i64[-1]["outer_iterations"]}
        line["speedup_vs_plain_fp64"] = value / v64
        S64.close()

    if extras and args.form == "mixed":
        # the precision form with FP32 storage of G^ (instead of FP16)
        line["fp32_ghat"] = measure_workload(args.workload, "mixed", 3, 1, stream,
                                             {"ghat_prec": N.DDPS_FP32})
        if args.workload in ("cd3d_64_slabs16", "cd3d_48_slabs8"):
            # variant: 6.3 solved directly (block LU of the block-tridiagonal G^)
            line["direct_reduced"] = measure_workload(args.workload, "direct", 3, 1, stream,
                                                      solve_only=True)
        # variant: ILU(0) block factors (approximate LU, Sec. 3)
        line["ilu0_factors"] = measure_workload(args.workload, "ilu", 3, 1, stream)
    S.close()
    del vals, f, x
    torch.cuda.empty_cache()

    if extras and args.workload == "cd3d_64_slabs16":
        # the other workloads, driver-visible: a short timed run of each
        line["workloads"] = {
            "cd2d_batch256": measure_workload("cd2d_batch256", "mixed", 3, 2, stream, profile=True),
            "randband_1m": measure_workload("randband_1m", "mixed", 2, 1, stream, profile=True),
        }
        line["workloads"]["cd3d_48_seq"] = sequence_result(args.form, 10, stream)

    # CPU oracle, bounded sample, rank 0 only
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_entry(P, nsys, args.workload)
        except Exception as ex:  # the GPU line is still printed
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "failed: %s" % ex}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sequence_result(form, eval_steps, stream, train_steps=100):
    """Time sequence of 48^3 systems, b(t) = 20 + 10 sin(2 pi t / 200), fixed
    source: zero-guess solves of steps 1..train_steps collect the reduced
    solutions z^(t), on which the step-change network is trained (the
    library's MLP kernels); then `eval_steps` steps from t = train_steps + 1
    are timed three times, each step factor + guess + solve: with the
    network's guess, with the previous step's z^ (warm start) and with z^ = 0
    (the paper's start)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_1008_1700_gb300 import Solver
    from paper_1008_1700_gb300.learned import StepGuess

    opts = form_options(form)
    P0 = W.cfg5(1)
    S = Solver(P0.rowptr, P0.colind, P0.block_ptr, **opts)
    f = torch.tensor(P0.f, device="cuda")
    x = torch.empty_like(f)
    t0 = time.perf_counter()
    zs, bs = [], []
    for t in range(1, train_steps + 1):
        S.factor(torch.tensor(W.cfg5(t).values, device="cuda"))
        S.set_reduced_guess(None)
        S.solve(f, x)
        zs.append(S.reduced_solution()[0].clone())
        bs.append(W.cfg5_coeff(t))
    model = StepGuess(torch.stack(zs), bs)
    train_s = time.perf_counter() - t0
    ts = list(range(train_steps + 1, train_steps + 1 + eval_steps))
    vals = [torch.tensor(W.cfg5(t).values, device="cuda") for t in ts]

    def run(mode):
        state = {"z": zs[-1], "b": bs[-1], "i": 0, "infos": []}

        def one():
            i = state["i"]
            t = ts[i]
            S.factor(vals[i])
            bt = W.cfg5_coeff(t)
            if mode == "learned":
                S.set_reduced_guess(model.predict(state["z"], bt, state["b"]))
            elif mode == "warm":
                S.set_reduced_guess(state["z"])
            else:
                S.set_reduced_guess(None)
            _, info = S.solve(f, x)
            state["z"] = S.reduced_solution()[0].clone()
            state["b"] = bt
            state["i"] += 1
            return info

        ms, infos = timed(stream, one, len(ts))
        return {"value": len(ts) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / len(ts),
                "first_inner_mean": float(np.mean([i["first_inner_iters"] for i in infos])),
                "inner_mean": float(np.mean([i["inner_iterations"] for i in infos])),
                "relres_max": float(max(i["relres_inf"] for i in infos)),
                "converged": all(i["status"] == "DDPS_OK" for i in infos)}

    run("learned")  # warm-up of the prediction path
    out = {"n": P0.n, "blocks": P0.p, "form": form, "train_steps": f"1-{train_steps}",
           "timed_steps": f"{ts[0]}-{ts[-1]}", "train_s": round(train_s, 2),
           "learned": run("learned"), "warm_start": run("warm"), "zero_guess": run("zero")}
    out["value"] = out["learned"]["value"]
    out["unit"] = UNIT
    S.close()
    return out


def run_sequence_bench(args):
    """The 48^3 learned-guess sequence as its own bench line (timed region:
    `steps` evaluation steps per guess strategy)."""
    import torch
    stream = torch.cuda.current_stream()
    r = sequence_result(args.form, args.steps, stream)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "ms_per_step": r["learned"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f16+f32+f64", "data": "synthetic",
        "config": {"workload": "cd3d_48_seq", "n": r["n"], "blocks": r["blocks"],
                   "train_steps": r["train_steps"], "timed_steps": r["timed_steps"],
                   "form": args.form},
        "train_s": r["train_s"], "learned": r["learned"], "warm_start": r["warm_start"],
        "zero_guess": r["zero_guess"],
    }
    print(json.dumps(line), flush=True)


def run_drop_sweep(args):
    """Sec. 3 column rule (drop column k of R_i when its inf-norm is at most
    delta times the largest of the block) on the 1M random-band workload, one
    row per delta: kept coupling columns, G^ entries, outer and inner
    iterations, factor and solve times and solves/s (mixed form), the way the
    paper varies its dropping threshold.  Times are CUDA events over `steps`
    factor + solve steps after one warm-up step."""
    import numpy as np
    import torch

    import workloads as W
    from paper_1008_1700_gb300 import Solver
    from paper_1008_1700_gb300 import native as N

    P = W.cfg4()
    vals = torch.tensor(P.values, device="cuda")
    f = torch.tensor(P.f, device="cuda")
    x = torch.empty_like(f)
    stream = torch.cuda.current_stream()
    rows = []
    for delta in (0.99, 0.9, 0.6, 0.3, 0.1, 1e-5):
        opts = form_options(args.form)
        opts.update(drop_mode=N.DDPS_DROP_COLUMN, drop_tol=delta)
        t0 = time.perf_counter()
        S = Solver(P.rowptr, P.colind, P.block_ptr, values_host=P.values, **opts)
        analyze_ms = (time.perf_counter() - t0) * 1e3
        sizes = S.sizes
        S.factor(vals)
        S.solve(f, x)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        fac_ms = sol_ms = 0.0
        info = None
        for _ in range(args.steps):
            e0.record(stream)
            S.factor(vals)
            e1.record(stream)
            _, info = S.solve(f, x)
            e2.record(stream)
            torch.cuda.synchronize()
            fac_ms += e0.elapsed_time(e1)
            sol_ms += e1.elapsed_time(e2)
        err = float(np.linalg.norm(x.cpu().numpy() - P.x_true) / np.linalg.norm(P.x_true))
        rows.append({"delta": delta, "m_interface": sizes["m"], "ghat_entries": sizes["ghat_entries"],
                     "outer_iterations": info["outer_iterations"],
                     "inner_iterations": info["inner_iterations"],
                     "factor_ms": round(fac_ms / args.steps, 2), "solve_ms": round(sol_ms / args.steps, 2),
                     "solves_per_s": round(args.steps / ((fac_ms + sol_ms) / 1e3), 4),
                     "relres_inf": info["relres_inf"], "rel_err_vs_xtrue": err,
                     "status": info["status"], "analyze_ms": round(analyze_ms, 1)})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        S.close()
        torch.cuda.empty_cache()
    print(json.dumps({"experiment": "drop_sweep", "rule": "column (Sec. 3)", "workload": "randband_1m",
                      "form": args.form, "steps": args.steps, "rows": rows}), flush=True)


def main():
    args = parse_args()
    if args.drop_sweep:
        run_drop_sweep(args)
        return
    if args.fp64_steps is None:
        args.fp64_steps = 0 if args.workload == "randband_1m" else 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cd3d_48_seq":
        run_sequence_bench(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
