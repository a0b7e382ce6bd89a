"""Benchmark: nAIR setup + solve to 1e-10 relative residual on one GB300.

A step is one pass of the whole hot path on one synthetic problem that is
already resident in HBM: the nAIR setup (diagonal-block inverses, strength,
C/F splitting, Neumann Delta, R, P, K = R A P on every level) followed by the
FGMRES solve preconditioned by V-cycles, to ||b - A x|| / ||b|| <= 1e-10.
The headline workload is the largest one that fits one GPU: the P3 DG
transport problem on a 512 x 512 x 2 jittered mesh with rotating flow and
log-normal absorption (5,242,880 unknowns, FP64).  value = unknowns / (setup +
solve time) in MDOF/s, summed over ranks, from the mean step time of the timed
steps (their median is reported beside it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nair|reference]
                    [--workload C5] [--precision fp64|mixed] [--variant-steps V]

With N > 1 (torchrun) every rank solves its own replica of the problem on its
own GPU with no communication on the data path (the solve does not shard).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import dgtransport  # noqa: E402

WORKLOADS = {
    "C1": "P1 DG, 32x32x2 mesh, constant flow (6144 DOFs), FP64",
    "C2": "P2 DG, 256x256x2 mesh, rotating flow, log-normal sigma_t (786432 DOFs), FP64",
    "C3": "P6 DG, 128x128x2 jittered mesh, constant flow (917504 DOFs)",
    "C5": "P3 DG, 512x512x2 jittered mesh, rotating flow, log-normal sigma_t (5242880 DOFs)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nair", choices=["nair", "reference"])
    ap.add_argument("--workload", default="C5", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--variant-steps", type=int, default=3,
                    help="timed steps of each variant (after one warm-up)")
    ap.add_argument("--neumann-degree", type=int, default=0,
                    help="profiling aid: this Neumann degree instead of the workload's")
    ap.add_argument("--mesh", type=int, default=0,
                    help="profiling aid: the workload on an N x N x 2 mesh instead of its own")
    ap.add_argument("--vcycles", type=int, default=0,
                    help="profiling aid: build the hierarchy (no CUDA graph) and apply this many "
                         "V-cycles to the right-hand side instead of benchmarking")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(workload, mesh=0):
    return dgtransport.make_problem(workload, N=mesh or None)


def oracle_sample(workload):
    """Mesh size of the bounded oracle sample: the same configuration on a mesh
    whose setup + solve takes a few seconds on the host cores."""
    cfg = dgtransport.CONFIGS[workload]
    dofs_per_cell = 2 * (cfg["p"] + 1) * (cfg["p"] + 2) // 2
    Ns = cfg["N"]
    while Ns > 16 and Ns * Ns * dofs_per_cell > 200_000:
        Ns //= 2
    return Ns


def _host_threads():
    return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, built with OpenMP (rows in parallel) and
    run on all host cores, on a bounded sample of the workload."""
    if world > 1 and rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle
    oracle.build()
    path = oracle.build_omp()
    Ns = oracle_sample(args.workload)
    P = dgtransport.make_problem(args.workload, N=Ns)
    k = P["neumann_degree"]
    times = []
    with oracle.use_library(path):
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            H = oracle.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=k)
            r = H.solve(P["rhs"])
            t1 = time.perf_counter()
            del H
            if it >= args.warmup:
                times.append(t1 - t0)
    tot = sum(times)
    value = P["n"] * len(times) / tot / 1e6
    cores = _host_threads()
    sample = (f"{args.workload} configuration on a {Ns}x{Ns}x2 mesh ({P['n']} DOFs), setup+solve, "
              f"{r['iterations']} iterations, OpenMP build on {cores} host threads")
    line = {"impl": "reference", "metric": "nAIR setup+solve MDOF/s to 1e-10 rel. residual",
            "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "sample_dofs": P["n"]},
            "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Nominal FP64 rate of one GB300 (2 FMA per clock per SM x 152 SMs x 2.07 GHz),
# used only when the live probe (nair_fp64_peak) fails.
FP64_NOMINAL_TFLOPS = 1.25

# DRAM traffic of the block-Jacobi sweep kernels per launch (dram__bytes_read.sum
# + dram__bytes_write.sum from one ncu capture, averaged over the sweeps of one
# V-cycle), by (workload, Neumann degree): (captured bytes per launch, algorithmic bytes per
# launch of the captured case, the profile that records it).  The capture may be
# of a smaller mesh of the same configuration; it is scaled to the measured
# workload by the ratio of algorithmic bytes per launch.  A workload is left out
# whenever the kernels have changed since its capture.
SWEEP_TRAFFIC = {
    ("C5", 6): (14.413e6, 10.5514e6,
                "profiles/sweep_traffic_C5.md: 256x256x2 mesh, degree 6, 80 sweeps of one V-cycle, "
                "scaled by algorithmic bytes per launch"),
}


def f_sweep_rows(rows, ci, cf, off, f_sweeps):
    """Rows updated by each F sweep of a cycle from a zero iterate: all F rows,
    then only the F rows with an off-diagonal F coupling to a row updated by the
    previous sweep (the C values do not change during the F sweeps, so any
    other row would recompute its previous value).  Boolean masks over rows."""
    F = cf == 0
    ff = off & F[rows] & F[ci]
    masks = [F]
    for _ in range(1, f_sweeps):
        dep = np.zeros_like(F)
        np.logical_or.at(dep, rows[ff], masks[-1][ci[ff]])
        masks.append(dep & F)
    return masks



def sweep_work(S, nlev, b, f_sweeps, c_sweeps=1, split=False, ymode=False, forms=None):
    """Algorithmic work of every block-Jacobi sweep of a cycle from a zero
    iterate, {(level, k): (flops, bytes)} for sweep k (F sweeps first).

    A sweep updates rows of one class: x_i = D_ii^{-1} (f_i - sum_{j != i} A_ij x_j),
    one FMA per exact nonzero of their off-diagonal blocks and b^2 FMAs per row
    for D^{-1}.  Its bytes: those nonzeros (8 B) and block column indices (4 B),
    the rows' D^{-1} blocks and right-hand side, one read of each distinct x
    block the rows reference, the write of the rows, and for every row of the
    other class that the output buffer lacks, a read and a write.  The first F
    sweep also writes its rows and copies into the second buffer.  F sweeps
    after the first update the rows of `f_sweep_rows`; they copy the rows the
    previous sweep updated that they do not, and the first C sweep copies those
    of the last F sweep.

    Level 0 with column-compressed coupling blocks (W of b columns) sweeps with
    the couplings scaled in advance, x_i = g_i - sum_j (D_ii^{-1} A_ij) x_j with
    g = D^{-1} f: b W FMAs per coupling block and no D^{-1} apply.

    With split (levels >= 1 in the scalar-row form), the first F sweep
    also writes h = f - A_FC x_C for its rows, and the later F sweeps, during
    which x_C does not change, read h and sum only the F-column couplings.

    With ymode as well (one C sweep), those levels' F sweeps iterate on
    y_F = D_FF x_F: no F sweep reads or applies D^{-1}; the later ones sum the
    right-scaled couplings A_ij D_jj^{-1}, whose nonzero rows are full (b
    nonzeros each); the C sweep takes the same scaled blocks for its F columns
    and converts every F row, x_F = D_FF^{-1} y_F (b^2 FMAs, the D^{-1} block
    and y read, x written).

    forms (the library's nair_sweep_forms per level, when given) replaces
    split and ymode level by level: split where a level takes the scalar-row
    form (2 or 3), ymode where its F sweeps run in y (3)."""
    work = {}
    for l in range(nlev):
        lev = S.level(l)
        if lev["coarsest"]:
            continue
        rp, ci, vals, cf = lev["row_ptr"], lev["col"], lev["vals"], lev["cf"]
        nnz_block = np.count_nonzero(vals.reshape(len(vals), -1), axis=1)
        nzr_block = np.count_nonzero(np.any(vals != 0, axis=2), axis=1)
        rows = np.repeat(np.arange(lev["E"]), np.diff(rp))
        off = ci != rows
        W = l0_width(vals[off], b) if l == 0 else 0
        short = 2 <= f_sweeps <= 8
        fm = f_sweep_rows(rows, ci, cf, off, f_sweeps if short else 1)
        C = cf == 1
        for k in range(f_sweeps + c_sweeps):
            dual = 1
            if k < f_sweeps:
                upd = fm[k] if short else fm[0]
                if k == 0:
                    copy, dual = C, 2 if short else 1
                else:
                    copy = (fm[k - 1] & ~fm[k]) if (short and k >= 2) else np.zeros_like(C)
            else:
                upd = C
                if k > f_sweeps:
                    copy = np.zeros_like(C)
                else:
                    copy = fm[f_sweeps - 1] if short else (cf == 0)
            sel = upd[rows] & off
            lsplit = (forms[l] in (2, 3)) if forms is not None else split
            fpart = lsplit and l >= 1 and short and 1 <= k < f_sweeps
            ylev = ((forms[l] == 3) if forms is not None else (ymode and split)) and l >= 1 and short \
                and c_sweeps == 1
            if fpart:  # later F sweeps: the F-column couplings only
                sel = sel & (cf[ci] == 0)
            if ylev and k == f_sweeps:  # the C sweep converts every F row
                copy = cf == 0
            nrow, ncopy = int(upd.sum()), int(copy.sum())
            nblk = int(sel.sum())
            xcols = len(np.unique(ci[sel]))
            if W:
                flops = 2.0 * nblk * b * W
                byts = 8.0 * nblk * b * W + 4.0 * nblk + 8.0 * nrow * b
            elif ylev:
                scaled = sel & (cf[ci] == 0) if k >= 1 else np.zeros_like(sel)
                nnz = int(nnz_block[sel & ~scaled].sum()) + b * int(nzr_block[scaled].sum())
                if k < f_sweeps:
                    flops = 2.0 * nnz
                    byts = 8.0 * nnz + 4.0 * nblk + 8.0 * nrow * b
                else:
                    flops = 2.0 * (nnz + (nrow + ncopy) * b * b)
                    byts = 8.0 * nnz + 4.0 * nblk + 8.0 * nrow * b * (b + 1) + 8.0 * ncopy * b * b
            else:
                nnz = int(nnz_block[sel].sum())
                flops = 2.0 * (nnz + nrow * b * b)
                byts = 8.0 * nnz + 4.0 * nblk + 8.0 * nrow * b * (b + 1)
            byts += 8.0 * b * xcols + 8.0 * b * (nrow + ncopy) * dual + 8.0 * b * ncopy
            if lsplit and l >= 1 and short and k == 0:  # h written
                byts += 8.0 * b * nrow
            if nrow or ncopy:
                work[(l, k)] = (flops, byts)
    return work


# (b, W) pairs with a level-0 column-compressed kernel (P1 to P6 DG blocks)
L0_WIDTHS = {3: 2, 6: 3, 10: 4, 15: 5, 21: 6, 28: 7}


def l0_width(offblocks, b):
    """W of the level-0 column compression (0 when the library does not compress):
    the largest number of nonzero columns of an off-diagonal block, raised to
    the width the kernels provide."""
    if b not in L0_WIDTHS or len(offblocks) == 0:
        return 0
    w = int(np.count_nonzero(np.any(offblocks != 0, axis=1), axis=1).max())
    return L0_WIDTHS[b] if max(w, 1) <= L0_WIDTHS[b] else 0


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json next to
    this file), else the earlier single measurement used as the fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def roofline(nair, params, rp, ci, v, sweep_ms, fp64_peak, workload):
    """Roofline of the dominant kernel, the block-Jacobi sweep (all levels).

    sweep_ms maps (level, sweep k of the cycle) to (sweeps, total ms) stamped on
    the device in untimed steps run right after the timed ones; the algorithmic
    work of each sweep comes from the hierarchy (rebuilt once, untimed, to read
    its level sizes).  FP64 sweeps are bound by the FP64 pipe (fp64_peak: the
    live FMA-throughput probe, TFLOP/s, and its source); FP32 sweeps by HBM."""
    S = nair.NairSolver(rp, ci, v, **params)
    fp64 = params.get("precision", "fp64") == "fp64"
    work = sweep_work(S, S.num_levels(), S.b, S.f_sweeps, max(S.params.c_sweeps, 0),
                      forms=S.sweep_forms())
    S.close()
    peak, peak_src = fp64_peak
    fl = by = t = 0.0
    launches = 0
    per_level = {}
    for (l, k), (n, ms) in sweep_ms.items():
        if (l, k) not in work:
            continue
        flops, byts = work[(l, k)]
        fl += flops * n
        by += byts * n
        t += ms * 1e-3
        launches += n
        a = per_level.setdefault(l, [0.0, 0.0, 0.0, 0])
        a[0] += flops * n
        a[1] += byts * n
        a[2] += ms * 1e-3
        a[3] += n
    hbm_peak, hbm_src = hbm_peak_gbs()
    by_level = []
    for l in sorted(per_level):
        lf, lb, lt, ln = per_level[l]
        if lt:
            by_level.append({"level": l, "sweeps": ln, "us_per_sweep": round(1e6 * lt / ln, 2),
                             "tflops": round(lf / lt / 1e12, 4), "frac_fp64": round(lf / lt / 1e12 / peak, 3),
                             "gbs": round(lb / lt / 1e9, 1), "frac_hbm": round(lb / lt / 1e9 / hbm_peak, 3)})
    tflops = fl / t / 1e12 if t else 0.0
    gbs = by / t / 1e9 if t else 0.0
    traffic = SWEEP_TRAFFIC.get((workload, params.get("neumann_degree"))) if fp64 else None
    alg = by / launches if launches else None
    if traffic and alg:
        traffic = (traffic[0] * alg / traffic[1], traffic[2])
    else:
        traffic = None
    out = {"bound": "alu" if fp64 else "hbm",
           "achieved": tflops if fp64 else gbs, "peak": peak if fp64 else hbm_peak,
           "unit": "TFLOP/s" if fp64 else "GB/s",
           "frac": (tflops / peak) if fp64 else (gbs / hbm_peak),
           "peak_source": (peak_src if fp64 else f"{hbm_src}: MEASURED_PEAKS.json hbm_gbs"),
           "traffic": traffic[0] if traffic else None,
           "traffic_source": traffic[1] if traffic else "no capture of the current kernels on this workload",
           "algorithmic_bytes_per_launch": by / launches if launches else None,
           "kernel": "block-Jacobi sweep: k_rowop, k_rowop_l0, k_scalar_rows (all levels)",
           "launches_per_step": None, "launches_stamped": launches,
           "kernel_ms_stamped": 1e3 * t,
           "tflops_achieved": tflops, "fp64_peak_tflops": peak,
           "hbm_achieved_gbs": gbs, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
           "by_level": by_level,
           "how": "device-clock stamps (first thread block past the dependency wait to last "
                  "thread block done) on every sweep, in untimed steps after the timed ones"}
    return out


def aggregate_ranks(total_ms, steps, dofs, world, device):
    """Whole-job throughput of replicated solves: the slowest rank's time (max over
    ranks) for `steps` steps, and MDOF/s = world * dofs / time per step."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item()) / steps
    return ms, world * dofs / (ms * 1e-3) / 1e6


def timed_steps(fn, steps, flush, stream):
    """Device time (CUDA events on the launching stream) of `steps` calls of fn,
    with an L2 flush before each call outside the timed events."""
    import torch
    total = 0.0
    out = None
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps, out


def conv_factor(rep):
    """Average convergence factor per iteration from the residual history."""
    h = rep["history"]
    return float((h[-1] / h[0]) ** (1.0 / max(1, rep["iterations"]))) if len(h) > 1 else 0.0


def measure_second_workload(nair, flush, stream, steps, device):
    """The paper's non-constant flows b1, b2, b3 (one system each) and the angle
    sweep: eight constant directions solved one after another and as one
    concurrent batch (a host thread and a stream per direction)."""
    import torch
    res = {}
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    for name in ("F1", "F2", "F3"):
        Pf = dgtransport.make_problem(name)
        args = (dev(Pf["row_ptr"]), dev(Pf["col"]), dev(Pf["vals"]))
        bf = dev(Pf["rhs"])

        def ff(args=args, bf=bf, k=Pf["neumann_degree"]):
            S = nair.NairSolver(*args, neumann_degree=k)
            xx, rep = S.solve(bf)
            S.close()
            return xx, rep
        ff()
        ms, (xx, rep) = timed_steps(ff, steps, flush, stream)
        res[f"flow_{name}_fp64"] = {"dofs": Pf["n"], "ms_per_step": ms, "mdof_s": Pf["n"] / (ms * 1e-3) / 1e6,
                                    "setup_ms": rep["setup_ms"], "solve_ms": rep["solve_ms"],
                                    "iterations": rep["iterations"], "rho": conv_factor(rep),
                                    "rel_res": rep["rel_res"]}
    angles = dgtransport.sweep_angles(8)
    probs = [dgtransport.make_problem("D", theta=t) for t in angles]
    systems = [(dev(Pd["row_ptr"]), dev(Pd["col"]), dev(Pd["vals"])) for Pd in probs]
    rhs = [dev(Pd["rhs"]) for Pd in probs]
    k = probs[0]["neumann_degree"]
    total = sum(Pd["n"] for Pd in probs)

    def seq():
        reps = []
        for sy, r in zip(systems, rhs):
            S = nair.NairSolver(*sy, neumann_degree=k)
            reps.append(S.solve(r)[1])
            S.close()
        return reps

    def bat():
        solvers = nair.setup_batch(systems, neumann_degree=k)
        _, reps = nair.solve_batch(solvers, rhs)
        for S in solvers:
            S.close()
        return reps
    for label, fn in (("sweep8_sequential_fp64", seq), ("sweep8_batched_fp64", bat)):
        fn()
        ms, reps = timed_steps(fn, steps, flush, stream)
        res[label] = {"directions": len(probs), "dofs_total": total, "ms_per_step": ms,
                      "mdof_s": total / (ms * 1e-3) / 1e6,
                      "theta": [round(t, 4) for t in angles],
                      "iterations": [r["iterations"] for r in reps],
                      "rho": [round(conv_factor(r), 4) for r in reps]}
    return res


def measure_variants(nair, params, rp, ci, v, bvec, P, x64, flush, stream, steps):
    """The mixed-precision form and the adjoint (forward + A^T solve) timed beside
    the FP64 solver on the same workload and tolerance, the F-cycle and Neumann
    degree 3 of the scaling study, scalar nAIR, the C2 workload, and the second
    workload (the paper's flows and a batched angle sweep)."""
    import torch
    dev = bvec.device
    n = P["n"]
    w = torch.from_numpy(dgtransport.functional_weights(n)).to(dev)
    mass = torch.from_numpy(np.ascontiguousarray(P["mass"])).to(dev)
    res = {}
    xref = x64.clone()

    def run(extra, adjoint=False, mode="transposed"):
        def f():
            S = nair.NairSolver(rp, ci, v, **dict(params, **extra, adjoint_mode=mode))
            xx, rep = S.solve(bvec)
            out = (xx, rep)
            if adjoint:
                lam, repa = S.adjoint_solve(w)
                out = (xx, rep, lam, repa)
            S.close()
            return out
        return f

    def timed(fn):
        fn()
        return timed_steps(fn, steps, flush, stream)

    for label, extra in (("forward_mixed", dict(precision="mixed")),
                         # Neumann degrees 2 to 4 and the F-cycle of the scaling study (Sec. 6)
                         ("forward_vcycle_k2_fp64", dict(neumann_degree=2)),
                         ("forward_vcycle_k3_fp64", dict(neumann_degree=3)),
                         ("forward_vcycle_k3_mixed", dict(neumann_degree=3, precision="mixed")),
                         ("forward_vcycle_k4_fp64", dict(neumann_degree=4)),
                         ("forward_vcycle_k5_fp64", dict(neumann_degree=5)),
                         ("forward_vcycle_k6_fp64", dict(neumann_degree=6)),
                         ("forward_vcycle_k7_fp64", dict(neumann_degree=7)),
                         ("forward_vcycle_k8_fp64", dict(neumann_degree=8)),
                         ("forward_fcycle_k4_fp64", dict(neumann_degree=4, cycle_type="F")),
                         ("forward_fcycle_k3_fp64", dict(neumann_degree=3, cycle_type="F")),
                         ("forward_fcycle_k3_mixed", dict(neumann_degree=3, cycle_type="F", precision="mixed")),
                         # scalar nAIR (block-diagonal scaling, coarsening by degree of freedom)
                         ("forward_scalar_fp64", dict(scalar=1)),
                         ("forward_scalar_mixed", dict(scalar=1, precision="mixed"))):
        ms, (xx, rep) = timed(run(extra))
        res[label] = {"ms_per_step": ms, "mdof_s": n / (ms * 1e-3) / 1e6, "setup_ms": rep["setup_ms"],
                      "solve_ms": rep["solve_ms"], "iterations": rep["iterations"], "rel_res": rep["rel_res"],
                      "cycle_complexity": rep["cycle_complexity"], "op_complexity": rep["op_complexity"],
                      "rel_diff_vs_fp64": float((xx - xref).norm() / xref.norm())}
    # the adjoint through the transposed forward hierarchy (default), also in
    # mixed precision, and by a second hierarchy built on A^T; gradients of
    # J = w . x (Eq. transport: dJ/dq = M^T lambda, dJ/dsigma_e = -lambda_e^T M_e x_e)
    ref = None
    for label, extra, mode in (("forward_adjoint_fp64", {}, "transposed"),
                               ("forward_adjoint_mixed", dict(precision="mixed"), "transposed"),
                               ("forward_adjoint_rebuild_fp64", {}, "rebuild")):
        ms, (xx, rep, lam, repa) = timed(run(extra, adjoint=True, mode=mode))
        gs, gq = nair.gradients(mass, lam, xx)
        if ref is None:
            ref = (lam.clone(), gs.clone(), gq.clone())
        res[label] = {
            "ms_per_step": ms, "setup_ms": rep["setup_ms"], "solve_ms": rep["solve_ms"],
            "iterations": rep["iterations"], "adjoint_setup_ms": repa["setup_ms"],
            "adjoint_solve_ms": repa["solve_ms"], "adjoint_iterations": repa["iterations"],
            "adjoint_rel_res": repa["rel_res"],
            "lambda_rel_diff_vs_fp64": float((lam - ref[0]).norm() / ref[0].norm()),
            "grad_sigma_rel_diff_vs_fp64": float((gs - ref[1]).norm() / ref[1].norm()),
            "grad_q_rel_diff_vs_fp64": float((gq - ref[2]).norm() / ref[2].norm())}
    # the C2 workload (P2 DG, 256 x 256 x 2, rotating flow), FP64 and mixed
    P2 = dgtransport.make_problem("C2")
    c2 = [torch.from_numpy(np.ascontiguousarray(P2[k2])).to(dev) for k2 in ("row_ptr", "col", "vals", "rhs")]
    for prec in ("fp64", "mixed"):
        def f2(prec=prec):
            S = nair.NairSolver(*c2[:3], neumann_degree=P2["neumann_degree"], precision=prec)
            xx, rep = S.solve(c2[3])
            S.close()
            return xx, rep
        ms, (xx, rep) = timed(f2)
        res[f"C2_forward_{prec}"] = {"dofs": P2["n"], "ms_per_step": ms, "mdof_s": P2["n"] / (ms * 1e-3) / 1e6,
                                     "setup_ms": rep["setup_ms"], "solve_ms": rep["solve_ms"],
                                     "iterations": rep["iterations"], "rel_res": rep["rel_res"]}
    res.update(measure_second_workload(nair, flush, stream, steps, dev))
    return res


def cpu_baseline(workload):
    """The oracle as it stands on a bounded sample of the workload (the same
    configuration on a coarser mesh): one setup + solve of its OpenMP build on
    all host threads (the reported value), and of its single-threaded build."""
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle
    oracle.build()
    path = oracle.build_omp()
    Ns = min(dgtransport.CONFIGS[workload]["N"], 2 * oracle_sample(workload))
    P = dgtransport.make_problem(workload, N=Ns)
    k = P["neumann_degree"]

    def once():
        t0 = time.perf_counter()
        H = oracle.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=k)
        r = H.solve(P["rhs"])
        del H
        return time.perf_counter() - t0, r["iterations"]

    with oracle.use_library(path):
        t_all, its = once()
    t_one, _ = once()
    cores = _host_threads()
    return {"value": P["n"] / t_all / 1e6, "unit": "MDOF/s", "cores": cores, "kind": "oracle",
            "sample": f"one setup+solve of the {workload} configuration on a {Ns}x{Ns}x2 mesh "
                      f"({P['n']} DOFs, {its} iterations): OpenMP build on {cores} host threads "
                      f"{t_all:.1f} s, single-threaded build {t_one:.1f} s",
            "single_thread": {"value": P["n"] / t_one / 1e6, "unit": "MDOF/s", "cores": 1}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1704_05001_gb300 as nair
    from paper_1704_05001_gb300 import build as nbuild
    nbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    P = make_inputs(args.workload, args.mesh)
    k = args.neumann_degree or P["neumann_degree"]
    params = dict(neumann_degree=k, precision=args.precision)
    if args.vcycles:
        S = nair.NairSolver(torch.from_numpy(P["row_ptr"]).to(dev), torch.from_numpy(P["col"]).to(dev),
                            torch.from_numpy(P["vals"]).to(dev), use_graphs=0, **params)
        f = torch.from_numpy(P["rhs"]).to(dev)
        for _ in range(args.vcycles):
            S.vcycle(f)
        torch.cuda.synchronize()
        print(json.dumps({"vcycles": args.vcycles, "levels": S.num_levels(),
                          "elements": [S.sizes(l)["E"] for l in range(S.num_levels())]}))
        return
    rp = torch.from_numpy(P["row_ptr"]).to(dev)
    ci = torch.from_numpy(P["col"]).to(dev)
    v = torch.from_numpy(P["vals"]).to(dev)
    bvec = torch.from_numpy(P["rhs"]).to(dev)
    x = torch.zeros_like(bvec)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    fp64_peak = (FP64_NOMINAL_TFLOPS, "nominal (probe failed)")
    if not args.no_extras:
        try:
            tf, mhz = nair.fp64_peak()
            fp64_peak = (tf, f"measured live by nair_fp64_peak (FP64 FMA-chain kernel, SM clock {mhz:.0f} MHz)")
        except Exception as e:  # noqa: BLE001 - a failed probe leaves the nominal figure, said so
            fp64_peak = (FP64_NOMINAL_TFLOPS, f"nominal (probe failed: {e})")

    def step(stamps=None):
        s = nair.NairSolver(rp, ci, v, **dict(params, sweep_timing=1 if stamps is not None else 0))
        x.zero_()
        _, rep = s.solve(bvec, x)
        if stamps is not None:
            for key, (n, ms) in s.sweep_site_timing().items():
                c, m = stamps.get(key, (0, 0.0))
                stamps[key] = (c + n, m + ms)
        s.close()
        return rep

    for _ in range(args.warmup):
        rep = step()
    launches0 = nair.kernel_launches()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = []
    setup_ms = solve_ms = 0.0
    reps = []
    for _ in range(args.steps):
        flush.fill_(1.0)   # L2 flush between timed steps (outside the events)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        setup_ms += rep["setup_ms"]
        solve_ms += rep["solve_ms"]
        reps.append(rep)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = (nair.kernel_launches() - launches0) // max(1, args.steps)
    ms, value = aggregate_ranks(sum(step_ms), args.steps, P["n"], world, dev)

    # device-clock stamps of every sweep, in separate untimed steps
    sweep_ms = {}
    if not args.no_extras:
        for _ in range(min(args.steps, 3)):
            step(sweep_ms)

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_extras:
        hp = {k2: torch.from_numpy(np.ascontiguousarray(P[k2])).pin_memory()
              for k2 in ("row_ptr", "col", "vals", "rhs")}
        xh = torch.empty(P["n"], dtype=torch.float64).pin_memory()
        h2d = sum(t2.numel() * t2.element_size() for t2 in hp.values())
        d2h = xh.numel() * xh.element_size()

        h2d_ms = [0.0]

        def e2e_step(timed=False):
            if timed:
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
            drp = hp["row_ptr"].to(dev, non_blocking=True)
            dci = hp["col"].to(dev, non_blocking=True)
            dv = hp["vals"].to(dev, non_blocking=True)
            db = hp["rhs"].to(dev, non_blocking=True)
            if timed:
                c1.record(stream)
            s = nair.NairSolver(drp, dci, dv, **params)
            xx, _ = s.solve(db)
            xh.copy_(xx, non_blocking=True)
            s.close()
            torch.cuda.synchronize()
            if timed:
                h2d_ms[0] += c0.elapsed_time(c1)

        e2e_step()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step(timed=True)
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e = {"value": world * P["n"] / (e2e_ms / args.steps * 1e-3) / 1e6, "unit": "MDOF/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               # the host-to-device copies alone (CUDA events around them, same steps)
               "h2d_ms_per_step": h2d_ms[0] / args.steps,
               "h2d_gbs": h2d / (h2d_ms[0] / args.steps * 1e-3) / 1e9 if h2d_ms[0] > 0 else None}

    variants = None
    if not args.no_extras:
        variants = measure_variants(nair, params, rp, ci, v, bvec, P, x, flush, stream,
                                    max(1, args.variant_steps))

    if rank != 0:
        return
    last = reps[-1]
    line = {
        "metric": "nAIR setup+solve MDOF/s to 1e-10 rel. residual",
        "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-in-f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "dofs": P["n"], "precision": args.precision,
                   "neumann_degree": k, "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "ms_per_step_median": float(np.median(step_ms)), "ms_per_step_all": [round(t, 3) for t in step_ms],
        "setup_ms": setup_ms / args.steps, "solve_ms": solve_ms / args.steps,
        "iterations": last["iterations"], "levels": last["levels"], "rel_res": last["rel_res"],
        "op_complexity": last["op_complexity"], "cycle_complexity": last["cycle_complexity"],
        "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e,
    }
    if variants:
        line["variants"] = variants
    if not args.no_extras:
        line["roofline"] = roofline(nair, params, rp, ci, v, sweep_ms, fp64_peak, args.workload)
        line["roofline"]["launches_per_step"] = line["roofline"]["launches_stamped"] // max(1, min(args.steps, 3))
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
