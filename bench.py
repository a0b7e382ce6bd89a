"""Benchmark: nAIR setup + solve to 1e-10 relative residual on one GB300.

A step is one pass of the whole hot path on one synthetic problem that is
already resident in HBM: the nAIR setup (diagonal-block inverses, strength,
C/F splitting, Neumann Delta, R, P, K = R A P on every level) followed by the
FGMRES solve preconditioned by V-cycles, to ||b - A x|| / ||b|| <= 1e-10.
The headline workload is the P2 DG transport problem on a 256 x 256 x 2
mesh with rotating flow and log-normal absorption (786,432 unknowns, FP64).
value = unknowns / (setup + solve time) in MDOF/s, summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nair|reference]
                    [--workload C2] [--precision fp64|mixed]

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
    ap.add_argument("--workload", default="C2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-extras", action="store_true")
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


def make_inputs(workload):
    P = dgtransport.make_problem(workload)
    return P


def run_reference(args, rank, world):
    """FP64 CPU oracle (single host thread) on a bounded sample of the workload."""
    import oracle
    oracle.build()
    if rank != 0:
        return
    # bounded sample: the same configuration on a coarser mesh (setup + solve)
    cfg = dgtransport.CONFIGS[args.workload]
    Ns = max(16, cfg["N"] // 4)
    P = dgtransport.make_problem(args.workload, N=Ns)
    k = P["neumann_degree"]
    times = []
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
    sample = f"{args.workload} configuration on a {Ns}x{Ns}x2 mesh ({P['n']} DOFs), setup+solve, {r['iterations']} iterations"
    line = {"impl": "reference", "metric": "nAIR setup+solve MDOF/s to 1e-10 rel. residual",
            "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "sample_dofs": P["n"]},
            "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# FP64 pipe of one GB300: 1.25 TFLOP/s dense FP64 (nominal figure of the part; an
# FMA-throughput probe on the box measured 1.249 TFLOP/s).
FP64_PEAK_TFLOPS = 1.25

# DRAM traffic of the block-Jacobi sweep kernel from an ncu capture (bytes per
# launch, averaged over the sweeps of one C2 V-cycle: dram__bytes_read.sum +
# dram__bytes_write.sum); None whenever the kernel has changed since the capture.
JACOBI_TRAFFIC = 13.04e6


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


def sweep_work(S, nlev, b, f_sweeps, c_sweeps=1):
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
    g = D^{-1} f: b W FMAs per coupling block and no D^{-1} apply."""
    work = {}
    for l in range(nlev):
        lev = S.level(l)
        if lev["coarsest"]:
            continue
        rp, ci, vals, cf = lev["row_ptr"], lev["col"], lev["vals"], lev["cf"]
        nnz_block = np.count_nonzero(vals.reshape(len(vals), -1), axis=1)
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
            nrow, ncopy = int(upd.sum()), int(copy.sum())
            nblk = int(sel.sum())
            xcols = len(np.unique(ci[sel]))
            if W:
                flops = 2.0 * nblk * b * W
                byts = 8.0 * nblk * b * W + 4.0 * nblk + 8.0 * nrow * b
            else:
                nnz = int(nnz_block[sel].sum())
                flops = 2.0 * (nnz + nrow * b * b)
                byts = 8.0 * nnz + 4.0 * nblk + 8.0 * nrow * b * (b + 1)
            byts += 8.0 * b * xcols + 8.0 * b * (nrow + ncopy) * dual + 8.0 * b * ncopy
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


def roofline(nair, params, rp, ci, v, sweep_ms):
    """Roofline of the dominant kernel, the block-Jacobi sweep (all levels).

    sweep_ms maps (level, sweep k of the cycle) to (sweeps, total ms) stamped on
    the device inside the timed steps; the algorithmic work of each sweep comes
    from the hierarchy (rebuilt once, untimed, to read its level sizes)."""
    S = nair.NairSolver(rp, ci, v, **params)
    work = sweep_work(S, S.num_levels(), S.b, S.f_sweeps, max(S.params.c_sweeps, 0))
    S.close()
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
    achieved = fl / t / 1e12 if t else 0.0
    hbm_peak, hbm_src = hbm_peak_gbs()
    by_level = []
    for l in sorted(per_level):
        lf, lb, lt, ln = per_level[l]
        if lt:
            by_level.append({"level": l, "sweeps": ln, "us_per_sweep": round(1e6 * lt / ln, 2),
                             "tflops": round(lf / lt / 1e12, 4), "frac_fp64": round(lf / lt / 1e12 / FP64_PEAK_TFLOPS, 3),
                             "gbs": round(lb / lt / 1e9, 1), "frac_hbm": round(lb / lt / 1e9 / hbm_peak, 3)})
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": JACOBI_TRAFFIC,
            "algorithmic_bytes_per_launch": by / launches if launches else None,
            "kernel": "block-Jacobi sweep: k_rowop, k_rowop_l0, k_sweep_rows (FP64, all levels)",
            "launches_per_step": None, "launches_timed": launches,
            "kernel_ms_timed": 1e3 * t,
            "hbm_achieved_gbs": by / t / 1e9 if t else 0.0,
            "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
            "by_level": by_level,
            "how": "device-clock stamps (first thread block past the dependency wait to last "
                   "thread block done) on every sweep inside the timed steps"}


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
    the FP64 solver on the same workload and tolerance."""
    import torch
    n = P["n"]
    w = torch.from_numpy(dgtransport.functional_weights(n)).to(bvec.device)
    res = {}
    xref = x64.clone()

    def fwd(prec):
        def f():
            S = nair.NairSolver(rp, ci, v, **dict(params, precision=prec))
            xx, rep = S.solve(bvec)
            S.close()
            return xx, rep
        return f

    def fwd_adj(prec, mode="transposed"):
        def f():
            S = nair.NairSolver(rp, ci, v, **dict(params, precision=prec, adjoint_mode=mode))
            xx, rep = S.solve(bvec)
            lam, repa = S.adjoint_solve(w)
            S.close()
            return xx, lam, rep, repa
        return f

    for prec in ("fp64", "mixed"):
        fwd(prec)()
        ms, (xx, rep) = timed_steps(fwd(prec), steps, flush, stream)
        res[f"forward_{prec}"] = {"ms_per_step": ms, "mdof_s": n / (ms * 1e-3) / 1e6,
                                 "setup_ms": rep["setup_ms"], "solve_ms": rep["solve_ms"],
                                 "iterations": rep["iterations"], "rel_res": rep["rel_res"],
                                 "rel_diff_vs_fp64": float((xx - xref).norm() / xref.norm())}
    # the F-cycle and Neumann degree 3 of the scaling study (Sec. 6), and scalar nAIR
    for label, extra in (("forward_vcycle_k3_fp64", dict(neumann_degree=3)),
                         ("forward_fcycle_k3_fp64", dict(neumann_degree=3, cycle_type="F")),
                         ("forward_fcycle_k3_mixed", dict(neumann_degree=3, cycle_type="F", precision="mixed")),
                         # scalar nAIR (block-diagonal scaling, coarsening by degree of freedom)
                         ("forward_scalar_fp64", dict(scalar=1)),
                         ("forward_scalar_mixed", dict(scalar=1, precision="mixed"))):
        def fk(extra=extra):
            S = nair.NairSolver(rp, ci, v, **dict(params, **extra))
            xx, rep = S.solve(bvec)
            S.close()
            return xx, rep
        fk()
        ms, (xx, rep) = timed_steps(fk, steps, flush, stream)
        res[label] = {"ms_per_step": ms, "mdof_s": n / (ms * 1e-3) / 1e6, "setup_ms": rep["setup_ms"],
                      "solve_ms": rep["solve_ms"], "iterations": rep["iterations"], "rel_res": rep["rel_res"],
                      "cycle_complexity": rep["cycle_complexity"], "op_complexity": rep["op_complexity"],
                      "rel_diff_vs_fp64": float((xx - xref).norm() / xref.norm())}
    res.update(measure_second_workload(nair, flush, stream, steps, bvec.device))
    lam_ref = None
    # the adjoint through the transposed forward hierarchy (default), and by a
    # second hierarchy built on A^T
    for prec, mode, label in (("fp64", "transposed", "forward_adjoint_fp64"),
                              ("mixed", "transposed", "forward_adjoint_mixed"),
                              ("fp64", "rebuild", "forward_adjoint_rebuild_fp64")):
        fwd_adj(prec, mode)()
        ms, (xx, lam, rep, repa) = timed_steps(fwd_adj(prec, mode), steps, flush, stream)
        if lam_ref is None:
            lam_ref = lam.clone()
        res[label] = {
            "ms_per_step": ms, "adjoint_setup_ms": repa["setup_ms"], "adjoint_solve_ms": repa["solve_ms"],
            "adjoint_iterations": repa["iterations"], "adjoint_rel_res": repa["rel_res"],
            "lambda_rel_diff_vs_fp64": float((lam - lam_ref).norm() / lam_ref.norm())}
    return res


def cpu_baseline(workload):
    """The oracle as it stands, one host thread, on a bounded sample (~10-30 s)."""
    import oracle
    oracle.build()
    cfg = dgtransport.CONFIGS[workload]
    # the full workload when it is small enough for ~10-30 s of one host thread
    Ns = cfg["N"] if cfg["N"] * cfg["N"] * (cfg["p"] + 1) ** 2 <= 256 * 256 * 9 else cfg["N"] // 2
    P = dgtransport.make_problem(workload, N=Ns)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=P["neumann_degree"])
    r = H.solve(P["rhs"])
    t = time.perf_counter() - t0
    return {"value": P["n"] / t / 1e6, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
            "sample": f"one setup+solve of the {workload} configuration on a {Ns}x{Ns}x2 mesh "
                      f"({P['n']} DOFs, {r['iterations']} iterations, {t:.1f} s)"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
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

    P = make_inputs(args.workload)
    k = P["neumann_degree"]
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

    sweep_ms = {}
    timed = {"on": False}

    def step():
        s = nair.NairSolver(rp, ci, v, **dict(params, sweep_timing=1 if timed["on"] else 0))
        x.zero_()
        _, rep = s.solve(bvec, x)
        if timed["on"]:
            for key, (n, ms) in s.sweep_site_timing().items():
                c, m = sweep_ms.get(key, (0, 0.0))
                sweep_ms[key] = (c + n, m + ms)
        s.close()
        return rep

    for _ in range(args.warmup):
        rep = step()
    launches0 = nair.kernel_launches()
    timed["on"] = not args.no_extras
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
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
        total_ms += e0.elapsed_time(e1)
        setup_ms += rep["setup_ms"]
        solve_ms += rep["solve_ms"]
        reps.append(rep)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    timed["on"] = False
    launches = (nair.kernel_launches() - launches0) // max(1, args.steps)
    ms, value = aggregate_ranks(total_ms, args.steps, P["n"], world, dev)

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_extras:
        hp = {k2: torch.from_numpy(np.ascontiguousarray(P[k2])).pin_memory()
              for k2 in ("row_ptr", "col", "vals", "rhs")}
        xh = torch.empty(P["n"], dtype=torch.float64).pin_memory()
        h2d = sum(t2.numel() * t2.element_size() for t2 in hp.values())
        d2h = xh.numel() * xh.element_size()

        def e2e_step():
            drp = hp["row_ptr"].to(dev, non_blocking=True)
            dci = hp["col"].to(dev, non_blocking=True)
            dv = hp["vals"].to(dev, non_blocking=True)
            db = hp["rhs"].to(dev, non_blocking=True)
            s = nair.NairSolver(drp, dci, dv, **params)
            xx, _ = s.solve(db)
            xh.copy_(xx, non_blocking=True)
            s.close()
            torch.cuda.synchronize()

        e2e_step()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e = {"value": world * P["n"] / (e2e_ms / args.steps * 1e-3) / 1e6, "unit": "MDOF/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    variants = None
    if not args.no_extras:
        variants = measure_variants(nair, params, rp, ci, v, bvec, P, x, flush, stream, args.steps)

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
        "setup_ms": setup_ms / args.steps, "solve_ms": solve_ms / args.steps,
        "iterations": last["iterations"], "levels": last["levels"], "rel_res": last["rel_res"],
        "op_complexity": last["op_complexity"], "cycle_complexity": last["cycle_complexity"],
        "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e,
    }
    if variants:
        line["variants"] = variants
    if not args.no_extras:
        line["roofline"] = roofline(nair, params, rp, ci, v, sweep_ms)
        line["roofline"]["launches_per_step"] = line["roofline"]["launches_timed"] // args.steps
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
