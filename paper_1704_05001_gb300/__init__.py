"""Python binding of the GB300 block-nAIR library (libnair.so, C ABI in include/nair.h).

nAIR is the reduction-based algebraic multigrid of arXiv 1704.05001 (Neumann
approximation to ideal restriction).  This module only marshals arguments:
every step of setup and solve runs in the library's CUDA kernels.  PyTorch
provides device memory and streams.  There is no CPU fallback: if the shared
library is missing or cannot be loaded, every call raises.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnair.so")

NAIR_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "SINGULAR_BLOCK", 3: "NOT_CONVERGED", 4: "BREAKDOWN",
          5: "OOM", 6: "CUDA", 7: "UNSUPPORTED"}
FP64, MIXED = 0, 1
ADJOINT_TRANSPOSED, ADJOINT_REBUILD = 0, 1
CYCLE_V, CYCLE_F = 0, 1

# nair_level_array
(A_ROWPTR, A_COL, A_VALS, DINV, CF, P_MAP, DELTA_ROWPTR, DELTA_COL, DELTA_VALS, R_ROWPTR, R_COL,
 R_VALS, STRONG, LAMBDA, L_ROWPTR, L_COL, L_VALS) = range(17)


class NairError(RuntimeError):
    def __init__(self, status, where, msg=""):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Bsr(ctypes.Structure):
    _fields_ = [("nb_rows", ctypes.c_int32), ("block_size", ctypes.c_int32), ("nnzb", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("strength_theta", ctypes.c_double), ("filter_tol", ctypes.c_double),
                ("filter_targets", ctypes.c_int32), ("neumann_degree", ctypes.c_int32),
                ("f_sweeps", ctypes.c_int32), ("c_sweeps", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("max_coarse", ctypes.c_int32),
                ("max_dense", ctypes.c_int32), ("cf_seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("gmres_restart", ctypes.c_int32),
                ("maxiter", ctypes.c_int32), ("tol", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("keep_setup_data", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("sweep_timing", ctypes.c_int32), ("adjoint_mode", ctypes.c_int32),
                ("cycle_type", ctypes.c_int32), ("scalar", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("levels", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("op_complexity", ctypes.c_double), ("cycle_complexity", ctypes.c_double),
                ("history", ctypes.c_void_p), ("history_cap", ctypes.c_int32),
                ("history_len", ctypes.c_int32)]


_lib = None

# every entry point of include/nair.h
EXPORTS = ["nair_default_params", "nair_setup", "nair_solve", "nair_adjoint_solve", "nair_vcycle",
           "nair_adjoint_vcycle",
           "nair_free", "nair_num_levels", "nair_level_sizes", "nair_get_level", "nair_block_inverse",
           "nair_assemble_sigma", "nair_mass_apply", "nair_gradients", "nair_kernel_launches",
           "nair_profile", "nair_profile_entry", "nair_block_inverse_noalloc", "nair_sweep_timing",
           "nair_setup_batch", "nair_solve_batch", "nair_adjoint_solve_batch", "nair_fp64_peak",
           "nair_last_error", "nair_sweep_forms"]


def lib():
    """Load libnair.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnair.so not built ({LIB_PATH}); run paper_1704_05001_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.nair_default_params.argtypes = [ctypes.POINTER(_Params)]
    L.nair_default_params.restype = None
    L.nair_setup.argtypes = [ctypes.POINTER(_Bsr), ctypes.POINTER(_Params), ctypes.POINTER(P)]
    L.nair_solve.argtypes = [P, P, P, ctypes.POINTER(_Info)]
    L.nair_adjoint_solve.argtypes = [P, P, P, ctypes.POINTER(_Info)]
    L.nair_vcycle.argtypes = [P, P, P]
    L.nair_adjoint_vcycle.argtypes = [P, P, P]
    L.nair_setup_batch.argtypes = [ctypes.POINTER(_Bsr), ctypes.POINTER(_Params), I32, ctypes.POINTER(P)]
    L.nair_solve_batch.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(P), ctypes.POINTER(P),
                                   ctypes.POINTER(_Info)]
    L.nair_adjoint_solve_batch.argtypes = L.nair_solve_batch.argtypes
    L.nair_free.argtypes = [P]
    L.nair_free.restype = None
    L.nair_num_levels.argtypes = [P, I32, ctypes.POINTER(I32)]
    L.nair_level_sizes.argtypes = [P, I32, I32, P]
    L.nair_sweep_forms.argtypes = [P, I32, I32, P]
    L.nair_get_level.argtypes = [P, I32, I32, I32, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.nair_block_inverse.argtypes = [I32, I32, P, P, P]
    L.nair_block_inverse_noalloc.argtypes = [I32, I32, P, P, P]
    L.nair_assemble_sigma.argtypes = [I32, I32, I64, P, P, P, P, P, P]
    L.nair_mass_apply.argtypes = [I32, I32, P, P, P, P]
    L.nair_gradients.argtypes = [I32, I32, P, P, P, P, P, P]
    L.nair_kernel_launches.argtypes = [ctypes.POINTER(I64)]
    L.nair_fp64_peak.argtypes = [I32, I32, ctypes.POINTER(D), ctypes.POINTER(D), P]
    L.nair_profile.argtypes = [I32]
    L.nair_sweep_timing.argtypes = [P, I32, I32, ctypes.POINTER(I64), ctypes.POINTER(D)]
    L.nair_profile_entry.argtypes = [I32, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(I64),
                                     ctypes.POINTER(D)]
    L.nair_last_error.argtypes = []
    L.nair_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "nair_default_params" and name != "nair_free" and name != "nair_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st, where):
    if st != NAIR_OK:
        raise NairError(st, where, lib().nair_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    c = ctypes.c_int64(0)
    _check(lib().nair_kernel_launches(ctypes.byref(c)), "nair_kernel_launches")
    return c.value


FP64_FMA, FP64_MMA, FP64_BOTH = 0, 1, 2


def fp64_peak(mode=FP64_FMA, iters=40000):
    """Measured FP64 throughput of the current GPU (nair_fp64_peak): fma chains
    (mode 0), FP64 tensor-core mma chains (1) or both at once (2).  Returns
    (TFLOP/s, SM clock in MHz during the measurement)."""
    t = ctypes.c_double(0)
    mhz = ctypes.c_double(0)
    _check(lib().nair_fp64_peak(mode, iters, ctypes.byref(t), ctypes.byref(mhz), _stream()), "nair_fp64_peak")
    return t.value, mhz.value


def profile(enable=True):
    """Turn per-kernel event timing on (clearing it) or off."""
    _check(lib().nair_profile(int(enable)), "nair_profile")


def profile_report():
    """{name: (timed scopes, total ms)} recorded since profile(True)."""
    out = {}
    buf = ctypes.create_string_buffer(256)
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0)
    idx = 0
    while lib().nair_profile_entry(idx, buf, 256, ctypes.byref(n), ctypes.byref(ms)) == NAIR_OK:
        out[buf.value.decode()] = (n.value, ms.value)
        idx += 1
    return out


def default_params():
    p = _Params()
    lib().nair_default_params(ctypes.byref(p))
    return p


_ENUMS = {"precision": {"fp64": FP64, "mixed": MIXED},
          "adjoint_mode": {"transposed": ADJOINT_TRANSPOSED, "rebuild": ADJOINT_REBUILD},
          "cycle_type": {"V": CYCLE_V, "F": CYCLE_F}}


def _make_params(params, stream=None):
    """nair_params from the defaults and keyword overrides; the work goes to
    ``stream`` (a torch.cuda.Stream) or to the current stream."""
    p = default_params()
    for k, v in params.items():
        if isinstance(v, str) and k in _ENUMS:
            v = _ENUMS[k][v]
        if not hasattr(p, k) or k == "stream":
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    p.stream = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _stream()
    return p


class NairSolver:
    """nAIR hierarchy on the current CUDA device (setup at construction).

    row_ptr, col: int32 CUDA tensors; vals: float64 CUDA tensor (nnzb, b, b).
    ``stream`` (a torch.cuda.Stream, default: the current stream) carries all
    of the solver's work.  Keyword arguments set fields of nair_params (strength_theta, filter_tol,
    neumann_degree, f_sweeps, c_sweeps, max_coarse, precision ("fp64" or
    "mixed"), gmres_restart, maxiter, tol, keep_setup_data, adjoint_mode
    ("transposed" or "rebuild"), cycle_type ("V" or "F"), scalar (0 or 1), ...).
    """

    def __init__(self, row_ptr, col, vals, stream=None, _handle=None, **params):
        L = lib()
        p = _make_params(params, stream)
        self.params = p
        self.b = int(vals.shape[-1])
        self.level_b = 1 if p.scalar else self.b  # block size of the hierarchy's levels
        self.f_sweeps = p.f_sweeps if p.f_sweeps > 0 else p.neumann_degree + 1
        self.E = int(row_ptr.shape[0] - 1)
        self.n = self.E * self.b
        self.device = vals.device
        self.stream = stream
        if _handle is not None:  # adopted from nair_setup_batch
            self._h = _handle
            return
        A = _Bsr(self.E, self.b, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(vals))
        h = ctypes.c_void_p()
        _check(L.nair_setup(ctypes.byref(A), ctypes.byref(p), ctypes.byref(h)), "nair_setup")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().nair_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _info(self, cap):
        info = _Info()
        hist = np.zeros(max(cap, 1))
        info.history = hist.ctypes.data_as(ctypes.c_void_p)
        info.history_cap = cap
        return info, hist

    @staticmethod
    def _report(info, hist, status):
        return dict(status=status, iterations=info.iterations, levels=info.levels,
                    rel_res=info.rel_res, setup_ms=info.setup_ms, solve_ms=info.solve_ms,
                    op_complexity=info.op_complexity, cycle_complexity=info.cycle_complexity,
                    history=hist[:min(info.history_len, len(hist))].copy())

    def _enter(self):
        # the solver's own stream waits for the inputs made on the current stream
        if self.stream is not None:
            self.stream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        if self.stream is not None:
            torch.cuda.current_stream().wait_stream(self.stream)

    def solve(self, b, x=None, check=True):
        """Solve A x = b (b: float64 CUDA tensor); returns (x, report)."""
        x = torch.zeros_like(b) if x is None else x
        info, hist = self._info(self.params.maxiter + self.params.maxiter // max(1, self.params.gmres_restart) + 4)
        self._enter()
        st = lib().nair_solve(self._h, _ptr(b), _ptr(x), ctypes.byref(info))
        self._leave()
        if check:
            _check(st, "nair_solve")
        return x, self._report(info, hist, st)

    def adjoint_solve(self, w, lam=None, check=True):
        """Solve A^T lambda = w; the first call forms the transposed operators
        (adjoint_mode "transposed") or the A^T hierarchy ("rebuild")."""
        lam = torch.zeros_like(w) if lam is None else lam
        info, hist = self._info(self.params.maxiter + self.params.maxiter // max(1, self.params.gmres_restart) + 4)
        self._enter()
        st = lib().nair_adjoint_solve(self._h, _ptr(w), _ptr(lam), ctypes.byref(info))
        self._leave()
        if check:
            _check(st, "nair_adjoint_solve")
        return lam, self._report(info, hist, st)

    def vcycle(self, f):
        x = torch.empty_like(f)
        self._enter()
        _check(lib().nair_vcycle(self._h, _ptr(f), _ptr(x)), "nair_vcycle")
        self._leave()
        return x

    def adjoint_vcycle(self, f):
        """The transposed cycle of the forward hierarchy: M^{-T} f."""
        x = torch.empty_like(f)
        self._enter()
        _check(lib().nair_adjoint_vcycle(self._h, _ptr(f), _ptr(x)), "nair_adjoint_vcycle")
        self._leave()
        return x

    def num_levels(self, adjoint=False):
        n = ctypes.c_int32(0)
        _check(lib().nair_num_levels(self._h, int(adjoint), ctypes.byref(n)), "nair_num_levels")
        return n.value

    def sweep_forms(self, transposed=False):
        """Relaxation form per level: -1 coarsest, 0 block-row kernel, 1 level-0
        column-compressed blocks, 2 packed scalar rows, 3 scalar rows with the F
        sweeps in y = D x (nair_sweep_forms)."""
        n = self.num_levels()
        out = np.zeros(max(n, 1), dtype=np.int32)
        _check(lib().nair_sweep_forms(self._h, int(transposed), n, out.ctypes.data_as(ctypes.c_void_p)),
               "nair_sweep_forms")
        return [int(v) for v in out[:n]]

    def sizes(self, level, adjoint=False):
        out = np.zeros(10, dtype=np.int64)
        _check(lib().nair_level_sizes(self._h, int(adjoint), level, out.ctypes.data_as(ctypes.c_void_p)),
               "nair_level_sizes")
        keys = ["E", "nnzb", "nC", "nF", "L_nnzb", "D_nnzb", "R_nnzb", "AP_nnzb", "coarsest", "cf_rounds"]
        return dict(zip(keys, (int(v) for v in out)))

    def _array(self, level, which, dtype, shape, adjoint):
        need = ctypes.c_size_t(0)
        _check(lib().nair_get_level(self._h, int(adjoint), level, which, None, 0, ctypes.byref(need)),
               "nair_get_level")
        out = np.zeros(need.value // np.dtype(dtype).itemsize, dtype=dtype)
        if need.value:
            _check(lib().nair_get_level(self._h, int(adjoint), level, which,
                                        out.ctypes.data_as(ctypes.c_void_p), need.value,
                                        ctypes.byref(need)), "nair_get_level")
        return out.reshape(shape) if shape is not None else out

    def sweep_timing(self):
        """{(level, "F"|"C"): (sweeps, total ms)} stamped on the device (sweep_timing=1)."""
        out = {}
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0)
        for l in range(self.num_levels()):
            for cls, nm in ((0, "F"), (1, "C")):
                _check(lib().nair_sweep_timing(self._h, l, cls, ctypes.byref(n), ctypes.byref(ms)),
                       "nair_sweep_timing")
                if n.value:
                    out[(l, nm)] = (n.value, ms.value)
        return out

    def sweep_site_timing(self):
        """{(level, k): (sweeps, total ms)} for sweep k of the cycle (F sweeps first),
        stamped on the device (sweep_timing=1)."""
        out = {}
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0)
        S = self.f_sweeps + max(self.params.c_sweeps, 0)
        for l in range(self.num_levels()):
            for k in range(S):
                _check(lib().nair_sweep_timing(self._h, l, 2 + k, ctypes.byref(n), ctypes.byref(ms)),
                       "nair_sweep_timing")
                if n.value:
                    out[(l, k)] = (n.value, ms.value)
        return out

    def level(self, l, adjoint=False):
        """Host copies of the arrays of level l (values as float64)."""
        s = self.sizes(l, adjoint)
        b = self.level_b
        d = dict(s)
        d["row_ptr"] = self._array(l, A_ROWPTR, np.int32, None, adjoint)
        d["col"] = self._array(l, A_COL, np.int32, None, adjoint)
        d["vals"] = self._array(l, A_VALS, np.float64, (-1, b, b), adjoint)
        d["dinv"] = self._array(l, DINV, np.float64, (-1, b, b), adjoint)
        d["cf"] = self._array(l, CF, np.int8, None, adjoint)
        d["strong"] = self._array(l, STRONG, np.uint8, None, adjoint)
        d["lam"] = self._array(l, LAMBDA, np.int32, None, adjoint)
        if not s["coarsest"]:
            d["ipc"] = self._array(l, P_MAP, np.int32, None, adjoint)
            d["R_rp"] = self._array(l, R_ROWPTR, np.int32, None, adjoint)
            d["R_ci"] = self._array(l, R_COL, np.int32, None, adjoint)
            d["R_v"] = self._array(l, R_VALS, np.float64, (-1, b, b), adjoint)
            if self.params.keep_setup_data:
                d["D_rp"] = self._array(l, DELTA_ROWPTR, np.int32, None, adjoint)
                d["D_ci"] = self._array(l, DELTA_COL, np.int32, None, adjoint)
                d["D_v"] = self._array(l, DELTA_VALS, np.float64, (-1, b, b), adjoint)
                d["L_rp"] = self._array(l, L_ROWPTR, np.int32, None, adjoint)
                d["L_ci"] = self._array(l, L_COL, np.int32, None, adjoint)
                d["L_v"] = self._array(l, L_VALS, np.float64, (-1, b, b), adjoint)
        return d


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[_ptr(t).value for t in ts])


def setup_batch(systems, streams=None, **params):
    """Set up independent systems concurrently (nair_setup_batch).

    systems: list of (row_ptr, col, vals) CUDA tensors; each system gets its
    own stream (new torch.cuda.Stream objects unless ``streams`` is given).
    Returns the NairSolver objects."""
    count = len(systems)
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(count)]
    cur = torch.cuda.current_stream()
    for st in streams:
        st.wait_stream(cur)  # the inputs were produced on the current stream
    A = (_Bsr * count)()
    P = (_Params * count)()
    for k, (rp, ci, v) in enumerate(systems):
        A[k] = _Bsr(int(rp.shape[0] - 1), int(v.shape[-1]), int(ci.shape[0]), _ptr(rp), _ptr(ci), _ptr(v))
        P[k] = _make_params(params, streams[k])
    hs = (ctypes.c_void_p * count)()
    _check(lib().nair_setup_batch(A, P, count, hs), "nair_setup_batch")
    return [NairSolver(rp, ci, v, stream=streams[k], _handle=ctypes.c_void_p(hs[k]), **params)
            for k, (rp, ci, v) in enumerate(systems)]


def _batch(fn, name, solvers, rhs, check):
    count = len(solvers)
    cur = torch.cuda.current_stream()
    xs = [torch.zeros_like(r) for r in rhs]
    for S in solvers:
        if S.stream is not None:
            S.stream.wait_stream(cur)
    cap = max(S.params.maxiter + S.params.maxiter // max(1, S.params.gmres_restart) + 4 for S in solvers)
    infos = (_Info * count)()
    hists = []
    for k in range(count):
        h = np.zeros(cap)
        hists.append(h)
        infos[k].history = h.ctypes.data_as(ctypes.c_void_p)
        infos[k].history_cap = cap
    hs = (ctypes.c_void_p * count)(*[S._h.value for S in solvers])
    st = fn(hs, count, _ptr_array(rhs), _ptr_array(xs), infos)
    if check:
        _check(st, name)
    for S in solvers:
        if S.stream is not None:
            cur.wait_stream(S.stream)
    return xs, [NairSolver._report(infos[k], hists[k], st) for k in range(count)]


def solve_batch(solvers, rhs, check=True):
    """Solve solvers[k] x_k = rhs[k] concurrently (nair_solve_batch); returns (xs, reports)."""
    return _batch(lib().nair_solve_batch, "nair_solve_batch", solvers, rhs, check)


def adjoint_solve_batch(solvers, w, check=True):
    """Solve A_k^T lambda_k = w[k] concurrently (nair_adjoint_solve_batch)."""
    return _batch(lib().nair_adjoint_solve_batch, "nair_adjoint_solve_batch", solvers, w, check)


def block_inverse(A):
    """Batched FP64 inverses of (nblk, b, b) blocks on the GPU (step a1)."""
    A = A.contiguous()
    out = torch.empty_like(A)
    _check(lib().nair_block_inverse(A.shape[0], A.shape[-1], _ptr(A), _ptr(out), _stream()),
           "nair_block_inverse")
    return out


def assemble_sigma(vals0, diag_pos, mass, sigma):
    out = torch.empty_like(vals0)
    _check(lib().nair_assemble_sigma(mass.shape[0], mass.shape[-1], vals0.shape[0], _ptr(diag_pos),
                                     _ptr(vals0), _ptr(mass), _ptr(sigma), _ptr(out), _stream()),
           "nair_assemble_sigma")
    return out


def mass_apply(mass, q):
    out = torch.empty_like(q)
    _check(lib().nair_mass_apply(mass.shape[0], mass.shape[-1], _ptr(mass), _ptr(q), _ptr(out), _stream()),
           "nair_mass_apply")
    return out


def gradients(mass, lam, x):
    E, b = mass.shape[0], mass.shape[-1]
    gs = torch.empty(E, dtype=torch.float64, device=mass.device)
    gq = torch.empty(E * b, dtype=torch.float64, device=mass.device)
    _check(lib().nair_gradients(E, b, _ptr(mass), _ptr(lam), _ptr(x), _ptr(gs), _ptr(gq), _stream()),
           "nair_gradients")
    return gs, gq


class NairSolve(torch.autograd.Function):
    """x = A(sigma)^{-1} M q for the DG transport operator, with A(sigma)'s
    diagonal blocks A0_ee + sigma_e M_e.  Backward solves A^T lambda = dJ/dx
    (by default with the transposed cycle of the forward hierarchy) and
    returns dJ/dq = M^T lambda, dJ/dsigma_e = -lambda_e^T M_e x_e.
    """

    @staticmethod
    def forward(ctx, q, sigma, row_ptr, col, vals0, diag_pos, mass, params):
        vals = assemble_sigma(vals0, diag_pos, mass, sigma)
        rhs = mass_apply(mass, q)
        solver = NairSolver(row_ptr, col, vals, **params)
        x, rep = solver.solve(rhs)
        ctx.solver = solver
        ctx.save_for_backward(mass, x)
        ctx.report = rep
        return x

    @staticmethod
    def backward(ctx, gx):
        mass, x = ctx.saved_tensors
        lam, _ = ctx.solver.adjoint_solve(gx.contiguous())
        gs, gq = gradients(mass, lam, x)
        ctx.solver.close()
        return gq, gs, None, None, None, None, None, None


def solve_host(row_ptr, col, vals, rhs, **params):
    """End-to-end call from host (pinned) arrays: copies in, setup, solve, copy out."""
    dev = torch.device("cuda")
    rp = torch.from_numpy(np.ascontiguousarray(row_ptr)).pin_memory().to(dev, non_blocking=True)
    ci = torch.from_numpy(np.ascontiguousarray(col)).pin_memory().to(dev, non_blocking=True)
    v = torch.from_numpy(np.ascontiguousarray(vals)).pin_memory().to(dev, non_blocking=True)
    b = torch.from_numpy(np.ascontiguousarray(rhs)).pin_memory().to(dev, non_blocking=True)
    s = NairSolver(rp, ci, v, **params)
    x, rep = s.solve(b)
    out = x.cpu()
    s.close()
    return out.numpy(), rep
