"""FP64 CPU oracle for block nAIR (arXiv 1704.05001) -- test infrastructure only.

The oracle is a plain C restatement of the method (``nair_oracle.c``), built
with gcc and loaded with ctypes.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may use it; the GPU library never imports it and
shares no code with it.  Every function in the C file cites the passage of
the paper it follows.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nair_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "singular block", 3: "not converged",
          4: "breakdown", 5: "out of memory"}

# level arrays exported by orc_level_get
A_RP, A_CI, A_V, DINV, CF, IPC, D_RP, D_CI, D_V, R_RP, R_CI, R_V, STRONG, LAM, L_RP, L_CI, L_V = range(17)


def build(force=False):
    """Compile the oracle with gcc (no contraction of multiply-adds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build_omp(force=False):
    """The same source built with OpenMP, for timing the oracle on all host
    cores (rows in parallel, each row's arithmetic unchanged; dot products in
    fixed chunks).  Not used by the parity tests."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp",
               "-shared", "-o", _LIB_OMP + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB_OMP + ".tmp", _LIB_OMP)
    return _LIB_OMP


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_setup.restype = P
            lib.orc_setup.argtypes = [I, I, P, P, P, D, D, I, I, I, I, I, ctypes.c_ulonglong,
                                      ctypes.POINTER(I)]
            lib.orc_setup_scalar.restype = P
            lib.orc_setup_scalar.argtypes = lib.orc_setup.argtypes
            lib.orc_free.argtypes = [P]
            lib.orc_num_levels.argtypes = [P]
            lib.orc_level_sizes.argtypes = [P, I, P]
            lib.orc_level_get.argtypes = [P, I, I, P]
            lib.orc_solve.argtypes = [P, P, P, I, I, I, I, D, P, I, ctypes.POINTER(I),
                                      ctypes.POINTER(I), ctypes.POINTER(D)]
            lib.orc_vcycle.argtypes = [P, P, P, I, I]
            lib.orc_vcycle_t.argtypes = [P, P, P, I, I]
            lib.orc_set_cycle.argtypes = [P, I]
            lib.orc_solve_t.argtypes = lib.orc_solve.argtypes
            lib.orc_block_inverse.argtypes = [I, P, P]
            lib.orc_transpose.argtypes = [I, I, P, P, P, P, P, P]
            lib.orc_gradients.argtypes = [I, I, P, P, P, P, P]
            lib.orc_filter.argtypes = [I, I, P, P, P, D]
            lib.orc_filter.restype = I
            _lib = lib
    return _lib


class use_library:
    """Context manager: route the oracle's calls to another build of nair_oracle.c
    (the mutation tests load deliberately broken copies this way)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("orc_setup", "orc_setup_scalar", "orc_free", "orc_num_levels", "orc_level_sizes", "orc_level_get",
                     "orc_solve", "orc_vcycle", "orc_solve_t", "orc_vcycle_t", "orc_set_cycle", "orc_block_inverse", "orc_transpose", "orc_gradients",
                     "orc_filter"):
            getattr(lib, name).argtypes = getattr(self._saved, name).argtypes
            getattr(lib, name).restype = getattr(self._saved, name).restype
        _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"oracle {where}: {STATUS.get(status, status)}")
        self.status = status


DEFAULTS = dict(theta=0.1, filter_tol=1e-4, filter_targets=3, neumann_degree=1, max_levels=25,
                max_coarse=None, max_dense=4096, seed=0, f_sweeps=None, c_sweeps=1,
                restart=50, maxiter=500, tol=1e-10, cycle="V")


def default_max_coarse(b):
    """Coarsest level: at most max(2, 192 // b) elements (dense solve of <= ~192 unknowns)."""
    return max(2, 192 // b)


class Hierarchy:
    """An oracle hierarchy built from a block-CSR matrix (host arrays).

    scalar=True builds scalar nAIR: the hierarchy (block size 1) of D^{-1} A,
    with the Krylov solve on A preconditioned by the cycle applied to D^{-1} v.
    """

    def __init__(self, row_ptr, col, vals, scalar=False, **params):
        lib = _load()
        p = dict(DEFAULTS)
        p.update(params)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        self.b = vals.shape[-1]
        self.scalar = bool(scalar)
        self.level_b = 1 if scalar else self.b  # block size of the hierarchy's levels
        if p["max_coarse"] is None:
            p["max_coarse"] = default_max_coarse(self.level_b)
        if p["f_sweeps"] is None:
            p["f_sweeps"] = p["neumann_degree"] + 1
        self.params = p
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        self.E = len(rp) - 1
        st = ctypes.c_int(0)
        setup = lib.orc_setup_scalar if scalar else lib.orc_setup
        self._h = setup(self.E, self.b, _p(rp), _p(ci), _p(vals), p["theta"],
                                p["filter_tol"], p["filter_targets"], p["neumann_degree"],
                                p["max_levels"], p["max_coarse"], p["max_dense"], p["seed"],
                                ctypes.byref(st))
        if not self._h:
            raise OracleError(st.value, "setup")
        self.nlev = lib.orc_num_levels(self._h)
        self.set_cycle(p["cycle"])

    def set_cycle(self, cycle):
        """Preconditioner cycle of the forward solve: "V" or "F"."""
        st = _load().orc_set_cycle(self._h, {"V": 0, "F": 1}[cycle])
        if st:
            raise OracleError(st, "set_cycle")
        self.params["cycle"] = cycle

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_free(h)
            self._h = None

    def sizes(self, l):
        out = np.zeros(9, dtype=np.int64)
        _load().orc_level_sizes(self._h, l, _p(out))
        keys = ["E", "nnzb", "nC", "nF", "L_nnzb", "D_nnzb", "R_nnzb", "AP_nnzb", "coarsest"]
        return dict(zip(keys, (int(v) for v in out)))

    def _get(self, l, which, shape, dtype):
        out = np.zeros(shape, dtype=dtype)
        if out.size:
            _load().orc_level_get(self._h, l, which, _p(out))
        return out

    def level(self, l):
        """All arrays of level l (host copies)."""
        s = self.sizes(l)
        b = self.level_b
        E, nC, nF = s["E"], s["nC"], s["nF"]
        d = dict(s)
        d["row_ptr"] = self._get(l, A_RP, E + 1, np.int32)
        d["col"] = self._get(l, A_CI, s["nnzb"], np.int32)
        d["vals"] = self._get(l, A_V, (s["nnzb"], b, b), np.float64)
        d["dinv"] = self._get(l, DINV, (E, b, b), np.float64)
        if not s["coarsest"] or nC + nF == E:
            d["cf"] = self._get(l, CF, E, np.int8)
            d["strong"] = self._get(l, STRONG, s["nnzb"], np.uint8)
            d["lam"] = self._get(l, LAM, E, np.int32)
        if not s["coarsest"]:
            d["ipc"] = self._get(l, IPC, E, np.int32)
            d["D_rp"] = self._get(l, D_RP, nF + 1, np.int32)
            d["D_ci"] = self._get(l, D_CI, s["D_nnzb"], np.int32)
            d["D_v"] = self._get(l, D_V, (s["D_nnzb"], b, b), np.float64)
            d["R_rp"] = self._get(l, R_RP, nC + 1, np.int32)
            d["R_ci"] = self._get(l, R_CI, s["R_nnzb"], np.int32)
            d["R_v"] = self._get(l, R_V, (s["R_nnzb"], b, b), np.float64)
            d["L_rp"] = self._get(l, L_RP, nF + 1, np.int32)
            d["L_ci"] = self._get(l, L_CI, s["L_nnzb"], np.int32)
            d["L_v"] = self._get(l, L_V, (s["L_nnzb"], b, b), np.float64)
        return d

    def solve(self, rhs, x0=None, transposed=False, **over):
        """FGMRES on A x = rhs with the V-cycle, or (transposed=True) on
        A^T x = rhs with the transposed cycle of the same hierarchy."""
        p = dict(self.params)
        p.update(over)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.zeros_like(rhs) if x0 is None else np.array(x0, dtype=np.float64)
        cap = p["maxiter"] + p["maxiter"] // max(1, p["restart"]) + 4
        hist = np.zeros(cap)
        hl = ctypes.c_int(0)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        fn = _load().orc_solve_t if transposed else _load().orc_solve
        st = fn(self._h, _p(rhs), _p(x), p["f_sweeps"], p["c_sweeps"], p["restart"],
                p["maxiter"], p["tol"], _p(hist), cap, ctypes.byref(hl),
                ctypes.byref(it), ctypes.byref(rr))
        return dict(x=x, status=st, history=hist[:hl.value].copy(), iterations=it.value,
                    relres=rr.value)

    def vcycle(self, f, f_sweeps=None, c_sweeps=None, transposed=False):
        """One cycle with zero initial guess: M^{-1} f with the hierarchy's cycle
        (V or F), or the transposed V-cycle M^{-T} f (transposed=True)."""
        p = self.params
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros_like(f)
        fn = _load().orc_vcycle_t if transposed else _load().orc_vcycle
        fn(self._h, _p(f), _p(x),
           p["f_sweeps"] if f_sweeps is None else f_sweeps,
           p["c_sweeps"] if c_sweeps is None else c_sweeps)
        return x


def block_inverse(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    X = np.zeros_like(A)
    st = _load().orc_block_inverse(A.shape[0], _p(A), _p(X))
    if st:
        raise OracleError(st, "block inverse")
    return X


def filter_blocks(row_ptr, col, vals, tol):
    """The block filter alone (Sec. 5.2): a copy of the square block-CSR matrix
    without the off-diagonal blocks X_ij with ||X_ij||_F^2 <= tol^2 ||X_ii||_F^2."""
    rp = np.array(row_ptr, dtype=np.int32)
    ci = np.array(col, dtype=np.int32)
    v = np.array(vals, dtype=np.float64)
    kept = _load().orc_filter(len(rp) - 1, v.shape[-1], _p(rp), _p(ci), _p(v), float(tol))
    return rp, ci[:kept].copy(), v[:kept].copy()


def transpose(row_ptr, col, vals):
    """Block transpose of a block-CSR matrix."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    E = len(rp) - 1
    b = v.shape[-1]
    trp = np.zeros(E + 1, dtype=np.int32)
    tci = np.zeros(len(ci), dtype=np.int32)
    tv = np.zeros_like(v)
    _load().orc_transpose(E, b, _p(rp), _p(ci), _p(v), _p(trp), _p(tci), _p(tv))
    return trp, tci, tv


def gradients(mass, lam, x):
    """(dJ/dsigma per element, dJ/dq per DOF) from the adjoint solution lam."""
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    E, b, _ = mass.shape
    gs = np.zeros(E)
    gq = np.zeros(E * b)
    _load().orc_gradients(E, b, _p(mass), _p(lam), _p(x), _p(gs), _p(gq))
    return gs, gq
