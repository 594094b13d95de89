"""Thin Python binding of the GB300 R-matrix library (include/rmat.h).

Argument marshalling only: every entry point forwards to the C ABI of
librmat_gb300.so with plain integers, floats and device pointers (for example
``tensor.data_ptr()`` of a torch CUDA tensor and
``torch.cuda.current_stream().cuda_stream``).  There is no Python or CPU
implementation of any step: importing the binding fails loudly when the
shared library has not been built (``paper_2512_11590_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librmat_gb300.so")

RMAT_OK = 0
RMAT_ECUDA = -100
RMAT_ENOMEM = -101
RMAT_ESTATE = -102
RMAT_ETIMEOUT = -103
RMAT_ENODEV = -104
RMAT_ESINGULAR = 1
RMAT_ENOCONV = 2
RMAT_ECHANFN = 3

RMAT_C128 = 0
RMAT_C64_3XTF32_IR = 1
RMAT_C64_SIMT_IR = 2
RMAT_C64_3XF16_IR = 3
RMAT_C64_1XF16_IR = 4

RMAT_PARAM_NB = 1
RMAT_PARAM_PANEL_CTAS = 2
RMAT_PARAM_SPIN_LIMIT = 3
RMAT_PARAM_TIMING = 4
RMAT_PARAM_EQUILIBRATE = 5
RMAT_PARAM_PAIRED = 6
RMAT_PARAM_METHOD = 7   # 0 factor M, 1 Woodbury-kinetic (factor S = I + (K^-1 x I) W)
RMAT_PARAM_REFINE = 8   # 0 classical refinement, m = 1..64 FGMRES-IR with <= m inner steps
RMAT_PARAM_SOLVE_LOOKAHEAD = 9   # 1 (default) look-ahead; 2 next rows inside the diagonal step; 0 off
RMAT_PARAM_PROP_CONCURRENT = 10  # 1 (default) propagation sectors on concurrent worker contexts
RMAT_PARAM_RESIDUAL = 11  # FP64 residual products: 0 auto, 1 FP64 MMA, 2 tensor couplings, 3 + kinetic
RMAT_PARAM_TC_BN = 12  # tile width of the factor's tensor-core updates: 256 (0) or 128
RMAT_PARAM_RESID_SUMS = 13  # compensated kinetic residual sums: -1 complex128 only, 0 off, 1 on
RMAT_PARAM_SOLVE_BLOCK = 14  # rows per tensor-path solve step: 256 (0) or 128
RMAT_PARAM_FACTOR = 15       # tensor precisions: 0 LU with partial pivoting, 1 LDL^T
RMAT_PARAM_FACTOR_LOOKAHEAD = 16  # pivoted paired LU: next pair's panels beside the far update
RMAT_PARAM_LA_PANEL_CTAS = 17     # CTAs of a look-ahead sub-panel (0 = every SM)
RMAT_PARAM_LA_MIN_ROWS = 18       # smallest far block that looks ahead (0 = 6144)
RMAT_PARAM_SOLVE_GROUPS = 19      # concurrent column groups of the tensor-path solves (0 = 1)
RMAT_PARAM_LA_BOTH_ROWS = 20      # smallest far block with both next panels beside it (0 = 20480)

RMAT_BATCH_LANES = 1
RMAT_BATCH_SPLIT_N = 2
RMAT_BATCH_GRAPH = 3
RMAT_BATCH_SMALL_N = 4   # small-system class in one persistent launch: -1 all that fit, 0 off
RMAT_BATCH_NB_LANE = 5
RMAT_BATCH_NB_SERIAL = 6
RMAT_BATCH_TC_BN = 7

EXPORTED = ("rmat_create", "rmat_destroy", "rmat_set_param", "rmat_mesh", "rmat_assemble",
            "rmat_load_dense", "rmat_factor", "rmat_solve", "rmat_collision", "rmat_get_stats",
            "rmat_reset_counters", "rmat_refine_history", "rmat_collision_noalloc",
            "rmat_batch_create", "rmat_batch_nopen", "rmat_batch_set", "rmat_batch_tune",
            "rmat_batch_run", "rmat_batch_info", "rmat_batch_destroy", "rmat_status_string",
            "rmat_sector_mesh", "rmat_propagate", "rmat_residual")


class rmat_problem(ct.Structure):
    _fields_ = [("nch", ct.c_int), ("nlag", ct.c_int), ("a", ct.c_double), ("hm", ct.c_double),
                ("bloch_B", ct.c_double), ("l", ct.POINTER(ct.c_int)),
                ("thresh", ct.POINTER(ct.c_double)), ("precision", ct.c_int),
                ("zz", ct.POINTER(ct.c_double))]


class RmatError(RuntimeError):
    def __init__(self, name, status, detail=""):
        self.status = status
        super().__init__(f"{name} -> {status} ({status_string(status)})"
                         + (f" at {detail}" if detail else ""))


_lib = None


def lib():
    """Load librmat_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2512_11590_gb300.build.build() "
                               "(nvcc, sm_103a); there is no fallback implementation")
        L = ct.CDLL(LIB_PATH)
        vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
        pd, pi = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)
        sig = {
            "rmat_create": (i, [ct.POINTER(vp), i, vp]),
            "rmat_destroy": (i, [vp]),
            "rmat_set_param": (i, [vp, i, ct.c_longlong]),
            "rmat_mesh": (i, [i, d, pd, pd, pd, pd, pd, pd]),
            "rmat_assemble": (i, [vp, ct.POINTER(rmat_problem), d, vp]),
            "rmat_load_dense": (i, [vp, i, i, vp, i, vp, i, i]),
            "rmat_factor": (i, [vp, pi]),
            "rmat_solve": (i, [vp, vp, i, i, d, pi, pd]),
            "rmat_collision": (i, [vp, vp, vp, pi]),
            "rmat_get_stats": (i, [vp, pd, i]),
            "rmat_reset_counters": (i, [vp]),
            "rmat_refine_history": (i, [vp, pd, i]),
            "rmat_residual": (i, [vp, vp, i, vp, i]),
            "rmat_collision_noalloc": (i, [ct.POINTER(rmat_problem), d, vp, vp, i, vp, vp, pi, vp]),
            "rmat_batch_create": (i, [vp, i, ct.POINTER(rmat_problem), pd, ct.POINTER(vp), i, d,
                                      ct.POINTER(vp)]),
            "rmat_batch_nopen": (i, [vp, pi]),
            "rmat_batch_set": (i, [vp, i, ct.c_longlong]),
            "rmat_batch_tune": (i, [vp, ct.POINTER(vp), pi, pi]),
            "rmat_batch_run": (i, [vp, ct.POINTER(vp), pi, pi]),
            "rmat_batch_info": (i, [vp, ct.POINTER(ct.c_longlong), i]),
            "rmat_batch_destroy": (i, [vp]),
            "rmat_status_string": (ct.c_char_p, [i]),
            "rmat_last_error": (i, [ct.c_char_p, i]),
            "rmat_sector_mesh": (i, [i, d, d, pd, pd, pd, pd, pd]),
            "rmat_propagate": (i, [vp, ct.POINTER(rmat_problem), d, i, pd, ct.POINTER(vp), i, d,
                                   vp, vp, pi]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().rmat_status_string(int(s)).decode()


def rmat_last_error() -> tuple:
    """(CUDA error code, "file:line name: description") of the last RMAT_ECUDA."""
    buf = ct.create_string_buffer(256)
    e = lib().rmat_last_error(buf, 256)
    return e, buf.value.decode()


def _check(name, s, ok=(RMAT_OK,)):
    if s not in ok:
        if s == RMAT_ECUDA:
            raise RmatError(name, s, rmat_last_error()[1])
        raise RmatError(name, s)
    return s


# ---- entry points (same names as the C ABI) ---------------------------------

def rmat_create(device: int = 0, stream: int = 0) -> int:
    h = ct.c_void_p()
    _check("rmat_create", lib().rmat_create(ct.byref(h), int(device), ct.c_void_p(stream or None)))
    return h.value


def rmat_destroy(ctx: int) -> None:
    _check("rmat_destroy", lib().rmat_destroy(ct.c_void_p(ctx)))


def rmat_set_param(ctx: int, key: int, value: int) -> None:
    _check("rmat_set_param", lib().rmat_set_param(ct.c_void_p(ctx), int(key), int(value)))


def rmat_mesh(nlag: int, a: float) -> dict:
    """Host mesh tables: x, omx, lam, r, f_a (nlag,) and T0 (nlag, nlag), float64."""
    out = {k: np.zeros(nlag) for k in ("x", "omx", "lam", "r", "f_a")}
    T0 = np.zeros((nlag, nlag))
    p = lambda arr: arr.ctypes.data_as(ct.POINTER(ct.c_double))  # noqa: E731
    _check("rmat_mesh", lib().rmat_mesh(int(nlag), float(a), p(out["x"]), p(out["omx"]),
                                         p(out["lam"]), p(out["r"]), p(out["f_a"]), p(T0)))
    out["T0"] = T0
    return out


def make_problem_struct(nch, nlag, a, hm, l, thresh, precision, bloch_B=0.0, zz=None):
    """rmat_problem plus the host arrays it points to (keep the tuple alive).

    zz: per-channel Z1 Z2 e^2 (MeV fm) of charged channels, None = all neutral."""
    l_arr = np.ascontiguousarray(l, dtype=np.int32)
    t_arr = np.ascontiguousarray(thresh, dtype=np.float64)
    z_arr = None if zz is None else np.ascontiguousarray(zz, dtype=np.float64)
    z_ptr = (ct.POINTER(ct.c_double)() if z_arr is None
             else z_arr.ctypes.data_as(ct.POINTER(ct.c_double)))
    s = rmat_problem(int(nch), int(nlag), float(a), float(hm), float(bloch_B),
                     l_arr.ctypes.data_as(ct.POINTER(ct.c_int)),
                     t_arr.ctypes.data_as(ct.POINTER(ct.c_double)), int(precision), z_ptr)
    return s, (l_arr, t_arr, z_arr)


def rmat_assemble(ctx: int, prob: rmat_problem, E: float, V_dev: int) -> None:
    _check("rmat_assemble", lib().rmat_assemble(ct.c_void_p(ctx), ct.byref(prob), float(E),
                                                ct.c_void_p(V_dev)))


def rmat_load_dense(ctx, n, nrhs, A_dev, lda, B_dev, ldb, precision) -> None:
    _check("rmat_load_dense", lib().rmat_load_dense(ct.c_void_p(ctx), int(n), int(nrhs),
                                                    ct.c_void_p(A_dev), int(lda),
                                                    ct.c_void_p(B_dev), int(ldb), int(precision)))


def rmat_factor(ctx: int, want_info: bool = True):
    """Returns (status, info); info is None when not requested (no synchronisation)."""
    if want_info:
        info = ct.c_int(0)
        s = lib().rmat_factor(ct.c_void_p(ctx), ct.byref(info))
        _check("rmat_factor", s, ok=(RMAT_OK, RMAT_ESINGULAR))
        return s, info.value
    s = lib().rmat_factor(ct.c_void_p(ctx), None)
    _check("rmat_factor", s)
    return s, None


def rmat_solve(ctx, X_dev, ldx, max_refine=0, tol=0.0):
    """Returns (status, iters, rel_resid); RMAT_ENOCONV is returned, not raised."""
    it = ct.c_int(0)
    rel = ct.c_double(0.0)
    s = lib().rmat_solve(ct.c_void_p(ctx), ct.c_void_p(X_dev), int(ldx), int(max_refine),
                         float(tol), ct.byref(it), ct.byref(rel))
    _check("rmat_solve", s, ok=(RMAT_OK, RMAT_ENOCONV))
    return s, it.value, rel.value


def rmat_collision(ctx, R_dev=0, U_dev=0) -> int:
    """Returns nopen."""
    nopen = ct.c_int(0)
    _check("rmat_collision", lib().rmat_collision(ct.c_void_p(ctx), ct.c_void_p(R_dev or None),
                                                  ct.c_void_p(U_dev or None), ct.byref(nopen)))
    return nopen.value


def rmat_sector_mesh(nlag: int, r1: float, r2: float) -> dict:
    """Sector mesh of (r1, r2): r, lam, fL, fR (nlag,) and Kf (nlag, nlag), float64."""
    out = {k: np.zeros(nlag) for k in ("r", "lam", "fL", "fR")}
    Kf = np.zeros((nlag, nlag))
    p = lambda arr: arr.ctypes.data_as(ct.POINTER(ct.c_double))  # noqa: E731
    _check("rmat_sector_mesh", lib().rmat_sector_mesh(int(nlag), float(r1), float(r2), p(out["r"]),
                                                      p(out["lam"]), p(out["fL"]), p(out["fR"]),
                                                      p(Kf)))
    out["Kf"] = Kf
    return out


def rmat_propagate(ctx, prob, E, radii, V_ptrs, max_refine=30, tol=1e-13, R_dev=0, U_dev=0):
    """R-matrix propagation over len(radii)-1 sectors; returns (status, nopen)."""
    ns = len(radii) - 1
    rad = np.ascontiguousarray(radii, dtype=np.float64)
    vp = (ct.c_void_p * ns)(*[int(v) for v in V_ptrs])
    nopen = ct.c_int(0)
    s = lib().rmat_propagate(ct.c_void_p(ctx), ct.byref(prob), float(E), int(ns),
                             rad.ctypes.data_as(ct.POINTER(ct.c_double)), vp, int(max_refine),
                             float(tol), ct.c_void_p(R_dev or None), ct.c_void_p(U_dev or None),
                             ct.byref(nopen))
    _check("rmat_propagate", s, ok=(RMAT_OK, RMAT_ENOCONV))
    return s, nopen.value


STAT_KEYS = ("N", "nrhs", "nb", "panel_ctas", "launches", "tu_launches", "tu_ms", "tu_flops",
             "assemble_ms", "factor_ms", "solve_ms", "refine_ms", "collision_ms",
             "panel_ms", "panel_launches", "apply_inv_ms", "apply_inv_launches",
             "solve_tc_ms", "solve_tc_launches", "resid_ms", "resid_launches", "gmres_inner",
             "backward_error", "factor_ldlt", "ldlt_lmax")


def rmat_get_stats(ctx) -> dict:
    buf = (ct.c_double * len(STAT_KEYS))()
    n = lib().rmat_get_stats(ct.c_void_p(ctx), buf, len(STAT_KEYS))
    return {k: buf[i] for i, k in enumerate(STAT_KEYS[:n])}


def rmat_reset_counters(ctx) -> None:
    _check("rmat_reset_counters", lib().rmat_reset_counters(ct.c_void_p(ctx)))


def rmat_residual(ctx, X_dev, ldx, R_dev, ldr) -> None:
    """R = Phi - C X (FP64) for a caller's X; column-major device buffers."""
    _check("rmat_residual", lib().rmat_residual(ct.c_void_p(ctx), ct.c_void_p(X_dev), int(ldx),
                                                ct.c_void_p(R_dev), int(ldr)))


def rmat_refine_history(ctx) -> list:
    n = lib().rmat_refine_history(ct.c_void_p(ctx), None, 0)
    buf = (ct.c_double * max(n, 1))()
    lib().rmat_refine_history(ct.c_void_p(ctx), buf, n)
    return [buf[k] for k in range(n)]


def rmat_collision_noalloc(prob, E, f_a_dev, X_dev, ldx, R_dev, U_dev, stream=0) -> int:
    """R and U from a solved X without allocating (see include/rmat.h). Returns nopen."""
    nopen = ct.c_int(0)
    _check("rmat_collision_noalloc",
           lib().rmat_collision_noalloc(ct.byref(prob), float(E), ct.c_void_p(f_a_dev),
                                        ct.c_void_p(X_dev), int(ldx), ct.c_void_p(R_dev or None),
                                        ct.c_void_p(U_dev or None), ct.byref(nopen),
                                        ct.c_void_p(stream or None)))
    return nopen.value


# ---- batches -------------------------------------------------------------------

def _ptrs(seq):
    return (ct.c_void_p * len(seq))(*[ct.c_void_p(int(p) or None) for p in seq])


def rmat_batch_create(ctx, probs, energies, V_ptrs, max_refine=30, tol=1e-13) -> int:
    """probs: list of rmat_problem (all one precision); returns the batch handle."""
    n = len(probs)
    arr = (rmat_problem * n)(*probs)
    E = (ct.c_double * n)(*[float(e) for e in energies])
    h = ct.c_void_p()
    _check("rmat_batch_create", lib().rmat_batch_create(ct.c_void_p(ctx), n, arr, E, _ptrs(V_ptrs),
                                                        int(max_refine), float(tol), ct.byref(h)))
    return h.value


def rmat_batch_nopen(b, n) -> list:
    out = (ct.c_int * n)()
    _check("rmat_batch_nopen", lib().rmat_batch_nopen(ct.c_void_p(b), out))
    return list(out)


def rmat_batch_set(b, key, value) -> None:
    _check("rmat_batch_set", lib().rmat_batch_set(ct.c_void_p(b), int(key), int(value)))


def rmat_batch_tune(b, U_ptrs):
    lanes, split = ct.c_int(0), ct.c_int(0)
    _check("rmat_batch_tune", lib().rmat_batch_tune(ct.c_void_p(b), _ptrs(U_ptrs), ct.byref(lanes),
                                                    ct.byref(split)))
    return lanes.value, split.value


def rmat_batch_run(b, U_ptrs):
    """Returns (status list, refinement-step list)."""
    n = len(U_ptrs)
    st = (ct.c_int * n)()
    it = (ct.c_int * n)()
    _check("rmat_batch_run", lib().rmat_batch_run(ct.c_void_p(b), _ptrs(U_ptrs), st, it))
    return list(st), list(it)


def rmat_batch_info(b) -> dict:
    keys = ("systems", "lanes", "split_n", "graph", "launches", "small_systems", "small_n",
            "nb_lane", "nb_serial", "tc_bn_lane")
    out = (ct.c_longlong * len(keys))()
    n = lib().rmat_batch_info(ct.c_void_p(b), out, len(keys))
    return dict(zip(keys, list(out)[:n]))


def rmat_batch_destroy(b) -> None:
    _check("rmat_batch_destroy", lib().rmat_batch_destroy(ct.c_void_p(b)))
