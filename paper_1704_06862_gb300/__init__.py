"""Thin ctypes binding of the GB300 JMCFIE/MLFMM library (``libsie.so``).

The functions below carry the names of the C ABI in ``include/sie.h`` and do
argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Device buffers are passed as torch CUDA tensors (or raw integer
device pointers); host arrays as numpy arrays.  There is no CPU fallback: if
the shared library is missing, importing a function raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsie.so")

SIE_PREC_FP64 = 0
SIE_PREC_MIXED = 1
SIE_PREC_NEAR64 = 2   # products only: FP64 near field + FP32 far field into the FP64 product

STATUS = {0: "SIE_OK", 1: "SIE_EINVAL", 2: "SIE_ENOMEM", 3: "SIE_ECUDA", 4: "SIE_ESTATE", 5: "SIE_ENOTCONV",
          6: "SIE_EBREAKDOWN", 7: "SIE_ETIMEOUT", 8: "SIE_EZEROPIVOT"}

EXPORTED = ["sie_create", "sie_destroy", "sie_last_error", "sie_build_mesh", "mlfmm_setup", "sie_fill_nearfield",
            "mlfmm_matvec", "sie_matvec_parts", "ilu_apply", "sie_plane_wave_rhs", "gmres_solve", "rcs_farfield", "rcs_farfield_prec",
            "sie_near_export", "sie_stage_timing", "sie_query", "ilu_apply_noalloc", "nnprec_train",
            "nnprec_params", "nnprec_loss_grad", "sie_device_status", "sie_set_param", "sie_autotune"]


class SieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class sie_mlfmm_opts(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("digits", ctypes.c_double)]


class sie_fill_opts(ctypes.Structure):
    _fields_ = [("outer_order", ctypes.c_int32), ("build_ilu", ctypes.c_int32), ("formulation", ctypes.c_int32)]


class sie_solve_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("tol", ctypes.c_double),
                ("prec", ctypes.c_int32), ("precond", ctypes.c_int32), ("method", ctypes.c_int32),
                ("no_graphs", ctypes.c_int32), ("residual_far_fp64", ctypes.c_int32)]


class sie_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsie.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sie_create": ([ctypes.POINTER(P), ctypes.c_int, P], I32),
        "sie_destroy": ([P], None),
        "sie_last_error": ([P], ctypes.c_char_p),
        "sie_build_mesh": ([P, P, I64, P, I64, P, P, I32, D, ctypes.POINTER(I64)], I32),
        "mlfmm_setup": ([P, ctypes.POINTER(sie_mlfmm_opts)], I32),
        "sie_fill_nearfield": ([P, ctypes.POINTER(sie_fill_opts)], I32),
        "mlfmm_matvec": ([P, P, P, I64, I32], I32),
        "sie_matvec_parts": ([P, P, P, I64, I32, I32], I32),
        "ilu_apply": ([P, P, P, I64, I32], I32),
        "sie_plane_wave_rhs": ([P, P, I64, P], I32),
        "gmres_solve": ([P, P, P, I64, ctypes.POINTER(sie_solve_opts), ctypes.POINTER(sie_solve_stats)], I32),
        "rcs_farfield": ([P, P, I64, P, I64, P], I32),
        "rcs_farfield_prec": ([P, P, I64, P, I64, I32, P], I32),
        "sie_near_export": ([P, P, P, P, ctypes.POINTER(I64)], I32),
        "sie_query": ([P, I32, ctypes.POINTER(I64)], I32),
        "sie_stage_timing": ([P, I32, I64, I32, I32, ctypes.POINTER(D)], I32),
        "ilu_apply_noalloc": ([P, P, P, I64, I32], I32),
        "nnprec_train": ([P, P, P], I32),
        "nnprec_params": ([P, P, I32], I32),
        "nnprec_loss_grad": ([P, P, P, I64, ctypes.POINTER(D), P], I32),
        "sie_device_status": ([P], I32),
        "sie_set_param": ([P, I32, I64], I32),
        "sie_autotune": ([P, I64, I32, P, P], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous")
        return t.ctypes.data
    raise TypeError(f"cannot pass {type(t)} as a pointer")


def _check(ctx, rc):
    if rc != 0:
        msg = load_library().sie_last_error(ctx)
        raise SieError(rc, msg.decode() if msg else "")
    return rc


# ----------------------------------------------------------------- C ABI, same names
def sie_create(device: int = 0, stream=None):
    ctx = ctypes.c_void_p()
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    rc = load_library().sie_create(ctypes.byref(ctx), device, s)
    if rc != 0:
        raise SieError(rc, "sie_create failed")
    return ctx


def sie_destroy(ctx):
    load_library().sie_destroy(ctx)


def sie_last_error(ctx) -> str:
    msg = load_library().sie_last_error(ctx)
    return msg.decode() if msg else ""


def sie_build_mesh(ctx, verts, tris, tri_regions, media, freq_hz):
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    r = np.ascontiguousarray(tri_regions, np.int32)
    m = np.ascontiguousarray(media, np.float64)
    n = ctypes.c_int64()
    _check(ctx, load_library().sie_build_mesh(ctx, _ptr(v), len(v), _ptr(t), len(t), _ptr(r), _ptr(m), len(m),
                                              float(freq_hz), ctypes.byref(n)))
    return n.value


def mlfmm_setup(ctx, levels, digits=3.0):
    o = sie_mlfmm_opts(int(levels), float(digits))
    _check(ctx, load_library().mlfmm_setup(ctx, ctypes.byref(o)))


FORM_JMCFIE, FORM_CTF, FORM_CNF, FORM_PMCHWT, FORM_ICTF = 0, 1, 2, 3, 4


def sie_fill_nearfield(ctx, outer_order=4, build_ilu=True, formulation=FORM_JMCFIE):
    o = sie_fill_opts(int(outer_order), 1 if build_ilu else 0, int(formulation))
    _check(ctx, load_library().sie_fill_nearfield(ctx, ctypes.byref(o)))


# Stream order between torch and the library.  The library works on its
# context's stream; torch tensors are filled and read on torch's current
# stream.  A call on device buffers first waits for torch's pending work on
# its inputs and outputs, and the asynchronous calls below wait for their own
# work before returning, so their results are ready for torch (and a bounded
# device wait that gave up is reported as SIE_ETIMEOUT).
def _torch_ready():
    import sys
    torch = sys.modules.get("torch")
    if torch is not None and torch.cuda.is_initialized():
        torch.cuda.current_stream().synchronize()


def _done(ctx):
    _check(ctx, load_library().sie_device_status(ctx))


def mlfmm_matvec(ctx, x, y, nrhs, prec=SIE_PREC_FP64):
    _torch_ready()
    _check(ctx, load_library().mlfmm_matvec(ctx, _ptr(x), _ptr(y), int(nrhs), int(prec)))
    _done(ctx)


def sie_matvec_parts(ctx, x, y, nrhs, prec=SIE_PREC_FP64, parts=3):
    _torch_ready()
    _check(ctx, load_library().sie_matvec_parts(ctx, _ptr(x), _ptr(y), int(nrhs), int(prec), int(parts)))
    _done(ctx)


def ilu_apply(ctx, r, z, nrhs, prec=SIE_PREC_FP64):
    _torch_ready()
    _check(ctx, load_library().ilu_apply(ctx, _ptr(r), _ptr(z), int(nrhs), int(prec)))
    _done(ctx)


def ilu_apply_noalloc(ctx, r, z, nrhs, prec=SIE_PREC_FP64):
    """ilu_apply without any device allocation (scratch: a fixed 16 MiB
    array inside the library; nrhs * n_rwg <= 174762)."""
    _torch_ready()
    _check(ctx, load_library().ilu_apply_noalloc(ctx, _ptr(r), _ptr(z), int(nrhs), int(prec)))
    _done(ctx)


def sie_plane_wave_rhs(ctx, inc, b):
    inc = np.ascontiguousarray(np.atleast_2d(inc), np.float64)
    _torch_ready()
    _check(ctx, load_library().sie_plane_wave_rhs(ctx, _ptr(inc), len(inc), _ptr(b)))
    _done(ctx)


SOLVE_FGMRES, SOLVE_BICGSTAB, SOLVE_CGS = 0, 1, 2


def gmres_solve(ctx, b, x, nrhs, restart=50, max_iters=1000, tol=1e-4, prec=SIE_PREC_FP64, precond=1,
                check=True, graphs=True, method=SOLVE_FGMRES, residual_far_fp64=False):
    """``gmres_solve`` of the C ABI on torch CUDA tensors b, x [nrhs, n_rwg, 2]
    (x: initial guess in, solution out).  method: SOLVE_FGMRES (restarted
    flexible GMRES), SOLVE_BICGSTAB or SOLVE_CGS; precond: 0 none, 1 ILU(0),
    2 ILU(0) with the learned correction (FGMRES only); prec: arithmetic of
    the inner product and preconditioner (SIE_PREC_FP64 or SIE_PREC_MIXED);
    graphs=False launches every step eagerly; residual_far_fp64=True makes the
    mixed form's true residual use the whole FP64 operator.  Returns one dict
    per right-hand side (iters, restarts, rel_residual, converged); with
    check=True a failed convergence raises SieError."""
    o = sie_solve_opts(int(restart), int(max_iters), float(tol), int(prec), int(precond), int(method),
                       0 if graphs else 1, 1 if residual_far_fp64 else 0)
    _torch_ready()
    st = (sie_solve_stats * int(nrhs))()
    rc = load_library().gmres_solve(ctx, _ptr(b), _ptr(x), int(nrhs), ctypes.byref(o), st)
    stats = [dict(iters=s.iters, restarts=s.restarts, rel_residual=s.rel_residual, converged=bool(s.converged))
             for s in st]
    if rc not in (0, 5) or (check and rc != 0):
        _check(ctx, rc)
    return stats


def rcs_farfield(ctx, x, nrhs, obs):
    obs = np.ascontiguousarray(obs, np.float64)
    out = np.zeros((int(nrhs), len(obs), 2), np.float64)
    _torch_ready()
    _check(ctx, load_library().rcs_farfield(ctx, _ptr(x), int(nrhs), _ptr(obs), len(obs), _ptr(out)))
    return out


def rcs_farfield_prec(ctx, x, nrhs, obs, prec=SIE_PREC_FP64):
    obs = np.ascontiguousarray(obs, np.float64)
    out = np.zeros((int(nrhs), len(obs), 2), np.float64)
    _torch_ready()
    _check(ctx, load_library().rcs_farfield_prec(ctx, _ptr(x), int(nrhs), _ptr(obs), len(obs), int(prec), _ptr(out)))
    return out


def sie_near_export(ctx):
    n = ctypes.c_int64()
    L = load_library()
    _check(ctx, L.sie_near_export(ctx, None, None, None, ctypes.byref(n)))
    rows = np.zeros(n.value, np.int32)
    cols = np.zeros(n.value, np.int32)
    vals = np.zeros((n.value, 4, 2), np.float64)
    _check(ctx, L.sie_near_export(ctx, _ptr(rows), _ptr(cols), _ptr(vals), ctypes.byref(n)))
    return rows, cols, vals[..., 0] + 1j * vals[..., 1]


def sie_stage_timing(ctx, stage, nrhs=1, prec=SIE_PREC_FP64, reps=10):
    ms = ctypes.c_double()
    _check(ctx, load_library().sie_stage_timing(ctx, int(stage), int(nrhs), int(prec), int(reps), ctypes.byref(ms)))
    return ms.value


class sie_nn_opts(ctypes.Structure):
    _fields_ = [("train_inc", ctypes.c_void_p), ("ntrain", ctypes.c_int32), ("record_restart", ctypes.c_int32),
                ("max_pairs", ctypes.c_int32), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_double), ("seed", ctypes.c_uint64)]


class sie_nn_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int32), ("samples", ctypes.c_int64), ("loss_first", ctypes.c_double),
                ("loss_last", ctypes.c_double), ("ms", ctypes.c_double), ("val_loss_ratio", ctypes.c_double),
                ("gamma", ctypes.c_double), ("enabled", ctypes.c_int32), ("gate_iters_ilu", ctypes.c_int32),
                ("gate_iters_nn", ctypes.c_int32)]


NN_PARAMS = 128 * 256 + 256 + 256 * 256 + 256 + 256 * 128 + 128


def nnprec_train(ctx, train_inc, record_restart=5, max_pairs=256, epochs=20, batch=2048, lr=1e-3, seed=2017):
    inc = np.ascontiguousarray(np.atleast_2d(train_inc), np.float64)
    o = sie_nn_opts(_ptr(inc), len(inc), int(record_restart), int(max_pairs), int(epochs), int(batch), float(lr),
                    int(seed))
    st = sie_nn_stats()
    _check(ctx, load_library().nnprec_train(ctx, ctypes.byref(o), ctypes.byref(st)))
    return dict(pairs=st.pairs, samples=st.samples, loss_first=st.loss_first, loss_last=st.loss_last, ms=st.ms,
                val_loss_ratio=st.val_loss_ratio, gamma=st.gamma, enabled=bool(st.enabled),
                gate_iters_ilu=st.gate_iters_ilu, gate_iters_nn=st.gate_iters_nn)


def nnprec_params(ctx, params=None):
    """Return the FP32 master parameters, or set them when ``params`` is given."""
    if params is None:
        out = np.zeros(NN_PARAMS, np.float32)
        _check(ctx, load_library().nnprec_params(ctx, _ptr(out), 0))
        return out
    p = np.ascontiguousarray(params, np.float32)
    _check(ctx, load_library().nnprec_params(ctx, _ptr(p), 1))
    return p


def nnprec_loss_grad(ctx, X, T):
    X = np.ascontiguousarray(X, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    loss = ctypes.c_double()
    g = np.zeros(NN_PARAMS, np.float32)
    _check(ctx, load_library().nnprec_loss_grad(ctx, _ptr(X), _ptr(T), len(X), ctypes.byref(loss), _ptr(g)))
    return loss.value, g


def sie_device_status(ctx):
    """Raises SieError (SIE_ETIMEOUT) if a bounded device-side wait gave up
    since the last call; synchronises the context's stream."""
    _check(ctx, load_library().sie_device_status(ctx))


def sie_set_param(ctx, key, value):
    """Runtime parameter: key 0 the wait limit of device-side barriers (polls),
    key 1 the single-RHS ILU(0) schedule (0 persistent launch, 1 one launch
    per colour step, the default)."""
    _check(ctx, load_library().sie_set_param(ctx, int(key), int(value)))


TUNING_KEYS = {"near_rb": 4, "ilu_rb": 5, "aggregation": 3, "receive_rb": 6, "m2l": 7, "receive_tc": 8}


def sie_autotune(ctx, nrhs, reps=3, path=None):
    """Autotune the block-RHS tile shapes for nrhs right-hand sides (kept in
    the context).  Returns {"nrhs", "near_rb", "ilu_rb", "aggregation",
    "receive_rb", "m2l", "receive_tc", "ms": [near, ilu, far]}; with a path, also writes it
    there as JSON (read back with apply_tuning)."""
    import json
    ch = np.zeros(6, np.int64)
    ms = np.zeros(3, np.float64)
    _check(ctx, load_library().sie_autotune(ctx, int(nrhs), int(reps), _ptr(ch), _ptr(ms)))
    out = {"nrhs": int(nrhs), "near_rb": int(ch[0]), "ilu_rb": int(ch[1]), "aggregation": int(ch[2]),
           "receive_rb": int(ch[3]), "m2l": int(ch[4]), "receive_tc": int(ch[5]), "ms": [float(v) for v in ms]}
    if path:
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
    return out


def apply_tuning(ctx, tuning):
    """Set the tile shapes of a sie_autotune result (a dict or a JSON path)."""
    import json
    if isinstance(tuning, str):
        with open(tuning) as f:
            tuning = json.load(f)
    sie_set_param(ctx, 2, 2 if tuning["aggregation"] else 0)
    for name, key in TUNING_KEYS.items():
        sie_set_param(ctx, key, tuning.get(name, {"m2l": -1, "receive_tc": -1}.get(name, 0)))


def sie_query(ctx, key):
    v = ctypes.c_int64()
    _check(ctx, load_library().sie_query(ctx, int(key), ctypes.byref(v)))
    return v.value


# ----------------------------------------------------------------- convenience (marshalling only)
class Solver:
    """Owns one context: mesh -> tree -> fill, then operator calls on torch tensors."""

    def __init__(self, mesh: dict, levels: int, digits: float = 3.0, freq_hz: float = 299792458.0,
                 device: int = 0, stream=None, outer_order: int = 4, build_ilu: bool = True,
                 formulation: int = FORM_JMCFIE):
        self.ctx = sie_create(device, stream)
        self.ne = sie_build_mesh(self.ctx, mesh["verts"], mesh["tris"], mesh["tri_regions"], mesh["media"], freq_hz)
        mlfmm_setup(self.ctx, levels, digits)
        sie_fill_nearfield(self.ctx, outer_order, build_ilu, formulation)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            sie_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, nrhs=1):
        import torch
        return torch.zeros((nrhs, self.ne, 2), dtype=torch.complex128, device="cuda")
