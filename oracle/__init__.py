"""FP64 CPU oracle for ordinary kriging of missing inter-slice voxels (arXiv 2303.09523).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import it.  It shares no code with
the CUDA library (``paper_2303_09523_gb300``) and neither imports the other.

The arithmetic lives in ``krig_oracle.c`` (Gaussian elimination with partial
pivoting on the bordered ordinary-kriging system, Appendix A with one constant
predictor; sub-block layout of Algorithm 1).  This module marshals numpy arrays
through ctypes (``krig_oracle.c`` also holds the universal-kriging solver of
Appendix A with polynomial drift, ``uk_solve`` / ``uk_voxels``), and holds one
numpy function of its own:
``empirical_variogram`` (the method-of-moments semivariogram of the known
slices, the data the variogram of Sec. 4.1.2 is fitted to).
"""
import ctypes
import os

import numpy as np

from . import build as _build

SPHERICAL, EXPONENTIAL, LINEAR = 0, 1, 2
_MODELS = {"spherical": SPHERICAL, "exponential": EXPONENTIAL, "linear": LINEAR}


class _Vg(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("pad", ctypes.c_int32), ("nugget", ctypes.c_double),
                ("sill", ctypes.c_double), ("range", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.POINTER(_Vg)
        i32 = ctypes.c_int32
        lib.orc_gamma.argtypes = [vp, ctypes.c_double]
        lib.orc_gamma.restype = ctypes.c_double
        lib.orc_gamma_grad.argtypes = [vp, ctypes.c_double, dp]
        lib.orc_gamma_grad.restype = None
        lib.orc_gauss_solve.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
        lib.orc_ok_solve.argtypes = [ctypes.c_int, dp, dp, vp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_krige_volume.argtypes = [dp, i32, i32, i32, i32, i32, i32, vp, i32, dp, dp]
        lib.orc_krige_voxels.argtypes = [dp, i32, i32, i32, i32, i32, vp, ctypes.c_int64, i64p, i32, dp, dp]
        lib.orc_loo.argtypes = [dp, i32, i32, i32, i32, i32, vp, i32, dp, dp, dp, dp]
        lib.orc_uk_solve.argtypes = [ctypes.c_int, dp, dp, vp, ctypes.c_int, dp, dp, dp, dp, dp]
        lib.orc_uk_voxels.argtypes = [dp, i32, i32, i32, i32, i32, i32, i32, vp, ctypes.c_int64, i64p, dp, dp]
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _vg(model="spherical", nugget=0.0, sill=1.0, range=8.0):
    m = _MODELS[model] if isinstance(model, str) else int(model)
    return _Vg(m, 0, float(nugget), float(sill), float(range))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st, what):
    if st != 0:
        raise OracleError("%s failed with status %d" % (what, st))


def max_threads() -> int:
    return _load().orc_max_threads()


def gamma(h, **vg) -> float:
    """Semivariogram value at lag ``h`` (gamma(0) = 0)."""
    v = _vg(**vg)
    return _load().orc_gamma(ctypes.byref(v), float(h))


def gamma_grad(h, **vg) -> np.ndarray:
    v = _vg(**vg)
    d = np.zeros(3)
    _load().orc_gamma_grad(ctypes.byref(v), float(h), _ptr(d))
    return d


def gauss_solve(A, B):
    """The oracle's own Gaussian elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    B = np.array(B, dtype=np.float64, order="C", copy=True)
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None].copy()
    m, nrhs = B.shape
    _check(_load().orc_gauss_solve(m, _ptr(A), _ptr(B), nrhs), "gauss_solve")
    return B[:, 0] if squeeze else B


def ok_solve(points, s0, values=None, grad=False, **vg):
    """Ordinary kriging at ``s0`` from ``points`` (K x 3).

    Returns dict with ``w`` (K), ``mu``, ``var``, ``est`` (if values given) and,
    with ``grad=True``, ``dw`` (K x 3) and ``dvar`` (3) w.r.t. (nugget, sill, range).
    """
    pts = np.ascontiguousarray(points, dtype=np.float64)
    K = pts.shape[0]
    s0 = np.ascontiguousarray(s0, dtype=np.float64)
    vals = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
    w = np.zeros(K)
    mu = np.zeros(1)
    var = np.zeros(1)
    est = np.zeros(1)
    dw = np.zeros((K, 3)) if grad else None
    dvar = np.zeros(3) if grad else None
    v = _vg(**vg)
    st = _load().orc_ok_solve(K, _ptr(pts), _ptr(s0), ctypes.byref(v), _ptr(vals), _ptr(w), _ptr(mu),
                              _ptr(var), _ptr(est), _ptr(dw), _ptr(dvar))
    _check(st, "ok_solve")
    out = {"w": w, "mu": float(mu[0]), "var": float(var[0])}
    if vals is not None:
        out["est"] = float(est[0])
    if grad:
        out["dw"] = dw
        out["dvar"] = dvar
    return out


DRIFTS = {"constant": 0, "z": 1, "xyz": 2}


def uk_solve(points, s0, drift="xyz", values=None, **vg):
    """Universal kriging at ``s0`` from ``points`` (K x 3) with polynomial drift
    ``constant`` ({1}: ordinary kriging), ``z`` ({1, z}) or ``xyz`` ({1, x, y, z})
    (Appendix A: one unbiasedness constraint and Lagrange multiplier per predictor).

    Returns dict with ``w`` (K), ``mu`` (one per predictor), ``var`` = w'gamma0 + mu'f0 and
    ``est`` (if values given).
    """
    d = DRIFTS[drift] if isinstance(drift, str) else int(drift)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    K = pts.shape[0]
    s0 = np.ascontiguousarray(s0, dtype=np.float64)
    vals = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
    w = np.zeros(K)
    mu = np.zeros(4)
    var = np.zeros(1)
    est = np.zeros(1)
    v = _vg(**vg)
    st = _load().orc_uk_solve(K, _ptr(pts), _ptr(s0), ctypes.byref(v), d, _ptr(vals), _ptr(w), _ptr(mu),
                              _ptr(var), _ptr(est))
    _check(st, "uk_solve")
    out = {"w": w, "mu": mu[:(1, 2, 4)[d]].copy(), "var": float(var[0])}
    if vals is not None:
        out["est"] = float(est[0])
    return out


def uk_voxels(slices, g, r, zyx, slabs=2, drift="xyz", **vg):
    """Universal kriging estimate and variance at output voxels ``zyx`` (M x 3, output z), from
    ``slabs`` known slices (2: the bracketing pair; 4: one more on each side where it exists),
    window (2r+1)^2 truncated at the in-plane border; known slices copied."""
    d = DRIFTS[drift] if isinstance(drift, str) else int(drift)
    s = np.ascontiguousarray(slices, dtype=np.float64)
    n, H, W = s.shape
    idx = np.ascontiguousarray(zyx, dtype=np.int64).reshape(-1, 3)
    est = np.empty(idx.shape[0])
    var = np.empty(idx.shape[0])
    v = _vg(**vg)
    st = _load().orc_uk_voxels(_ptr(s), n, H, W, g, r, slabs, d, ctypes.byref(v), idx.shape[0],
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(est), _ptr(var))
    _check(st, "uk_voxels")
    return est, var


def n_out(n, g):
    return (n - 1) * g + 1


def krige_volume(slices, g, r, k_sub=1, threads=0, want_var=True, **vg):
    """Whole-volume kriging (Algorithm 1 steps 2-4, merged as in Sec. 4.2).

    ``slices``: (n, H, W) array, converted to float64.  Returns (out, var),
    each ((n-1)g+1, H, W) float64; ``var`` is None if ``want_var`` is False.
    """
    s = np.ascontiguousarray(slices, dtype=np.float64)
    n, H, W = s.shape
    out = np.empty((n_out(n, g), H, W))
    var = np.empty_like(out) if want_var else None
    v = _vg(**vg)
    st = _load().orc_krige_volume(_ptr(s), n, H, W, g, r, k_sub, ctypes.byref(v), threads, _ptr(out), _ptr(var))
    _check(st, "krige_volume")
    return out, var


def krige_voxels(slices, g, r, zyx, threads=0, **vg):
    """Estimate and variance at selected output voxels ``zyx`` (M x 3, output z)."""
    s = np.ascontiguousarray(slices, dtype=np.float64)
    n, H, W = s.shape
    idx = np.ascontiguousarray(zyx, dtype=np.int64).reshape(-1, 3)
    est = np.empty(idx.shape[0])
    var = np.empty(idx.shape[0])
    v = _vg(**vg)
    st = _load().orc_krige_voxels(_ptr(s), n, H, W, g, r, ctypes.byref(v), idx.shape[0],
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), threads, _ptr(est), _ptr(var))
    _check(st, "krige_voxels")
    return est, var


def loo(slices, g, r, threads=0, want_pred=False, want_grad_theta=False, want_grad_slices=False, **vg):
    """Leave-one-slice-out CV loss; optional predictions and gradients.

    Returns dict: ``loss``, and ``pred`` ((n-2), H, W), ``grad_theta`` (3:
    nugget, sill, range), ``grad_slices`` (n, H, W) when requested.
    """
    s = np.ascontiguousarray(slices, dtype=np.float64)
    n, H, W = s.shape
    loss = np.zeros(1)
    pred = np.empty((n - 2, H, W)) if want_pred else None
    gt = np.zeros(3) if want_grad_theta else None
    gs = np.zeros((n, H, W)) if want_grad_slices else None
    v = _vg(**vg)
    st = _load().orc_loo(_ptr(s), n, H, W, g, r, ctypes.byref(v), threads, _ptr(loss), _ptr(pred), _ptr(gt), _ptr(gs))
    _check(st, "loo")
    out = {"loss": float(loss[0])}
    if want_pred:
        out["pred"] = pred
    if want_grad_theta:
        out["grad_theta"] = gt
    if want_grad_slices:
        out["grad_slices"] = gs
    return out


def empirical_variogram(slices, max_lag):
    """Sums of squared increments of the known slices per lag vector, and pair counts.

    The paper uses a variogram gamma(h) (Sec. 4.1.2) without saying how it is
    estimated; the classical method-of-moments estimate is
    gamma(h) = sum over pairs (z_i - z_j)^2 / (2 N(h)).  Lag vectors here are
    (dx, dy) in pixels, |dx|, |dy| <= max_lag, within one known slice (s = 0)
    or from known slice k to k + 1 (s = 1).  For each (s, dy, dx):
        sums[s, dy+L, dx+L]   = sum_{k, y, x} (S[k, y, x] - S[k+s, y+dy, x+dx])^2
        counts[s, dy+L, dx+L] = number of terms (both voxels inside the stack),
    summed in float64 over whole arrays (numpy).
    """
    S = np.asarray(slices, dtype=np.float64)
    n, H, W = S.shape
    L = int(max_lag)
    q = 2 * L + 1
    sums = np.zeros((2, q, q))
    counts = np.zeros((2, q, q), dtype=np.int64)
    for s in (0, 1):
        if n - s <= 0:
            continue
        for dy in range(-L, L + 1):
            ya, yb = max(0, -dy), min(H, H - dy)  # y with 0 <= y + dy < H
            for dx in range(-L, L + 1):
                xa, xb = max(0, -dx), min(W, W - dx)
                if yb <= ya or xb <= xa:
                    continue
                a = S[0:n - s, ya:yb, xa:xb]
                b = S[s:n, ya + dy:yb + dy, xa + dx:xb + dx]
                d = a - b
                sums[s, dy + L, dx + L] = float(np.sum(d * d))
                counts[s, dy + L, dx + L] = d.size
    return sums, counts



def sub_blocks(n, k):
    """Algorithm 1, step 2: the n - 1 gaps cut into k sub-blocks of whole gaps (the first (n-1) % k
    blocks one gap longer); block b holds known slices a_b .. a_{b+1}.  Returns [a_0, ..., a_k]."""
    q, rem = divmod(n - 1, k)
    a = [0]
    for b in range(k):
        a.append(a[-1] + q + (1 if b < rem else 0))
    return a


def clamp_block_minmax(out, slices, g, k):
    """The reading of Algorithm 1's per-block "maximum and minimum possible value": every missing
    voxel of block b (output slices strictly between a_b g and a_{b+1} g) clamped to [min, max] of
    the block's known slices a_b .. a_{b+1}.  Known slices are unchanged; NaN stays NaN."""
    res = np.array(out, dtype=np.float64, copy=True)
    S = np.asarray(slices, dtype=np.float64)
    a = sub_blocks(S.shape[0], k)
    for b in range(k):
        lo = float(S[a[b]:a[b + 1] + 1].min())
        hi = float(S[a[b]:a[b + 1] + 1].max())
        for z in range(a[b] * g + 1, a[b + 1] * g):
            if z % g:
                blk = res[z]
                res[z] = np.where(blk < lo, lo, np.where(blk > hi, hi, blk))
    return res
