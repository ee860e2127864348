"""Thin ctypes binding over ``libkrig.so`` (C ABI in ``include/krig.h``).

Argument marshalling only: every step of the kriging path runs in the
library's CUDA kernels.  PyTorch supplies device memory (the workspace and the
caller's tensors) and the CUDA stream.  There is no fallback: if the library
is missing, ``lib()`` raises.
"""
import ctypes
import os
import struct

from . import build as _build

KRIG_OK, KRIG_EINVAL, KRIG_ENOMEM, KRIG_ECUDA, KRIG_ESINGULAR, KRIG_ETIMEOUT, KRIG_EWORKSPACE, KRIG_EUNSUPPORTED = range(8)
STATUS_NAMES = ["KRIG_OK", "KRIG_EINVAL", "KRIG_ENOMEM", "KRIG_ECUDA", "KRIG_ESINGULAR", "KRIG_ETIMEOUT",
                "KRIG_EWORKSPACE", "KRIG_EUNSUPPORTED"]
SPHERICAL, EXPONENTIAL = 0, 1
F64, F32, U16 = 0, 1, 2
FORM_P64, FORM_PMX, FORM_DS = 0, 1, 2
FORMS = {"P64": FORM_P64, "PMX": FORM_PMX, "DS": FORM_DS}
MODELS = {"spherical": SPHERICAL, "exponential": EXPONENTIAL}
FLAG_DS_FP64_SOLVE = 0x1
FLAG_LOO = 0x2
FLAG_DRIFT_Z = 0x4
FLAG_DRIFT_XYZ = 0x8
FLAG_SLABS4 = 0x10
FLAG_CLAMP_BLOCK_MINMAX = 0x20
FLAG_FAULT_TIMEOUT = 0x100
MAX_VOLUMES = 64
TIMING_KINDS = 4


class VolumeDesc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("n_known", ctypes.c_int32),
                ("zfactor", ctypes.c_int32), ("n_sub_blocks", ctypes.c_int32), ("half_w", ctypes.c_int32),
                ("in_dtype", ctypes.c_int32), ("in_scale", ctypes.c_float)]


class Variogram(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("pad", ctypes.c_int32), ("nugget", ctypes.c_double),
                ("sill", ctypes.c_double), ("range", ctypes.c_double)]


class KrigError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libkrig.so.  Raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libkrig.so is not built (%s); run __graft_entry__.build()" % path)
        _build.build()
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.krig_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(VolumeDesc), ctypes.c_int32, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]
    L.krig_plan_create.restype = ctypes.c_int
    L.krig_plan_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.krig_plan_set_workspace.restype = ctypes.c_int
    L.krig_interpolate.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
    L.krig_interpolate.restype = ctypes.c_int
    L.krig_loo_forward.argtypes = [vp, ctypes.POINTER(vp), vp, ctypes.POINTER(vp), vp, vp]
    L.krig_loo_forward.restype = ctypes.c_int
    L.krig_backward.argtypes = [vp, ctypes.POINTER(vp), vp, vp, ctypes.POINTER(vp), vp, ctypes.c_int32, vp]
    L.krig_backward.restype = ctypes.c_int
    L.krig_plan_autotune.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.c_int32, vp,
                                     ctypes.POINTER(ctypes.c_int32)]
    L.krig_plan_autotune.restype = ctypes.c_int
    L.krig_plan_device_status.argtypes = [vp, vp]
    L.krig_plan_device_status.restype = ctypes.c_int
    L.krig_plan_set_timing.argtypes = [vp, ctypes.c_int32]
    L.krig_plan_set_timing.restype = ctypes.c_int
    L.krig_plan_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.krig_plan_get_timing.restype = ctypes.c_int
    L.krig_last_error.argtypes = []
    L.krig_last_error.restype = ctypes.c_char_p
    L.krig_plan_destroy.argtypes = [vp]
    L.krig_plan_destroy.restype = None
    L.krig_measure_fma_peak.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.krig_measure_fma_peak.restype = ctypes.c_int
    L.krig_version.argtypes = []
    L.krig_version.restype = ctypes.c_int32
    L.krig_empirical_variogram.argtypes = [ctypes.POINTER(VolumeDesc), vp, ctypes.c_int32, vp,
                                           ctypes.POINTER(ctypes.c_int64), vp]
    L.krig_empirical_variogram.restype = ctypes.c_int
    L.krig_similarity_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.krig_similarity_workspace_bytes.restype = ctypes.c_size_t
    L.krig_similarity.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_size_t, vp, vp]
    L.krig_similarity.restype = ctypes.c_int
    L.krig_marching_cubes_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.krig_marching_cubes_workspace_bytes.restype = ctypes.c_size_t
    L.krig_marching_cubes.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, vp,
                                      ctypes.c_int64, vp, vp, ctypes.c_size_t, vp]
    L.krig_marching_cubes.restype = ctypes.c_int
    L.krig_marching_cubes_table.argtypes = [ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_uint8)]
    L.krig_marching_cubes_table.restype = None
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.krig_plan_schedule.argtypes = [vp, i32p, i32p]
    L.krig_plan_schedule.restype = ctypes.c_int
    L.krig_plan_set_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    L.krig_plan_set_schedule.restype = ctypes.c_int
    L.krig_plan_variance_table.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), i32p, i32p, i32p, i32p,
                                           vp]
    L.krig_plan_variance_table.restype = ctypes.c_int
    _lib = L
    return L


def _check(st):
    if st != KRIG_OK:
        raise KrigError(st, lib().krig_last_error().decode(errors="replace"))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def dtype_code(torch_dtype):
    import torch
    return {torch.float64: F64, torch.float32: F32, torch.uint16: U16}[torch_dtype]


def variogram_bytes(params) -> bytes:
    """Pack a list of dicts (model, nugget, sill, range) as krig_variogram structs."""
    out = b""
    for p in params:
        m = p["model"]
        m = MODELS[m] if isinstance(m, str) else int(m)
        out += struct.pack("<iiddd", m, 0, float(p["nugget"]), float(p["sill"]), float(p["range"]))
    return out


def variogram_tensor(params, device="cuda"):
    """Device buffer of krig_variogram structs (uint8 tensor, 32 bytes per volume)."""
    import torch
    raw = variogram_bytes(params)
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)


class Plan:
    """A kriging plan over one or more volumes, with a torch-allocated workspace."""

    def __init__(self, descs, form="DS", flags=0, device=None, workspace=True):
        L = lib()
        self._lib = L
        n = len(descs)
        arr = (VolumeDesc * n)()
        for i, d in enumerate(descs):
            arr[i] = VolumeDesc(int(d["H"]), int(d["W"]), int(d["n_known"]), int(d["zfactor"]),
                                int(d["n_sub_blocks"]), int(d["half_w"]), int(d["in_dtype"]),
                                float(d.get("in_scale", 1.0)))
        self.descs = [dict(d) for d in descs]
        self.form = FORMS[form] if isinstance(form, str) else int(form)
        h = ctypes.c_void_p()
        nbytes = ctypes.c_size_t()
        _check(L.krig_plan_create(ctypes.byref(h), arr, n, self.form, flags, ctypes.byref(nbytes)))
        self.handle = h
        self.workspace_bytes = nbytes.value
        self.workspace = None
        if workspace:
            import torch
            dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=dev)
            _check(L.krig_plan_set_workspace(h, _ptr(self.workspace), self.workspace_bytes))

    def interpolate(self, slices, outs, params, variances=None, stream=None):
        n = len(self.descs)
        S = (ctypes.c_void_p * n)(*[t.data_ptr() for t in slices])
        O = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
        V = None
        if variances is not None:
            V = (ctypes.c_void_p * n)(*[(0 if t is None else t.data_ptr()) for t in variances])
        _check(self._lib.krig_interpolate(self.handle, S, O, V, _ptr(params), _stream(stream)))

    def loo_forward(self, slices, params, loss, preds=None, stream=None):
        """Leave-one-slice-out loss per volume into ``loss`` (device float64 [n_vols])."""
        n = len(self.descs)
        S = (ctypes.c_void_p * n)(*[t.data_ptr() for t in slices])
        Pp = None
        if preds is not None:
            Pp = (ctypes.c_void_p * n)(*[(0 if t is None else t.data_ptr()) for t in preds])
        _check(self._lib.krig_loo_forward(self.handle, S, _ptr(params), Pp, _ptr(loss), _stream(stream)))

    def backward(self, slices, params, grad_loss, grad_slices=None, grad_params=None, accumulate=False, stream=None):
        """Gradients of the LOO loss (times grad_loss) w.r.t. slices and (nugget, sill, range)."""
        n = len(self.descs)
        S = (ctypes.c_void_p * n)(*[t.data_ptr() for t in slices])
        G = None
        if grad_slices is not None:
            G = (ctypes.c_void_p * n)(*[(0 if t is None else t.data_ptr()) for t in grad_slices])
        _check(self._lib.krig_backward(self.handle, S, _ptr(params), _ptr(grad_loss), G, _ptr(grad_params),
                                       1 if accumulate else 0, _stream(stream)))

    def autotune(self, slices, outs, params, iters=5, stream=None):
        """Pick the fastest work-item length on this data (bit-identical results); returns it."""
        n = len(self.descs)
        S = (ctypes.c_void_p * n)(*[t.data_ptr() for t in slices])
        O = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
        c = ctypes.c_int32()
        _check(self._lib.krig_plan_autotune(self.handle, S, O, _ptr(params), iters, _stream(stream), ctypes.byref(c)))
        return c.value

    def capture(self, slices, outs, params, variances=None, stream=None):
        """Capture one interpolate call into a CUDA graph; returns the torch.cuda.CUDAGraph.

        Replaying it re-runs the call on the same buffers; new variogram values
        written into ``params`` (device memory) take effect at the next replay.
        """
        import torch
        s = torch.cuda.Stream() if stream is None else stream
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.interpolate(slices, outs, params, variances, s)  # warm-up outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.interpolate(slices, outs, params, variances, s)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def schedule(self):
        """(gaps per work item, stencil blocks per SM; 0 = as many as fit): krig_plan_schedule."""
        c, b = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.krig_plan_schedule(self.handle, ctypes.byref(c), ctypes.byref(b)))
        return c.value, b.value

    def set_schedule(self, chunk, blocks_per_sm=0):
        """Set the DS schedule (krig_plan_set_schedule), e.g. a kept autotune result."""
        _check(self._lib.krig_plan_set_schedule(self.handle, int(chunk), int(blocks_per_sm)))

    def variance_table(self, v=0, stream=None):
        """Volume v's kriging variance by geometry class (krig_plan_variance_table): returns
        (table [ncy, ncx, 8] float32, cx [W] int32, cy [H] int32); the variance of (x, y, j g + t)
        is table[cy[y], cx[x], t - 1]."""
        import numpy as np
        d = self.descs[v]
        ncx, ncy = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.krig_plan_variance_table(self.handle, v, None, None, None, ctypes.byref(ncx), ctypes.byref(ncy),
                                                  _stream(stream)))
        table = np.zeros((ncy.value, ncx.value, 8), dtype=np.float32)
        cx = np.zeros(int(d["W"]), dtype=np.int32)
        cy = np.zeros(int(d["H"]), dtype=np.int32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        _check(self._lib.krig_plan_variance_table(self.handle, v, table.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  cx.ctypes.data_as(i32p), cy.ctypes.data_as(i32p), None, None,
                                                  _stream(stream)))
        return table, cx, cy

    def device_status(self, stream=None):
        _check(self._lib.krig_plan_device_status(self.handle, _stream(stream)))

    def set_timing(self, enable=True):
        _check(self._lib.krig_plan_set_timing(self.handle, 1 if enable else 0))

    def get_timing(self):
        ms = (ctypes.c_double * TIMING_KINDS)()
        cnt = (ctypes.c_int64 * TIMING_KINDS)()
        _check(self._lib.krig_plan_get_timing(self.handle, ms, cnt))
        return list(ms), list(cnt)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.krig_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fma_peak(fp64: bool) -> float:
    """FP32 or FP64 fused multiply-add peak of the current device, GFLOP/s."""
    g = ctypes.c_double()
    _check(lib().krig_measure_fma_peak(1 if fp64 else 0, ctypes.byref(g)))
    return g.value


def empirical_variogram(slices, max_lag, in_scale=1.0, stream=None):
    """Method-of-moments variogram data of a known-slice stack (device tensor n x H x W,
    float64 / float32 / uint16): krig_empirical_variogram.  Returns (sums, counts): sums a
    device float64 tensor [2, 2L+1, 2L+1] of squared increments per lag vector (s, dy, dx),
    counts a numpy int64 array of pair counts in the same layout; gamma = sums / (2 counts)."""
    import numpy as np
    import torch
    if not slices.is_contiguous():
        raise ValueError("slices must be contiguous")
    n, H, W = slices.shape
    d = VolumeDesc(H=H, W=W, n_known=n, zfactor=1, n_sub_blocks=1, half_w=0, in_dtype=dtype_code(slices.dtype),
                   in_scale=in_scale)
    q = max(2 * int(max_lag) + 1, 1)  # an invalid max_lag is rejected by the library
    sums = torch.empty((2, q, q), dtype=torch.float64, device=slices.device)
    counts = np.zeros((2, q, q), dtype=np.int64)
    _check(lib().krig_empirical_variogram(ctypes.byref(d), ctypes.c_void_p(slices.data_ptr()), int(max_lag),
                                          ctypes.c_void_p(sums.data_ptr()),
                                          counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _stream(stream)))
    return sums, counts


SIMILARITY_FIELDS = ("rmse", "mi", "mi_gg", "ed", "ssim", "h_g", "h_r", "h_gr")


def similarity(G, R, stream=None):
    """Appendix D metrics of every image pair of two device float32 stacks (n, H, W) (or single
    images (H, W)): krig_similarity.  Returns a device float64 tensor [n, 8] in the order of
    ``SIMILARITY_FIELDS``."""
    import torch
    if G.shape != R.shape or G.dtype != torch.float32 or R.dtype != torch.float32:
        raise ValueError("G and R must be float32 tensors of one shape")
    G3 = G.contiguous().reshape(-1, G.shape[-2], G.shape[-1])
    R3 = R.contiguous().reshape(-1, R.shape[-2], R.shape[-1])
    n, H, W = G3.shape
    L = lib()
    nb = L.krig_similarity_workspace_bytes(n, H, W)
    work = torch.empty(max(int(nb), 256), dtype=torch.uint8, device=G.device)
    out = torch.empty((n, 8), dtype=torch.float64, device=G.device)
    _check(L.krig_similarity(ctypes.c_void_p(G3.data_ptr()), ctypes.c_void_p(R3.data_ptr()), n, H, W,
                             ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.c_void_p(out.data_ptr()),
                             _stream(stream)))
    return out


def marching_cubes(vol, iso, max_tri=None, stream=None):
    """Iso-surface triangles of a device float32 volume (D, H, W): krig_marching_cubes.  Returns
    (tri, n): tri a device float32 tensor [min(n, max_tri), 3, 3] of vertex (x, y, z), n the number of
    triangles of the surface.  Without ``max_tri`` a first call with no output sizes the buffer."""
    import torch
    v = vol.contiguous()
    if v.dtype != torch.float32 or v.dim() != 3:
        raise ValueError("vol must be a float32 tensor (D, H, W)")
    D, H, W = v.shape
    L = lib()
    nb = L.krig_marching_cubes_workspace_bytes(D, H, W)
    work = torch.empty(max(int(nb), 256), dtype=torch.uint8, device=v.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=v.device)

    def call(buf, m):
        _check(L.krig_marching_cubes(ctypes.c_void_p(v.data_ptr()), D, H, W, float(iso),
                                     None if buf is None else ctypes.c_void_p(buf.data_ptr()), int(m),
                                     ctypes.c_void_p(cnt.data_ptr()), ctypes.c_void_p(work.data_ptr()), work.numel(),
                                     _stream(stream)))

    if max_tri is None:
        call(None, 0)
        max_tri = int(cnt.item())
    tri = torch.empty((max(int(max_tri), 1), 3, 3), dtype=torch.float32, device=v.device)
    call(tri, max_tri)
    n = int(cnt.item())
    return tri[:min(n, int(max_tri))], n


def marching_cubes_table():
    """The case table of the library (numpy int8 [256, 16], uint8 [256])."""
    import numpy as np
    tri = np.zeros((256, 16), dtype=np.int8)
    nt = np.zeros(256, dtype=np.uint8)
    lib().krig_marching_cubes_table(tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                    nt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return tri, nt


def desc_for(slices_shape, zfactor, half_w, n_sub_blocks, dtype_code_, in_scale=1.0):
    n, H, W = slices_shape
    return dict(H=H, W=W, n_known=n, zfactor=zfactor, n_sub_blocks=n_sub_blocks, half_w=half_w,
                in_dtype=dtype_code_, in_scale=in_scale)


def out_dtype(dtype_code_):
    import torch
    return torch.float64 if dtype_code_ == F64 else torch.float32


def krige(volumes, form="DS", want_var=False, flags=0, stream=None):
    """Interpolate a list of volumes in one call.

    ``volumes``: list of dicts with ``slices`` (CUDA tensor, n x H x W of
    float64 / float32 / uint16), ``zfactor``, ``half_w``, ``n_sub_blocks``,
    ``variogram`` (dict) and, for uint16, ``in_scale``.  Returns (outs, vars).
    """
    import torch
    descs, outs, vars_, params = [], [], [], []
    for v in volumes:
        s = v["slices"]
        code = dtype_code(s.dtype)
        d = desc_for(tuple(s.shape), v["zfactor"], v["half_w"], v["n_sub_blocks"], code, v.get("in_scale", 1.0))
        descs.append(d)
        n, H, W = s.shape
        nout = (n - 1) * v["zfactor"] + 1
        outs.append(torch.empty((nout, H, W), dtype=out_dtype(code), device=s.device))
        vars_.append(torch.empty((nout, H, W), dtype=torch.float32, device=s.device) if want_var else None)
        params.append(v["variogram"])
    plan = Plan(descs, form=form, flags=flags, device=volumes[0]["slices"].device)
    pt = variogram_tensor(params, device=volumes[0]["slices"].device)
    plan.interpolate([v["slices"].contiguous() for v in volumes], outs, pt, vars_ if want_var else None, stream)
    plan.device_status(stream)
    plan.close()
    return outs, vars_


def variogram_from_theta(theta, model, device=None):
    """Device krig_variogram buffer (uint8, 32 bytes) from a float64 tensor (nugget, sill, range).

    Argument marshalling with tensor views only: the int32 model code and the
    three doubles are written into one 4-double buffer.
    """
    import torch
    code = MODELS[model] if isinstance(model, str) else int(model)
    buf = torch.zeros(4, dtype=torch.float64, device=device if device is not None else theta.device)
    buf[1:4] = theta.detach().to(torch.float64)
    buf.view(torch.int32)[0] = code
    return buf.view(torch.uint8)


_loo_plans = {}


def _loo_plan(shape, dtype_code_, zfactor, half_w, n_sub_blocks, in_scale, device):
    key = (tuple(shape), dtype_code_, zfactor, half_w, n_sub_blocks, float(in_scale), str(device))
    p = _loo_plans.get(key)
    if p is None:
        d = desc_for(tuple(shape), zfactor, half_w, n_sub_blocks, dtype_code_, in_scale)
        p = Plan([d], form="DS", flags=FLAG_LOO, device=device)
        _loo_plans[key] = p
    return p


def _make_loo_function():
    import torch

    class KrigLOO(torch.autograd.Function):
        """Leave-one-slice-out MSE of the kriging interpolator, differentiable w.r.t. the slices
        (float32 / float64 tensors) and theta = (nugget, sill, range) (float64 tensor)."""

        @staticmethod
        def forward(ctx, slices, theta, zfactor, half_w, n_sub_blocks, model):
            code = dtype_code(slices.dtype)
            s = slices.contiguous()
            plan = _loo_plan(s.shape, code, zfactor, half_w, n_sub_blocks, 1.0, s.device)
            params = variogram_from_theta(theta, model, s.device)
            loss = torch.empty(1, dtype=torch.float64, device=s.device)
            plan.loo_forward([s], params, loss)
            ctx.save_for_backward(s, params)
            ctx.plan = plan
            ctx.slices_dtype = slices.dtype
            return loss[0]

        @staticmethod
        def backward(ctx, grad_out):
            s, params = ctx.saved_tensors
            plan = ctx.plan
            gl = grad_out.detach().to(torch.float64).reshape(1).contiguous()
            gs = torch.empty(s.shape, dtype=torch.float32, device=s.device) if ctx.needs_input_grad[0] else None
            gp = torch.empty(3, dtype=torch.float64, device=s.device) if ctx.needs_input_grad[1] else None
            plan.backward([s], params, gl, [gs] if gs is not None else None, gp)
            if gs is not None:
                gs = gs.to(ctx.slices_dtype)
            return gs, gp, None, None, None, None

    return KrigLOO


_KrigLOO = None


def loo_loss(slices, theta, zfactor, half_w, n_sub_blocks=1, model="spherical"):
    """Differentiable leave-one-slice-out loss (torch.autograd)."""
    global _KrigLOO
    if _KrigLOO is None:
        _KrigLOO = _make_loo_function()
    return _KrigLOO.apply(slices, theta, zfactor, half_w, n_sub_blocks, model)
