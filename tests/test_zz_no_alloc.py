"""krig_interpolate_noalloc: the DS interpolation for callers that may not allocate
device memory (their host application owns the device memory pool, or their loop
cannot take cudaMalloc's device-wide synchronisation).  It keeps its scratch in a
static device array inside the library.

Checked through the C ABI against krig_interpolate (the workspace-based entry
point) within the parity tolerance, on two calls in a row with different volumes,
so a stale scratch from the first call must not leak into the second.  The file
is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _noalloc_fn():
    L = binding.lib()
    fn = L.krig_interpolate_noalloc
    fn.argtypes = [ctypes.POINTER(binding.VolumeDesc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _run_noalloc(fn, vol, t, params, check=1):
    code = binding.dtype_code(t.dtype)
    d = binding.VolumeDesc(vol.H, vol.W, vol.n, vol.zfactor, vol.n_sub_blocks, vol.half_w, code, vol.in_scale)
    out = torch.empty((vol.n_out, vol.H, vol.W), dtype=binding.out_dtype(code), device=t.device)
    var = torch.empty((vol.n_out, vol.H, vol.W), dtype=torch.float32, device=t.device)
    st = fn(ctypes.byref(d), t.data_ptr(), out.data_ptr(), var.data_ptr(), params.data_ptr(), check,
            torch.cuda.current_stream().cuda_stream)
    return st, out, var


def _reference(vol, t):
    outs, vars_ = binding.krige([dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w,
                                      n_sub_blocks=vol.n_sub_blocks, variogram=vol.variogram(),
                                      in_scale=vol.in_scale)], form="DS", want_var=True)
    return outs[0], vars_[0]


def test_noalloc_matches_workspace_entry_point_twice():
    fn = _noalloc_fn()
    vols = [phantoms.random_stack(7, 70, 90, 6, 2, k=3, seed=31, model="exponential"),  # 50-point, float32
            phantoms.spine(n=6, H=48, W=64, g=4, k=2)]                                 # 18-point, uint16
    for vol in vols:
        t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
        params = binding.variogram_tensor([vol.variogram()], device=t.device)
        st, out, var = _run_noalloc(fn, vol, t, params)
        assert st == binding.KRIG_OK, binding.lib().krig_last_error()
        torch.cuda.synchronize()
        ref, rvar = _reference(vol, t)
        err = float((out.double() - ref.double()).abs().max() / ref.double().abs().max())
        verr = float((var.double() - rvar.double()).abs().max() / rvar.double().abs().max())
        assert err <= TOL and verr <= TOL
        assert torch.equal(out[::vol.zfactor].double(), ref[::vol.zfactor].double())


def test_noalloc_rejects_volume_beyond_static_scratch():
    fn = _noalloc_fn()
    vol = phantoms.random_stack(4, 32, 32, 4, 2, k=1, seed=32)
    t = torch.from_numpy(vol.slices.astype(np.float64)).cuda()  # float64 with half_w 2: tables exceed 64 KiB
    params = binding.variogram_tensor([vol.variogram()], device=t.device)
    st, _, _ = _run_noalloc(fn, vol, t, params)
    assert st == binding.KRIG_EINVAL
    assert b"scratch" in binding.lib().krig_last_error()


def test_noalloc_reports_singular_then_recovers():
    """A singular variogram (nugget = sill = 0) is reported as KRIG_ESINGULAR; the next call
    in the same shared scratch starts from a cleared status word, returns KRIG_OK and matches
    the workspace entry point."""
    fn = _noalloc_fn()
    vol = phantoms.random_stack(5, 40, 52, 3, 1, k=2, seed=33)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    bad = binding.variogram_tensor([dict(model="spherical", nugget=0.0, sill=0.0, range=8.0)], device=t.device)
    st, _, _ = _run_noalloc(fn, vol, t, bad)
    assert st == binding.KRIG_ESINGULAR
    assert b"singular" in binding.lib().krig_last_error()
    good = binding.variogram_tensor([vol.variogram()], device=t.device)
    st, out, var = _run_noalloc(fn, vol, t, good)
    assert st == binding.KRIG_OK, binding.lib().krig_last_error()
    ref, rvar = _reference(vol, t)
    err = float((out.double() - ref.double()).abs().max() / ref.double().abs().max())
    assert err <= TOL
    assert torch.equal(out[::vol.zfactor], ref[::vol.zfactor])
