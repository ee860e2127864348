"""GPU parity: every form of the CUDA path against the FP64 oracle, element by element.

Tolerances (written here, derived from the arithmetic): interpolated intensities and
kriging variances within 1e-5 of the oracle, normwise (max |gpu - oracle| <=
1e-5 * max |oracle| per volume); known slices bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu

TOL = 1e-5
FORMS = ["DS", "P64", "PMX"]


def _to_dev(vol, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(vol.slices))
    if dtype is not None and t.dtype != torch.uint16:
        t = t.to(dtype)
    return t.cuda()


def _spec(vol, t, **over):
    d = dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
             variogram=vol.variogram(), in_scale=vol.in_scale)
    d.update(over)
    return d


def _normwise(got, exp):
    return float(np.abs(got - exp).max() / max(np.abs(exp).max(), 1e-300))


def _check_full(vol, form, t=None, flags=0):
    t = _to_dev(vol) if t is None else t
    outs, vars_ = binding.krige([_spec(vol, t)], form=form, want_var=True, flags=flags)
    vals = t.double().cpu().numpy() if t.dtype != torch.uint16 else vol.values_f64()
    exp, evar = oracle.krige_volume(vals, vol.zfactor, vol.half_w, k_sub=vol.n_sub_blocks, **vol.variogram())
    got = outs[0].double().cpu().numpy()
    gvar = vars_[0].double().cpu().numpy()
    g = vol.zfactor
    assert np.array_equal(got[::g], vals), "known slices must be copied bit-exactly"
    assert np.all(gvar[::g] == 0.0)
    e1 = _normwise(got, exp)
    e2 = _normwise(gvar, evar)
    assert e1 <= TOL, "%s estimate normwise error %.3g" % (form, e1)
    assert e2 <= TOL, "%s variance normwise error %.3g" % (form, e2)
    return got, gvar


@pytest.mark.parametrize("form", FORMS)
def test_tiny_ellipsoids_f64(form):
    """9 known 64x64 float64 slices, g 4 (33 output slices), 2 sub-blocks, spherical, 18 points."""
    _check_full(phantoms.tiny_ellipsoids(), form)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_ragged_exponential_r2(form, dtype):
    """Ragged in-plane size (not a tile multiple), 50-point window, exponential model, 3 sub-blocks."""
    vol = phantoms.random_stack(6, 37, 45, 3, 2, k=3, seed=11, model="exponential")
    _check_full(vol, form, _to_dev(vol, dtype))


@pytest.mark.parametrize("form", FORMS)
def test_uint16_spine(form):
    """uint16 storage scaled to float32 (values float32(u) * scale), as the spine stack is stored."""
    vol = phantoms.spine(n=6, H=40, W=72, g=4, k=2)
    _check_full(vol, form)


@pytest.mark.parametrize("form", FORMS)
def test_half_width_zero_and_large_g(form):
    vol = phantoms.random_stack(4, 9, 10, 8, 0, k=1, seed=3)
    _check_full(vol, form)


@pytest.mark.parametrize("form", FORMS)
def test_window_wider_than_volume(form):
    """W, H < 2r+1: every pixel is truncated on both sides."""
    vol = phantoms.random_stack(5, 3, 2, 3, 2, k=2, seed=4)
    _check_full(vol, form)


@pytest.mark.parametrize("form", FORMS)
def test_single_pixel_and_two_slices(form):
    vol = phantoms.random_stack(2, 1, 1, 5, 1, k=1, seed=5)
    _check_full(vol, form)


@pytest.mark.parametrize("form", FORMS)
def test_zfactor_one_is_copy(form):
    vol = phantoms.random_stack(4, 20, 24, 1, 1, k=3, seed=6)
    t = _to_dev(vol)
    outs, _ = binding.krige([_spec(vol, t)], form=form)
    assert torch.equal(outs[0], t)


@pytest.mark.parametrize("g,r,model,nugget", [(2, 1, "spherical", 0.0), (3, 2, "exponential", 0.02),
                                              (5, 2, "spherical", 0.05), (7, 1, "exponential", 0.0),
                                              (8, 2, "exponential", 0.01)])
def test_ds_mirror_split_geometries(g, r, model, nugget):
    """The DS class solve splits each class system into its Z-mirror halves: odd and even g
    (with and without a middle target), g = 2 (no difference system), nugget on and off."""
    vol = phantoms.random_stack(4, 29, 35, g, r, k=2, seed=40 + g, model=model)
    vol.nugget = nugget
    _check_full(vol, "DS")


def test_ds_fp64_solve_flag_matches():
    vol = phantoms.random_stack(5, 40, 70, 6, 2, k=2, seed=7, model="exponential")
    a, _ = _check_full(vol, "DS")
    b, _ = _check_full(vol, "DS", flags=binding.FLAG_DS_FP64_SOLVE)
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()


def test_partition_independence_bit_identical():
    """Algorithm 1: the Z sub-block count changes the schedule, not the result."""
    vol = phantoms.random_stack(9, 50, 66, 3, 1, k=1, seed=8)
    t = _to_dev(vol)
    ref, _ = binding.krige([_spec(vol, t, n_sub_blocks=1)], form="DS")
    for k in (2, 3, 8):
        out, _ = binding.krige([_spec(vol, t, n_sub_blocks=k)], form="DS")
        assert torch.equal(out[0], ref[0])


@pytest.mark.parametrize("form", FORMS)
def test_batched_equals_single(form):
    """Many uneven volumes in one launch give bit-identical results to one launch per volume."""
    vols = [phantoms.random_stack(5, 33, 70, 4, 1, k=2, seed=20),
            phantoms.random_stack(7, 64, 64, 6, 2, k=3, seed=21, model="exponential"),
            phantoms.spine(n=5, H=24, W=40, g=3, k=2),
            phantoms.tiny_ellipsoids(n=4, H=20, W=18, g=2, k=1)]
    ts = [_to_dev(v) for v in vols]
    batch, bvar = binding.krige([_spec(v, t) for v, t in zip(vols, ts)], form=form, want_var=True)
    for v, t, bo, bv in zip(vols, ts, batch, bvar):
        so, sv = binding.krige([_spec(v, t)], form=form, want_var=True)
        assert torch.equal(bo, so[0])
        assert torch.equal(bv, sv[0])


def test_singular_system_reported():
    vol = phantoms.random_stack(3, 8, 8, 2, 1, k=1, seed=9)
    t = _to_dev(vol)
    for form in FORMS:
        with pytest.raises(binding.KrigError) as ei:
            binding.krige([_spec(vol, t, variogram=dict(model="spherical", nugget=0.0, sill=0.0, range=8.0))],
                          form=form)
        assert ei.value.status == binding.KRIG_ESINGULAR


# ---------------------------------------------------------------- full-size cases, sampled
def _sample(nout, H, W, g, count, seed):
    rng = np.random.default_rng(seed)
    z = rng.integers(0, nout, count)
    y = rng.integers(0, H, count)
    x = rng.integers(0, W, count)
    pts = [np.stack([z, y, x], 1)]
    # borders and corners of a few missing slices
    for zz in (1, g // 2 + 1, nout - 2):
        for yy in (0, 1, 2, H - 3, H - 2, H - 1):
            xs = np.arange(W)
            pts.append(np.stack([np.full(W, zz), np.full(W, yy), xs], 1))
        for xx in (0, 1, 2, W - 3, W - 2, W - 1):
            ys = np.arange(H)
            pts.append(np.stack([np.full(H, zz), ys, np.full(H, xx)], 1))
    return np.concatenate(pts).astype(np.int64)


def _check_sampled(vol, form, count=20000):
    t = _to_dev(vol)
    outs, vars_ = binding.krige([_spec(vol, t)], form=form, want_var=True)
    got = outs[0].double().cpu().numpy()
    gvar = vars_[0].double().cpu().numpy()
    vals = vol.values_f64()
    g = vol.zfactor
    assert np.array_equal(got[::g], vals)
    idx = _sample(got.shape[0], vol.H, vol.W, g, count, seed=1)
    est, var = oracle.krige_voxels(vals, g, vol.half_w, idx, **vol.variogram())
    ge = got[idx[:, 0], idx[:, 1], idx[:, 2]]
    gv = gvar[idx[:, 0], idx[:, 1], idx[:, 2]]
    # normwise against the whole oracle volume's scale: the known slices bound it
    scale = max(np.abs(est).max(), np.abs(vals).max())
    assert np.abs(ge - est).max() <= TOL * scale
    assert np.abs(gv - var).max() <= TOL * np.abs(var).max()


@pytest.mark.parametrize("form", FORMS)
def test_spine_full_size_sampled(form):
    """24 known 256x256 uint16 slices, g 4 (93 slices), 4 sub-blocks, 18 points."""
    _check_sampled(phantoms.spine(), form)


@pytest.mark.parametrize("form", ["DS", "PMX", "P64"])
def test_brain_full_size_sampled(form):
    """32 known 512x512 float32 slices, g 6 (187 slices), 8 sub-blocks, exponential, 50 points (the
    plain FP64 form too: its warp-per-voxel 50-point solve at full size)."""
    _check_sampled(phantoms.brain(), form, count=8000)
