"""Universal kriging on the GPU (plan flags KRIG_FLAG_DRIFT_Z / _XYZ / _SLABS4) against the FP64
oracle's orc_uk_voxels: every drift and neighbourhood, ragged sizes, the first and last gaps of a
four-slice neighbourhood, every input type, full-size samples of the spine and brain stacks, and
the exact reproduction of a linear field by the {1, x, y, z} drift."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu
TOL = 1e-5
DRIFTS = {"constant": 0, "z": binding.FLAG_DRIFT_Z, "xyz": binding.FLAG_DRIFT_XYZ}


def _flags(drift, slabs):
    return DRIFTS[drift] | (binding.FLAG_SLABS4 if slabs == 4 else 0)


def _run(vol, t, drift, slabs):
    return binding.krige([dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                               variogram=vol.variogram(), in_scale=vol.in_scale)], form="DS",
                         want_var=True, flags=_flags(drift, slabs))


def _sample(vol, count, seed):
    rng = np.random.default_rng(seed)
    zs = [z for z in range(vol.n_out) if z % vol.zfactor]
    z = rng.choice(zs, count)
    # always include the first and last gaps and the four borders
    z[:4] = [zs[0], zs[-1], zs[0], zs[-1]]
    y = rng.integers(0, vol.H, count)
    x = rng.integers(0, vol.W, count)
    y[:4] = [0, vol.H - 1, vol.H - 1, 0]
    x[:4] = [0, vol.W - 1, 0, vol.W - 1]
    return np.stack([z, y, x], 1)


def _check(vol, t, drift, slabs, count=1500, seed=0):
    outs, vars_ = _run(vol, t, drift, slabs)
    torch.cuda.synchronize()
    out = outs[0].double().cpu().numpy()
    var = vars_[0].double().cpu().numpy()
    vals = vol.values_f64() if t.dtype == torch.uint16 else t.double().cpu().numpy()
    idx = _sample(vol, count, seed)
    est, s2 = oracle.uk_voxels(vals, vol.zfactor, vol.half_w, idx, slabs=slabs, drift=drift, **vol.variogram())
    got = out[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert np.abs(got - est).max() <= TOL * np.abs(est).max()
    gv = var[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert np.abs(gv - s2).max() <= TOL * np.abs(s2).max()
    known = vals if t.dtype != torch.uint16 else vol.values_f64()
    assert np.array_equal(out[::vol.zfactor], known)
    return out


@pytest.mark.parametrize("drift", ["constant", "z", "xyz"])
@pytest.mark.parametrize("slabs", [2, 4])
@pytest.mark.parametrize("r", [1, 2])
def test_ragged_stacks(drift, slabs, r):
    vol = phantoms.random_stack(6, 37, 45, 3, r, k=2, seed=60 + r, model="exponential" if r == 2 else "spherical")
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    _check(vol, t, drift, slabs, count=800, seed=r)


@pytest.mark.parametrize("n,g", [(2, 3), (3, 2), (4, 5)])
def test_first_and_last_gaps_of_four_slabs(n, g):
    vol = phantoms.random_stack(n, 20, 28, g, 1, k=1, seed=70 + n)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    _check(vol, t, "xyz", 4, count=600, seed=n)


def test_input_types_and_zero_radius():
    vol = phantoms.tiny_ellipsoids(n=5, H=24, W=30, g=4, k=2)
    for dt in (torch.float64, torch.float32):
        t = torch.from_numpy(vol.slices.astype(np.float64)).to(dt).cuda()
        _check(vol, t, "xyz", 4, count=600)
    sp = phantoms.spine(n=5, H=32, W=40, g=3, k=2)
    _check(sp, torch.from_numpy(np.ascontiguousarray(sp.slices)).cuda(), "z", 4, count=600)
    r0 = phantoms.random_stack(5, 16, 24, 4, 0, k=2, seed=75)
    _check(r0, torch.from_numpy(np.ascontiguousarray(r0.slices)).cuda(), "z", 2, count=400)


def test_constant_drift_two_slabs_is_ordinary_kriging():
    vol = phantoms.random_stack(6, 33, 41, 4, 2, k=3, seed=76, model="exponential")
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    uk, _ = _run(vol, t, "constant", 2)
    ok, _ = binding.krige([dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                                variogram=vol.variogram())], form="DS")
    err = (uk[0].double() - ok[0].double()).abs().max() / ok[0].double().abs().max()
    assert float(err) <= TOL


def test_linear_field_reproduced_by_xyz_drift():
    """Kriging with the drift {1, x, y, z} is exact for a field linear in x, y, z (the weights
    reproduce every drift function), here at every missing voxel of a 4-slab stack."""
    n, H, W, g = 7, 40, 52, 4
    z = (np.arange(n) * g)[:, None, None]
    y = np.arange(H)[None, :, None]
    x = np.arange(W)[None, None, :]
    field = (0.3 + 0.01 * x - 0.02 * y + 0.015 * z).astype(np.float64)
    vol = phantoms.random_stack(n, H, W, g, 2, k=2, seed=77)
    vol.slices = field
    t = torch.from_numpy(field).cuda()
    outs, _ = _run(vol, t, "xyz", 4)
    zz = np.arange(vol.n_out)[:, None, None]
    exact = 0.3 + 0.01 * x - 0.02 * y + 0.015 * zz
    assert np.abs(outs[0].double().cpu().numpy() - exact).max() <= 1e-9


@pytest.mark.parametrize("which", ["spine", "brain"])
def test_full_size_sampled(which):
    vol = phantoms.spine() if which == "spine" else phantoms.brain()
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    _check(vol, t, "xyz", 4, count=400 if which == "brain" else 1200, seed=5)
