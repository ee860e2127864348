"""KRIG_FLAG_CLAMP_BLOCK_MINMAX: the DS estimates clamped to the known range of their Z sub-block,
against the oracle's clamp of its own FP64 estimates (ragged stacks, every input type, and a
full-size sample of the brain stack, whose exponential variogram gives negative weights and so
estimates outside the known range)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _gpu(vol, t, clamp=True):
    outs, _ = binding.krige([dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                                  variogram=vol.variogram(), in_scale=vol.in_scale)], form="DS",
                            flags=binding.FLAG_CLAMP_BLOCK_MINMAX if clamp else 0)
    return outs[0].double().cpu().numpy()


def _binary_stack(dtype, n=7, H=37, W=45, g=2, k=3, seed=82):
    """Random 0 / 1 slices with alternate rows flipped: with a spherical range of 3 some weights are
    negative enough that estimates leave the known range (by up to about 0.1)."""
    rng = np.random.default_rng(seed)
    S = np.where(rng.random((n, H, W)) > 0.5, 1.0, 0.0)
    S[:, ::2, :] = 1.0 - S[:, ::2, :]
    if dtype == torch.uint16:
        u16, scale = phantoms.to_u16(S)
        return phantoms.Volume("binary_u16", u16, g, 1, k, "spherical", 0.0, 0.25, 3.0, in_scale=scale)
    return phantoms.Volume("binary", S.astype(np.float64), g, 2, k, "spherical", 0.0, 0.25, 3.0)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.uint16])
def test_clamped_volume_matches_oracle(dtype):
    vol = _binary_stack(dtype)
    if dtype == torch.uint16:
        t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
        vals = vol.values_f64()
    else:
        t = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dtype).cuda()
        vals = t.double().cpu().numpy()
    got = _gpu(vol, t)
    raw, _ = oracle.krige_volume(vals, vol.zfactor, vol.half_w, k_sub=vol.n_sub_blocks, **vol.variogram())
    exp = oracle.clamp_block_minmax(raw, vals, vol.zfactor, vol.n_sub_blocks)
    assert np.abs(got - exp).max() <= TOL * np.abs(exp).max()
    assert np.array_equal(got[::vol.zfactor], vals)
    assert np.abs(exp - raw).max() > 0.01  # the clamp does change estimates here
    unclamped = _gpu(vol, t, clamp=False)
    assert np.abs(unclamped - raw).max() <= TOL * np.abs(raw).max()


def test_brain_full_size_sampled_clamp():
    vol = phantoms.brain()
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    got = _gpu(vol, t)
    vals = vol.slices.astype(np.float64)
    g, k = vol.zfactor, vol.n_sub_blocks
    a = oracle.sub_blocks(vol.n, k)
    rng = np.random.default_rng(2)
    m = 6000
    j = rng.integers(0, vol.n - 1, m)
    idx = np.stack([j * g + rng.integers(1, g, m), rng.integers(0, vol.H, m), rng.integers(0, vol.W, m)], 1)
    est, _ = oracle.krige_voxels(vals, g, vol.half_w, idx, **vol.variogram())
    b = np.searchsorted(np.array(a), j, side="right") - 1
    lo = np.array([vals[a[i]:a[i + 1] + 1].min() for i in range(k)])[b]
    hi = np.array([vals[a[i]:a[i + 1] + 1].max() for i in range(k)])[b]
    exp = np.where(est < lo, lo, np.where(est > hi, hi, est))
    ge = got[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert np.abs(ge - exp).max() <= TOL * np.abs(vals).max()
