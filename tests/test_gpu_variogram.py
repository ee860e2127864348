"""GPU empirical variogram (krig_empirical_variogram) against the FP64 oracle.

Per lag vector the squared-increment sums agree with the oracle within 1e-5 relative
(float32 differences and squares, float64 above rows of at most 64 pixels); the pair counts
are exact.  Cases: float32, float64 and uint16 stacks, ragged sizes, lags wider than the
slice, max_lag 0 and 16, one known slice.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu


def _check(vals, t, L, in_scale=1.0):
    sums, counts = binding.empirical_variogram(t, L, in_scale=in_scale)
    torch.cuda.synchronize()
    got = sums.cpu().numpy()
    ref, ref_counts = oracle.empirical_variogram(vals, L)
    assert np.array_equal(counts, ref_counts)
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-12 * scale)
    return got, counts


@pytest.mark.parametrize("n,H,W,L,dtype", [
    (5, 37, 45, 3, torch.float32),     # ragged tiles, W not a multiple of 4
    (4, 70, 131, 8, torch.float32),    # several bands and column tiles
    (3, 16, 64, 16, torch.float64),    # lags as wide as the halo allows
    (2, 5, 6, 8, torch.float32),       # lags wider than the slice: no pairs there
    (6, 33, 20, 0, torch.float32),     # zero lag only: s = 0 sums are 0
    (1, 40, 50, 4, torch.float32),     # one known slice: no s = 1 pairs
])
def test_empirical_variogram_matches_oracle(n, H, W, L, dtype):
    vol = phantoms.random_stack(n, H, W, 2, 1, seed=90 + n + H + L)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dtype).cuda()
    got, counts = _check(t.double().cpu().numpy(), t, L)
    q = 2 * L + 1
    assert got[0, L, L] == 0.0  # zero lag within a slice
    assert np.all(got[counts == 0] == 0.0)


def test_empirical_variogram_uint16_spine():
    vol = phantoms.spine(n=7, H=64, W=96, g=4, k=2)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    assert t.dtype == torch.uint16
    _check(vol.values_f64(), t, 6, in_scale=vol.in_scale)


def test_empirical_variogram_full_spine_at_the_benchmarked_lag():
    """The benchmarked case: the whole spine stack (24 x 256 x 256 uint16), every lag vector up to 8
    (8.6e8 voxel pairs, FP32 row sums then FP64), against the oracle."""
    vol = phantoms.spine()
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    got, counts = _check(vol.values_f64(), t, 8, in_scale=vol.in_scale)
    assert int(counts.sum()) == 860964800


def test_empirical_variogram_rejects_bad_arguments():
    t = torch.zeros((3, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.KrigError):
        binding.empirical_variogram(t, 17)
    with pytest.raises(binding.KrigError):
        binding.empirical_variogram(t, -1)
