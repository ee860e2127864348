"""Marching cubes on the GPU (krig_marching_cubes) against the FP64 oracle (oracle/downstream.py):
the same triangles in the same order, vertices within float32 rounding, on closed surfaces,
random fields with every corner configuration, a kriged phantom volume, ragged and degenerate
sizes and a truncated output buffer."""
import numpy as np
import pytest
import torch

from oracle import downstream as ds
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu


def _compare(vol, iso):
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    exp = ds.marching_cubes(vol, np.float32(iso))
    tri, n = binding.marching_cubes(torch.from_numpy(vol).cuda(), float(np.float32(iso)))
    got = tri.double().cpu().numpy()
    assert n == len(exp) and got.shape == exp.shape
    # float32 vertex arithmetic against the FP64 oracle: half an ulp of the largest coordinate
    assert np.abs(got - exp).max() <= 1e-6 * max(vol.shape) + 1e-7
    return got, exp


def test_sphere_and_torus():
    z, y, x = np.mgrid[0:30, 0:33, 0:35].astype(np.float64)
    _compare(9.0 - np.sqrt((x - 17.2) ** 2 + (y - 16.1) ** 2 + (z - 14.6) ** 2), 0.0)
    q = np.sqrt((x - 17.5) ** 2 + (y - 16.5) ** 2) - 10.0
    got, _ = _compare(3.5 - np.sqrt(q ** 2 + (z - 14.5) ** 2), 0.0)
    assert ds.mesh_signed_volume(got) > 0


@pytest.mark.parametrize("shape,seed", [((12, 13, 14), 1), ((2, 2, 2), 2), ((3, 5, 7), 3), ((40, 2, 9), 4),
                                        ((9, 37, 70), 5)])
def test_random_fields(shape, seed):
    rng = np.random.default_rng(seed)
    _compare(rng.random(shape), 0.5)


def test_kriged_phantom_volume():
    vol = phantoms.tiny_ellipsoids(n=6, H=40, W=44, g=3, k=2)
    s = torch.from_numpy(vol.slices.astype(np.float32)).cuda()
    outs, _ = binding.krige([dict(slices=s, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                                  variogram=vol.variogram())])
    v = outs[0].cpu().numpy()
    for iso in (0.1, 0.4, 0.8):
        _compare(v, iso)


def test_constant_volume_and_truncated_buffer():
    tri, n = binding.marching_cubes(torch.full((5, 6, 7), 0.3, device="cuda"), 0.5)
    assert n == 0 and tri.shape[0] == 0
    rng = np.random.default_rng(9)
    vol = torch.from_numpy(rng.random((10, 11, 12)).astype(np.float32)).cuda()
    full, n = binding.marching_cubes(vol, 0.5)
    part, n2 = binding.marching_cubes(vol, 0.5, max_tri=n // 3)
    assert n2 == n and part.shape[0] == n // 3
    assert torch.equal(part, full[:n // 3])
