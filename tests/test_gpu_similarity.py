"""The Appendix D similarity metrics on the GPU (krig_similarity) against the FP64 oracle
(oracle/downstream.py): hand-worked golden images, self-comparison, ragged and degenerate sizes,
a stack of interpolated spine slices against the phantom's noise-free truth."""
import os

import numpy as np
import pytest
import torch

from oracle import downstream as ds
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-9


def _oracle_row(G, R):
    lo, hi = ds.joint_range(G, R)
    return np.array([ds.rmse(G, R), ds.mutual_information(G, R), ds.mutual_information(G, G),
                     ds.entropy_difference(G, R), ds.ssim_global(G, R), ds.entropy(G, lo, hi),
                     ds.entropy(R, lo, hi), np.nan])


def _check(got, G, R):
    exp = _oracle_row(G, R)
    for k in range(7):
        assert got[k] == pytest.approx(exp[k], rel=TOL, abs=1e-12), (binding.SIMILARITY_FIELDS[k], got[k], exp[k])


def _gpu(G, R):
    g = torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).cuda()
    r = torch.from_numpy(np.ascontiguousarray(R, dtype=np.float32)).cuda()
    return binding.similarity(g, r).cpu().numpy()


def test_golden_images():
    for line in open(os.path.join(GOLDEN, "similarity_values.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        metric, g, r, val = [p.strip() for p in line.split("|")]
        G = np.array([[float(v) for v in row.split()] for row in g.split("/")], dtype=np.float32)
        R = np.array([[float(v) for v in row.split()] for row in r.split("/")], dtype=np.float32)
        got = _gpu(G, R)[0]
        k = {"rmse": 0, "mi": 1, "ed": 3, "ssim": 4}[metric]
        assert got[k] == pytest.approx(float(val), abs=1e-12)


@pytest.mark.parametrize("H,W", [(37, 45), (3, 5), (256, 256), (130, 67)])
def test_random_pairs_against_oracle(H, W):
    rng = np.random.default_rng(H * 1000 + W)
    G = (0.3 + 0.5 * rng.random((4, H, W))).astype(np.float32)
    R = (G + 0.05 * rng.normal(size=G.shape)).astype(np.float32)
    got = _gpu(G, R)
    for i in range(G.shape[0]):
        _check(got[i], G[i].astype(np.float64), R[i].astype(np.float64))


def test_self_comparison_and_constant_reconstruction():
    rng = np.random.default_rng(7)
    G = rng.random((50, 60)).astype(np.float32)
    got = _gpu(np.stack([G, G]), np.stack([G, np.full_like(G, 0.5)]))
    assert got[0, 0] == 0.0 and got[0, 3] == 0.0
    assert got[0, 4] == pytest.approx(1.0, abs=1e-12)
    assert got[0, 1] == pytest.approx(got[0, 2], rel=1e-12)   # MI(G, G) = H(G)
    _check(got[1], G.astype(np.float64), np.full(G.shape, 0.5))
    assert got[1, 1] == pytest.approx(0.0, abs=1e-12)         # nothing shared with a constant


def test_interpolated_spine_slices_against_truth():
    """The analogue of the paper's slice comparison: each interpolated slice of the spine phantom
    (DS kriging on the GPU) against the noise-free phantom slice at the same z."""
    vol = phantoms.spine(n=10, H=96, W=112, g=4, k=3, with_truth=True)
    s = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    outs, _ = binding.krige([dict(slices=s, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                                  variogram=vol.variogram(), in_scale=vol.in_scale)])
    miss = [z for z in range(vol.n_out) if z % vol.zfactor]
    R = outs[0][miss].contiguous()
    G = torch.from_numpy(vol.truth[miss].astype(np.float32)).cuda()
    got = binding.similarity(G, R).cpu().numpy()
    Rh = R.double().cpu().numpy()
    Gh = G.double().cpu().numpy()
    for i in (0, len(miss) // 2, len(miss) - 1):
        _check(got[i], Gh[i], Rh[i])
    varied = Gh.reshape(len(miss), -1).std(axis=1) > 0  # slices that cut the anatomy (others are background)
    assert varied.any() and np.median(got[varied, 4]) > 0.9


def test_constant_ground_truth():
    """A ground-truth slice that misses the anatomy is constant: zero variance and covariance exactly
    (two-pass moments), entropy 0, as in the oracle."""
    rng = np.random.default_rng(11)
    G = np.full((64, 32), np.float32(0.1))
    R = (0.1 + 0.01 * rng.normal(size=G.shape)).astype(np.float32)
    got = _gpu(G, R)[0]
    _check(got, G.astype(np.float64), R.astype(np.float64))
    assert got[2] == 0.0 and got[5] == 0.0
