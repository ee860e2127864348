"""The seeded synthetic workloads match the configurations they stand in for (shapes, storage
types, Z factors, sub-blocks, windows, variogram models, value structure) and are reproducible.
CPU only; they feed the GPU tests, the oracle and the benchmark alike."""
import numpy as np
import pytest

from paper_2303_09523_gb300 import phantoms


def test_tiny_case():
    v = phantoms.tiny_ellipsoids(with_truth=True)
    assert v.slices.shape == (9, 64, 64) and v.slices.dtype == np.float64
    assert (v.zfactor, v.n_sub_blocks, v.half_w, v.model, v.nugget, v.range) == (4, 2, 1, "spherical", 0.0, 8.0)
    assert v.n_out == 33
    # nested ellipsoids of intensity 0.2 / 0.6 / 1.0 on a zero background, before the noise
    assert set(np.unique(v.truth)) <= {0.0, 0.2, 0.6, 1.0} and len(np.unique(v.truth)) == 4
    assert v.sill == pytest.approx(np.var(v.slices), rel=1e-12)


def test_spine_case():
    v = phantoms.spine()
    assert v.slices.shape == (24, 256, 256) and v.slices.dtype == np.uint16
    assert (v.zfactor, v.n_sub_blocks, v.half_w, v.model) == (4, 4, 1, "spherical")
    assert v.n_out == 93 and v.n_missing == 23 * 3 * 256 * 256
    vals = v.values_f64()
    assert vals.dtype == np.float64 and 0.0 <= vals.min() and vals.max() < 1.5  # u16 times its scale
    assert v.sill == pytest.approx(np.var(vals), rel=1e-12)


def test_brain_case():
    v = phantoms.brain()
    assert v.slices.shape == (32, 512, 512) and v.slices.dtype == np.float32
    assert (v.zfactor, v.n_sub_blocks, v.half_w, v.model) == (6, 8, 2, "exponential")
    assert v.n_out == 187


def test_batch_mix_case():
    vols = phantoms.batch_mix()
    assert len(vols) == 16
    for v in vols:
        assert v.slices.dtype == np.float32
        assert v.H == v.W and 128 <= v.H <= 512 and v.H % 64 == 0
        assert 12 <= v.n <= 40 and 2 <= v.zfactor <= 6 and v.half_w in (1, 2)
        assert 1 <= v.n_sub_blocks <= v.n - 1
    assert {v.half_w for v in vols} == {1, 2}  # 18- and 50-point windows both present
    assert {v.model for v in vols} == {"spherical", "exponential"}


def test_workloads_are_reproducible():
    a, b = phantoms.spine(n=5, H=32, W=40), phantoms.spine(n=5, H=32, W=40)
    assert np.array_equal(a.slices, b.slices) and a.in_scale == b.in_scale
    c = phantoms.spine(n=5, H=32, W=40, seed=123)
    assert not np.array_equal(a.slices, c.slices)
