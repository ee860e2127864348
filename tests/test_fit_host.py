"""Host-side variogram fitting helpers (no GPU): distance classes of the empirical variogram
and the weighted least-squares model fit."""
import math

import numpy as np
import pytest

from paper_2303_09523_gb300 import fit


@pytest.mark.parametrize("model,theta", [("spherical", (0.05, 0.8, 9.0)), ("exponential", (0.0, 1.3, 4.5))])
def test_wls_recovers_theta_from_exact_curve(model, theta):
    pytest.importorskip("scipy")
    h = np.arange(1.0, 21.0)
    gamma = fit.variogram_model(h, model, *theta)
    n = 1000.0 + 10.0 * h
    r = fit.fit_variogram_wls(h, gamma, n, model)
    assert np.allclose(r["theta"], theta, rtol=1e-6, atol=1e-6)  # nugget 0 sits on its bound
    assert r["cost"] < 1e-10


def test_variogram_model_shapes():
    # spherical reaches nugget + sill at the range and stays there; exponential reaches 95 % of the sill there
    assert fit.variogram_model(6.0, "spherical", 0.1, 1.0, 6.0) == pytest.approx(1.1)
    assert fit.variogram_model(9.0, "spherical", 0.1, 1.0, 6.0) == pytest.approx(1.1)
    assert fit.variogram_model(3.0, "spherical", 0.0, 1.0, 6.0) == pytest.approx(1.5 * 0.5 - 0.5 * 0.125)
    assert fit.variogram_model(6.0, "exponential", 0.0, 1.0, 6.0) == pytest.approx(1.0 - math.exp(-3.0))


def test_variogram_bins_pool_by_rounded_length():
    """L = 1, zfactor 2: in-slice lags of length 1 and sqrt 2 pool into class 1, lags to the next
    slice (lengths 2, sqrt 5, sqrt 6) into class 2; the zero lag is left out."""
    L, g = 1, 2
    q = 2 * L + 1
    rng = np.random.default_rng(3)
    sums = rng.uniform(1.0, 2.0, size=(2, q, q))
    counts = rng.integers(10, 20, size=(2, q, q)).astype(np.int64)
    h, gamma, n = fit.variogram_bins(sums, counts, g)
    assert len(h) == 2
    m0 = np.ones((q, q), bool)
    m0[L, L] = False
    n1, s1 = counts[0][m0].sum(), sums[0][m0].sum()
    len0 = np.sqrt(np.add.outer(np.arange(-L, L + 1) ** 2, np.arange(-L, L + 1) ** 2))
    h1 = (len0[m0] * counts[0][m0]).sum() / n1
    n2, s2 = counts[1].sum(), sums[1].sum()
    h2 = (np.sqrt(len0 ** 2 + g * g) * counts[1]).sum() / n2
    assert np.allclose(n, [n1, n2]) and np.allclose(gamma, [s1 / (2 * n1), s2 / (2 * n2)])
    assert np.allclose(h, [h1, h2])


def test_fit_log_keeps_complete_records_only(tmp_path):
    path = str(tmp_path / "fit.jsonl")
    assert fit.fit_log_last(path) is None
    fit.fit_log_append(path, {"step": 0, "x": 1.5})
    fit.fit_log_append(path, {"step": 1, "x": 2.5})
    with open(path, "a") as f:
        f.write('{"step": 2, "x": 3')  # interrupted mid-write
    assert fit.fit_log_last(path) == {"step": 1, "x": 2.5}


def test_loo_fit_resumes_exactly(tmp_path, monkeypatch):
    """An interrupted fit resumed from its log ends with the same parameters, bit for bit, as an
    uninterrupted one (the loss is replaced by a smooth CPU function of theta here)."""
    torch = pytest.importorskip("torch")

    def fake_loss(slices, th, zfactor, half_w, n_sub_blocks, model):
        return (torch.log(th[2]) - 1.3) ** 2 + (torch.log(th[0] / th[1]) + 2.0) ** 2 + 0.01 * slices.sum()

    monkeypatch.setattr(fit.binding, "loo_loss", fake_loss)
    s = torch.zeros((3, 4, 4), dtype=torch.float64)
    full = fit.fit_variogram_loo(s, 2, 1, 1, "spherical", 0.5, steps=12)
    path = str(tmp_path / "fit.jsonl")
    fit.fit_variogram_loo(s, 2, 1, 1, "spherical", 0.5, steps=5, log_path=path)
    rest = fit.fit_variogram_loo(s, 2, 1, 1, "spherical", 0.5, steps=12, log_path=path, resume=True)
    assert rest["theta"] == full["theta"]
    assert rest["losses"] == full["losses"][5:]
    assert fit.fit_log_last(path)["step"] == 11


def test_wls_range_is_bounded_by_the_observed_lags():
    """A straight line gamma = c h (no sill within the data) drives an unbounded fit off along the
    range-sill ridge; the bounded fit stops at three times the longest class and says so."""
    import numpy as np
    pytest.importorskip("scipy")
    from paper_2303_09523_gb300 import fit
    h = np.arange(1.0, 13.0)
    gamma = 0.01 * h
    n = np.full(h.shape, 1000.0)
    r = fit.fit_variogram_wls(h, gamma, n, "spherical")
    assert r["theta"][2] <= 3.0 * 12.0 + 1e-9 and r["range_at_bound"]
