"""Pins for the FP64 oracle: each test checks it against something the paper or the
mathematics fixes, never against a retyped copy of its own formula.

Passages: Sec. 4.1.2 (weighted linear sum, minimum error variance, unbiasedness),
Appendix A (extended system with Lagrange multiplier; p = 1, q_1 = 1 gives ordinary
kriging), Algorithm 1 (Z sub-blocks, NaN-padded partial matrix, merge by offsets).
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_variogram():
    rows = []
    with open(os.path.join(GOLDEN, "variogram_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            m, nug, sill, rng, h, val = line.split()
            rows.append((m, float(nug), float(sill), float(rng), float(h), float(val)))
    return rows


SPH = dict(model="spherical", nugget=0.0, sill=1.0, range=8.0)


# ---------------------------------------------------------------- variogram
@pytest.mark.parametrize("row", _golden_variogram())
def test_variogram_golden(row):
    m, nug, sill, rng, h, val = row
    assert oracle.gamma(h, model=m, nugget=nug, sill=sill, range=rng) == pytest.approx(val, abs=1e-15)


@pytest.mark.parametrize("model", ["spherical", "exponential", "linear"])
def test_variogram_gradient_fd(model):
    vg = dict(model=model, nugget=0.05, sill=1.3, range=7.0)
    for h in (0.5, 1.0, 3.0, 6.5, 9.0):
        d = oracle.gamma_grad(h, **vg)
        for p, key in enumerate(("nugget", "sill", "range")):
            e = 1e-6
            hi = dict(vg); hi[key] += e
            lo = dict(vg); lo[key] -= e
            fd = (oracle.gamma(h, **hi) - oracle.gamma(h, **lo)) / (2 * e)
            assert d[p] == pytest.approx(fd, rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- solver
def test_gauss_solve_matches_lapack():
    rng = np.random.default_rng(1)
    for m in (2, 5, 19, 51):
        A = rng.normal(size=(m, m))
        A[-1, -1] = 0.0  # bordered systems have a zero corner: pivoting is required
        B = rng.normal(size=(m, 3))
        x = oracle.gauss_solve(A, B)
        assert np.allclose(x, np.linalg.solve(A, B), rtol=1e-9, atol=1e-9)


def test_gauss_solve_singular():
    with pytest.raises(oracle.OracleError):
        oracle.gauss_solve(np.zeros((3, 3)), np.ones(3))
    with pytest.raises(oracle.OracleError):
        oracle.gauss_solve([[1.0, 2.0], [2.0, 4.0]], [1.0, 1.0])


# ---------------------------------------------------------------- P1 datum
def test_datum_reproduction_zero_nugget():
    """Kriging is an exact interpolator at zero nugget: at a datum w = e_i, mu = 0, var = 0."""
    pts = np.array([[dx, dy, dz] for dz in (-2.0, 2.0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], float)
    for i in (0, 4, 13):
        for vg in (SPH, dict(model="exponential", nugget=0.0, sill=0.7, range=5.0)):
            res = oracle.ok_solve(pts, pts[i], **vg)
            e = np.zeros(len(pts)); e[i] = 1.0
            assert np.abs(res["w"] - e).max() < 1e-12
            assert abs(res["mu"]) < 1e-12
            assert abs(res["var"]) < 1e-12


# ---------------------------------------------------------------- P2 two-point closed form
def _gamma_table(model, nugget, sill, rng):
    t = {}
    for m, nug, s, a, h, val in _golden_variogram():
        if (m, nug, s, a) == (model, nugget, sill, rng):
            t[h] = val
    return t


def test_two_point_closed_form():
    """K = 2 (r = 0): w_lower = 1/2 + (gamma(g-t) - gamma(t)) / (2 gamma(g)), from the 3x3 bordered system."""
    gam = _gamma_table("spherical", 0.0, 1.0, 8.0)
    g = 4
    for t in (1, 2, 3):
        wl = 0.5 + (gam[float(g - t)] - gam[float(t)]) / (2 * gam[float(g)])
        mu = gam[float(g - t)] - gam[float(g)] * wl
        var = wl * gam[float(t)] + (1 - wl) * gam[float(g - t)] + mu
        pts = np.array([[0, 0, -t], [0, 0, g - t]], float)
        res = oracle.ok_solve(pts, [0, 0, 0], **SPH)
        assert res["w"][0] == pytest.approx(wl, abs=1e-14)
        assert res["w"][1] == pytest.approx(1 - wl, abs=1e-14)
        assert res["mu"] == pytest.approx(mu, abs=1e-14)
        assert res["var"] == pytest.approx(var, abs=1e-14)


def test_two_point_volume_indexing():
    """Through the whole-volume path with r = 0 each missing voxel is w_l S_j + w_u S_j+1."""
    gam = _gamma_table("spherical", 0.0, 1.0, 8.0)
    g = 4
    rng = np.random.default_rng(3)
    s = rng.random((4, 5, 7))
    out, var = oracle.krige_volume(s, g, 0, k_sub=2, **SPH)
    for j in range(3):
        assert np.array_equal(out[j * g], s[j])
        for t in range(1, g):
            wl = 0.5 + (gam[float(g - t)] - gam[float(t)]) / (2 * gam[float(g)])
            assert np.allclose(out[j * g + t], wl * s[j] + (1 - wl) * s[j + 1], atol=1e-13)
    assert np.array_equal(out[3 * g], s[3])
    assert np.all(var[::g] == 0.0)


# ---------------------------------------------------------------- P3 pure nugget
def test_pure_nugget_is_window_mean():
    """Range < 1: every lag >= 1 sits on the sill, so w_i = 1/K and the estimate is the window mean.

    With c = nugget + sill: mu = c/K and var = c + c/K.  Checks the neighbourhood window,
    its truncation at the in-plane border, and both bracketing slices.
    """
    vg = dict(model="spherical", nugget=0.2, sill=0.8, range=0.5)
    c = 1.0
    rng = np.random.default_rng(4)
    n, H, W, g = 3, 6, 8, 3
    s = rng.random((n, H, W))
    for r in (1, 2):
        out, var = oracle.krige_volume(s, g, r, k_sub=1, **vg)
        for j in range(n - 1):
            for t in range(1, g):
                for y in range(H):
                    for x in range(W):
                        y0, y1, x0, x1 = max(0, y - r), min(H, y + r + 1), max(0, x - r), min(W, x + r + 1)
                        win = np.concatenate([s[j, y0:y1, x0:x1].ravel(), s[j + 1, y0:y1, x0:x1].ravel()])
                        K = win.size
                        assert out[j * g + t, y, x] == pytest.approx(win.mean(), abs=1e-13)
                        assert var[j * g + t, y, x] == pytest.approx(c + c / K, abs=1e-13)


# ---------------------------------------------------------------- P4 linear variogram
def test_linear_variogram_is_linear_interpolation():
    """gamma(h) = h with K = 2 gives w_lower = 1 - t/g: plain linear interpolation along Z."""
    rng = np.random.default_rng(5)
    for g in (2, 3, 4, 6):
        s = rng.random((5, 4, 6))
        out, _ = oracle.krige_volume(s, g, 0, k_sub=2, model="linear", nugget=0.0, sill=1.0, range=1.0)
        for j in range(4):
            for t in range(g + 1):
                exp = (1 - t / g) * s[j] + (t / g) * s[j + 1]
                assert np.allclose(out[j * g + t], exp, atol=1e-13)


# ---------------------------------------------------------------- P5, P6 invariants
def test_weights_sum_to_one():
    rng = np.random.default_rng(6)
    for _ in range(20):
        K = int(rng.integers(2, 40))
        pts = rng.integers(-3, 4, size=(K, 3)).astype(float)
        pts = np.unique(pts, axis=0)
        s0 = rng.normal(size=3) * 0.3
        vg = dict(model=rng.choice(["spherical", "exponential"]), nugget=float(rng.random() * 0.1),
                  sill=float(0.5 + rng.random()), range=float(2 + rng.random() * 8))
        res = oracle.ok_solve(pts, s0, **vg)
        assert abs(res["w"].sum() - 1.0) < 1e-12


def test_constant_field():
    s = np.full((5, 9, 11), 0.37)
    for model in ("spherical", "exponential"):
        out, _ = oracle.krige_volume(s, 3, 2, k_sub=2, model=model, nugget=0.0, sill=1.0, range=6.0)
        assert np.abs(out - 0.37).max() < 1e-13


# ---------------------------------------------------------------- P7 optimality (definition of kriging)
def _est_variance(w, pts, s0, vg):
    """Var(zhat - Z(s0)) for sum(w) = 1: 2 sum w_i gamma(s_i - s0) - sum_ij w_i w_j gamma(s_i - s_j)."""
    K = len(w)
    G = np.array([[oracle.gamma(np.linalg.norm(pts[i] - pts[j]), **vg) for j in range(K)] for i in range(K)])
    g0 = np.array([oracle.gamma(np.linalg.norm(pts[i] - s0), **vg) for i in range(K)])
    return 2 * w @ g0 - w @ G @ w


def test_weights_minimise_estimation_variance():
    """Sec. 4.1.2: the weights minimise the error variance subject to sum(w) = 1.

    The oracle's variance must equal the estimation variance at its weights, and any
    perturbation that keeps sum(w) = 1 must not lower it.
    """
    rng = np.random.default_rng(7)
    pts = np.array([[dx, dy, dz] for dz in (-2.0, 3.0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], float)
    for vg in (SPH, dict(model="exponential", nugget=0.05, sill=1.2, range=6.0)):
        for s0 in ([0, 0, 0], [0.4, -0.3, 0.5]):
            s0 = np.array(s0, float)
            res = oracle.ok_solve(pts, s0, **vg)
            v0 = _est_variance(res["w"], pts, s0, vg)
            assert res["var"] == pytest.approx(v0, rel=1e-10, abs=1e-13)
            for _ in range(50):
                d = rng.normal(size=len(pts)) * 0.05
                d -= d.mean()
                assert _est_variance(res["w"] + d, pts, s0, vg) >= v0 - 1e-13


def test_covariance_form_equivalence():
    """Appendix A writes the system with covariances C = C(0) - gamma and multiplier phi = -mu."""
    pts = np.array([[dx, dy, dz] for dz in (-1.0, 4.0) for dy in (-2, 0, 2) for dx in (-2, -1, 0, 1, 2)], float)
    vg = dict(model="exponential", nugget=0.1, sill=0.9, range=7.0)
    s0 = np.zeros(3)
    K = len(pts)
    c00 = vg["nugget"] + vg["sill"]
    C = np.array([[c00 - oracle.gamma(np.linalg.norm(pts[i] - pts[j]), **vg) for j in range(K)] for i in range(K)])
    c0 = np.array([c00 - oracle.gamma(np.linalg.norm(p - s0), **vg) for p in pts])
    Cext = np.block([[C, np.ones((K, 1))], [np.ones((1, K)), np.zeros((1, 1))]])
    lam = np.linalg.solve(Cext, np.append(c0, 1.0))
    res = oracle.ok_solve(pts, s0, **vg)
    assert np.allclose(res["w"], lam[:K], atol=1e-12)
    assert res["mu"] == pytest.approx(-lam[K], abs=1e-12)
    assert res["var"] == pytest.approx(c00 - lam[:K] @ c0 - lam[K], abs=1e-12)


# ---------------------------------------------------------------- P8 symmetry
def test_d4_and_z_reversal():
    rng = np.random.default_rng(8)
    s = rng.random((4, 7, 7))
    vg = dict(model="exponential", nugget=0.0, sill=1.0, range=8.0)
    g, r = 3, 2
    ref, _ = oracle.krige_volume(s, g, r, **vg)
    for f_in, f_out in (
        (lambda a: a[:, :, ::-1], lambda a: a[:, :, ::-1]),
        (lambda a: a[:, ::-1, :], lambda a: a[:, ::-1, :]),
        (lambda a: a.transpose(0, 2, 1), lambda a: a.transpose(0, 2, 1)),
        (lambda a: a[::-1], lambda a: a[::-1]),
    ):
        out, _ = oracle.krige_volume(np.ascontiguousarray(f_in(s)), g, r, **vg)
        assert np.abs(out - f_out(ref)).max() < 1e-12


def test_z_reversal_weights():
    """w_t[lower] = w_{g-t}[upper] for the same in-plane offsets."""
    g = 5
    lower = [[dx, dy, 0.0] for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    for t in range(1, g):
        pa = np.array([[p[0], p[1], -t] for p in lower] + [[p[0], p[1], g - t] for p in lower])
        pb = np.array([[p[0], p[1], -(g - t)] for p in lower] + [[p[0], p[1], t] for p in lower])
        wa = oracle.ok_solve(pa, [0, 0, 0], **SPH)["w"]
        wb = oracle.ok_solve(pb, [0, 0, 0], **SPH)["w"]
        assert np.allclose(wa[:9], wb[9:], atol=1e-13)
        assert np.allclose(wa[9:], wb[:9], atol=1e-13)


# ---------------------------------------------------------------- P9 partition independence
def test_subblock_partition_independence():
    """Algorithm 1: results do not depend on the number of Z sub-blocks (bit-identical)."""
    rng = np.random.default_rng(9)
    s = rng.random((9, 6, 5))
    ref, rv = oracle.krige_volume(s, 3, 1, k_sub=1, **SPH)
    for k in (2, 3, 4, 8):
        out, var = oracle.krige_volume(s, 3, 1, k_sub=k, **SPH)
        assert np.array_equal(out, ref)
        assert np.array_equal(var, rv)


def test_voxels_match_volume():
    rng = np.random.default_rng(10)
    s = rng.random((5, 9, 10))
    out, var = oracle.krige_volume(s, 4, 2, k_sub=2, model="exponential", nugget=0.0, sill=1.0, range=8.0)
    idx = np.stack([rng.integers(0, out.shape[0], 40), rng.integers(0, 9, 40), rng.integers(0, 10, 40)], 1)
    est, v = oracle.krige_voxels(s, 4, 2, idx, model="exponential", nugget=0.0, sill=1.0, range=8.0)
    assert np.array_equal(est, out[idx[:, 0], idx[:, 1], idx[:, 2]])
    assert np.array_equal(v, var[idx[:, 0], idx[:, 1], idx[:, 2]])


def test_invalid_arguments():
    s = np.zeros((3, 4, 4))
    with pytest.raises(oracle.OracleError):
        oracle.krige_volume(s, 2, 1, k_sub=3, **SPH)  # more blocks than gaps
    with pytest.raises(oracle.OracleError):
        oracle.krige_volume(s, 2, 1, model="spherical", nugget=0.0, sill=0.0, range=8.0)  # gamma == 0: singular


# ---------------------------------------------------------------- LOO loss and gradients
def test_loo_linear_midpoint():
    """Linear variogram, K = 2: each interior slice is predicted by the midpoint of its neighbours."""
    rng = np.random.default_rng(11)
    s = rng.random((6, 5, 4))
    res = oracle.loo(s, 3, 0, want_pred=True, model="linear", nugget=0.0, sill=1.0, range=1.0)
    mid = 0.5 * (s[:-2] + s[2:])
    assert np.allclose(res["pred"], mid, atol=1e-13)
    assert res["loss"] == pytest.approx(np.mean((mid - s[1:-1]) ** 2), rel=1e-12)


def _loo_fd_theta(s, g, r, vg, key, h):
    hi = dict(vg); hi[key] += h
    lo = dict(vg); lo[key] -= h
    return (oracle.loo(s, g, r, **hi)["loss"] - oracle.loo(s, g, r, **lo)["loss"]) / (2 * h)


@pytest.mark.parametrize("model", ["spherical", "exponential"])
def test_loo_grad_theta_fd(model):
    rng = np.random.default_rng(12)
    s = rng.random((5, 8, 9))
    vg = dict(model=model, nugget=0.03, sill=0.8, range=5.0)
    res = oracle.loo(s, 2, 1, want_grad_theta=True, **vg)
    for p, key in enumerate(("nugget", "sill", "range")):
        fd = _loo_fd_theta(s, 2, 1, vg, key, 1e-3)
        assert res["grad_theta"][p] == pytest.approx(fd, rel=1e-4, abs=1e-9)


def test_loo_grad_slices_fd():
    """L is quadratic in S, so a central difference is exact up to rounding."""
    rng = np.random.default_rng(13)
    s = rng.random((5, 7, 6))
    vg = dict(model="spherical", nugget=0.0, sill=1.0, range=6.0)
    res = oracle.loo(s, 3, 1, want_grad_slices=True, **vg)
    for _ in range(25):
        m, y, x = int(rng.integers(0, 5)), int(rng.integers(0, 7)), int(rng.integers(0, 6))
        h = 1e-3
        sp = s.copy(); sp[m, y, x] += h
        sm = s.copy(); sm[m, y, x] -= h
        fd = (oracle.loo(sp, 3, 1, **vg)["loss"] - oracle.loo(sm, 3, 1, **vg)["loss"]) / (2 * h)
        assert res["grad_slices"][m, y, x] == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_loo_grad_homogeneity():
    """Weights are 0-homogeneous in (nugget, sill): nugget dL/dnugget + sill dL/dsill = 0;
    at zero nugget they do not depend on the sill at all."""
    rng = np.random.default_rng(14)
    s = rng.random((6, 8, 8))
    vg = dict(model="spherical", nugget=0.07, sill=0.9, range=6.0)
    gt = oracle.loo(s, 3, 1, want_grad_theta=True, **vg)["grad_theta"]
    assert abs(vg["nugget"] * gt[0] + vg["sill"] * gt[1]) < 1e-12 * max(1.0, np.abs(gt).max())
    vg0 = dict(vg, nugget=0.0)
    gt0 = oracle.loo(s, 3, 1, want_grad_theta=True, **vg0)["grad_theta"]
    assert abs(gt0[1]) < 1e-14


# ---------------------------------------------------------------------------
# empirical variogram (method-of-moments semivariogram of the known slices)
# ---------------------------------------------------------------------------
def test_empirical_variogram_brute_force():
    S = np.random.default_rng(11).normal(size=(3, 5, 7))
    L = 2
    sums, counts = oracle.empirical_variogram(S, L)
    n, H, W = S.shape
    for s in (0, 1):
        for dy in range(-L, L + 1):
            for dx in range(-L, L + 1):
                tot, cnt = 0.0, 0
                for k in range(n - s):
                    for y in range(H):
                        for x in range(W):
                            if 0 <= y + dy < H and 0 <= x + dx < W:
                                tot += (S[k, y, x] - S[k + s, y + dy, x + dx]) ** 2
                                cnt += 1
                assert counts[s, dy + L, dx + L] == cnt
                assert sums[s, dy + L, dx + L] == pytest.approx(tot, rel=1e-12, abs=1e-300)


def test_empirical_variogram_linear_ramp_closed_form():
    """S = a x + b y + c k: every pair at lag (dx, dy, s) differs by a dx + b dy + c s, so
    gamma = (a dx + b dy + c s)^2 / 2 and the counts are (n - s)(H - |dy|)(W - |dx|)."""
    n, H, W, L = 4, 9, 11, 3
    a, b, c = 0.7, -0.3, 1.9
    k, y, x = np.meshgrid(np.arange(n), np.arange(H), np.arange(W), indexing="ij")
    S = a * x + b * y + c * k
    sums, counts = oracle.empirical_variogram(S, L)
    for s in (0, 1):
        for dy in range(-L, L + 1):
            for dx in range(-L, L + 1):
                N = (n - s) * (H - abs(dy)) * (W - abs(dx))
                assert counts[s, dy + L, dx + L] == N
                gam = sums[s, dy + L, dx + L] / (2 * N)
                assert gam == pytest.approx((a * dx + b * dy + c * s) ** 2 / 2, rel=1e-12, abs=1e-12)


def test_empirical_variogram_constant_and_symmetry():
    n, H, W, L = 3, 6, 5, 2
    sums, counts = oracle.empirical_variogram(np.full((n, H, W), 3.25), L)
    assert np.all(sums == 0.0) and np.all(counts > 0)
    S = np.random.default_rng(12).normal(size=(n, H, W))
    sums, _ = oracle.empirical_variogram(S, L)
    # within one slice the pair sets of (dx, dy) and (-dx, -dy) are the same pairs
    assert np.allclose(sums[0], sums[0][::-1, ::-1], rtol=1e-12, atol=0)
    assert sums[0, L, L] == 0.0  # zero lag
    # lags past the slice give no pairs
    sums, counts = oracle.empirical_variogram(np.zeros((2, 2, 3)), 3)
    assert counts[0, 3, 0] == 0 and counts[0, 3 + 2, 3] == 0 and counts[1, 3, 3] == 2 * 3


# ---------------------------------------------------------------------------
# universal kriging / kriging with external drift (Appendix A, p > 1)
# ---------------------------------------------------------------------------
_UK_VG = [dict(model="spherical", nugget=0.0, sill=1.0, range=6.0),
          dict(model="exponential", nugget=0.05, sill=0.8, range=4.0)]


def _uk_points(seed, K=14):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(-3.0, 3.0, size=(K, 3))
    s0 = rng.uniform(-1.0, 1.0, size=3)
    return pts, s0


@pytest.mark.parametrize("vg", _UK_VG)
def test_uk_constant_drift_is_ordinary_kriging(vg):
    pts, s0 = _uk_points(21)
    vals = np.random.default_rng(22).normal(size=len(pts))
    o = oracle.ok_solve(pts, s0, vals, **vg)
    u = oracle.uk_solve(pts, s0, "constant", vals, **vg)
    assert np.array_equal(o["w"], u["w"]) and o["est"] == u["est"]
    assert u["var"] == pytest.approx(o["var"], rel=1e-13) and u["mu"][0] == pytest.approx(o["mu"], rel=1e-13)


@pytest.mark.parametrize("vg", _UK_VG)
def test_uk_reproduces_its_drift_and_honours_the_constraints(vg):
    pts, s0 = _uk_points(23)
    lin = lambda p: 1.5 + 0.7 * p[..., 0] - 0.4 * p[..., 1] + 2.1 * p[..., 2]
    zlin = lambda p: -0.3 + 1.7 * p[..., 2]
    u = oracle.uk_solve(pts, s0, "xyz", lin(pts), **vg)
    assert u["est"] == pytest.approx(lin(s0), abs=1e-11)
    F = np.column_stack([np.ones(len(pts)), pts])
    assert np.allclose(F.T @ u["w"], np.concatenate([[1.0], s0]), atol=1e-12)
    uz = oracle.uk_solve(pts, s0, "z", zlin(pts), **vg)
    assert uz["est"] == pytest.approx(zlin(s0), abs=1e-11)
    assert np.allclose(np.column_stack([np.ones(len(pts)), pts[:, 2]]).T @ uz["w"], [1.0, s0[2]], atol=1e-12)
    # the z drift alone does not reproduce a trend in x: the drift terms matter
    xlin = lambda p: 2.0 * p[..., 0]
    assert abs(oracle.uk_solve(pts, s0, "z", xlin(pts), **vg)["est"] - xlin(s0)) > 1e-6


@pytest.mark.parametrize("vg", _UK_VG)
@pytest.mark.parametrize("drift", ["z", "xyz"])
def test_uk_weights_minimise_the_estimation_variance(vg, drift):
    """Under the constraints F'w = f0 (with sum w = 1), the estimation variance in the variogram
    form is 2 w'gamma0 - w'Gamma w; the solver's weights give its minimum, equal to w'gamma0 + mu'f0,
    and every feasible perturbation raises it."""
    pts, s0 = _uk_points(24)
    u = oracle.uk_solve(pts, s0, drift, None, **vg)
    K = len(pts)
    G = np.array([[oracle.gamma(np.linalg.norm(pts[i] - pts[j]), **vg) for j in range(K)] for i in range(K)])
    g0 = np.array([oracle.gamma(np.linalg.norm(pts[i] - s0), **vg) for i in range(K)])
    var = lambda w: 2.0 * w @ g0 - w @ G @ w
    assert var(u["w"]) == pytest.approx(u["var"], rel=1e-10)
    F = np.column_stack([np.ones(K), pts[:, 2]]) if drift == "z" else np.column_stack([np.ones(K), pts])
    _, _, Vt = np.linalg.svd(F.T)
    null = Vt[F.shape[1]:]  # directions with F'v = 0
    rng = np.random.default_rng(25)
    for _ in range(20):
        v = null.T @ rng.normal(size=null.shape[0])
        assert var(u["w"] + 0.05 * v) > var(u["w"])


@pytest.mark.parametrize("slabs", [2, 4])
def test_uk_voxels_reproduce_a_linear_volume(slabs):
    """A stack sampled from a + b x + c y + d z (known slice j at z = j g) is reproduced at every
    missing voxel by the {1, x, y, z} drift, including gaps at the stack ends where the 4-slice
    neighbourhood is truncated; known slices are copied."""
    n, H, W, g, r = 5, 7, 8, 3, 1
    k, y, x = np.meshgrid(np.arange(n), np.arange(H), np.arange(W), indexing="ij")
    f = lambda z, yy, xx: 0.4 + 0.11 * xx - 0.07 * yy + 0.05 * z
    S = f(k * g, y, x)
    zz, yy, xx = np.meshgrid(np.arange((n - 1) * g + 1), np.arange(H), np.arange(W), indexing="ij")
    zyx = np.stack([zz.ravel(), yy.ravel(), xx.ravel()], 1)
    est, var = oracle.uk_voxels(S, g, r, zyx, slabs=slabs, drift="xyz", model="exponential", nugget=0.02,
                                sill=1.0, range=5.0)
    assert np.allclose(est, f(zyx[:, 0], zyx[:, 1], zyx[:, 2]), atol=1e-10)
    known = zyx[:, 0] % g == 0
    assert np.all(var[known] == 0.0) and np.all(var[~known] > 0.0)


def test_uk_voxels_constant_drift_two_slabs_is_the_ok_volume():
    vol = np.random.default_rng(26).normal(size=(4, 9, 10))
    g, r = 4, 1
    rng = np.random.default_rng(27)
    zyx = np.stack([rng.integers(0, (4 - 1) * g + 1, 300), rng.integers(0, 9, 300), rng.integers(0, 10, 300)], 1)
    vg = dict(model="spherical", nugget=0.01, sill=1.0, range=7.0)
    e1, v1 = oracle.uk_voxels(vol, g, r, zyx, slabs=2, drift="constant", **vg)
    e2, v2 = oracle.krige_voxels(vol, g, r, zyx, **vg)
    assert np.array_equal(e1, e2)
    assert np.allclose(v1, v2, rtol=1e-12, atol=1e-15)


def test_uk_voxels_neighbourhood_is_the_stated_slab_window():
    """The 4-slice neighbourhood of a target in gap j at offset t: known slices j-1 .. j+2 that
    exist, the (2r+1)^2 window around (x, y) in each, cut at the border, at dz = (jj - j) g - t;
    the 2-slice one uses j and j+1.  Built here point by point and solved directly."""
    n, H, W, g, r = 6, 8, 9, 3, 1
    S = np.random.default_rng(28).normal(size=(n, H, W))
    vg = dict(model="spherical", nugget=0.02, sill=1.0, range=6.0)
    for slabs in (2, 4):
        for (j, t, y, x) in [(0, 1, 0, 0), (1, 2, 4, 5), (4, 1, 7, 8), (2, 2, 3, 0)]:
            pts, vals = [], []
            for jj in (range(j - 1, j + 3) if slabs == 4 else range(j, j + 2)):
                if not 0 <= jj < n:
                    continue
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        if 0 <= y + dy < H and 0 <= x + dx < W:
                            pts.append((dx, dy, (jj - j) * g - t))
                            vals.append(S[jj, y + dy, x + dx])
            ref = oracle.uk_solve(np.array(pts, float), np.zeros(3), "xyz", np.array(vals), **vg)
            est, var = oracle.uk_voxels(S, g, r, [[j * g + t, y, x]], slabs=slabs, drift="xyz", **vg)
            assert est[0] == pytest.approx(ref["est"], rel=1e-12, abs=1e-14)
            assert var[0] == pytest.approx(ref["var"], rel=1e-12)


def test_sub_blocks_partition_the_gaps():
    """Algorithm 1 step 2 as read: k blocks of whole gaps, the first (n-1) % k one gap longer."""
    assert oracle.sub_blocks(24, 4) == [0, 6, 12, 18, 23]
    assert oracle.sub_blocks(32, 8) == [0, 4, 8, 12, 16, 20, 24, 28, 31]
    assert oracle.sub_blocks(9, 2) == [0, 4, 8]
    assert oracle.sub_blocks(2, 1) == [0, 1]


def test_clamp_block_minmax_hand_worked():
    """Three known 1 x 2 slices, g = 2, two blocks: block 0 holds slices 0, 1 (range [0, 2]), block 1
    slices 1, 2 (range [1, 5]); output slices 1 and 3 are the missing ones."""
    S = np.array([[[0.0, 2.0]], [[1.0, 1.5]], [[5.0, 3.0]]])
    out = np.array([[[0.0, 2.0]], [[-1.0, 2.5]], [[1.0, 1.5]], [[0.5, 7.0]], [[5.0, 3.0]]])
    exp = np.array([[[0.0, 2.0]], [[0.0, 2.0]], [[1.0, 1.5]], [[1.0, 5.0]], [[5.0, 3.0]]])
    assert np.array_equal(oracle.clamp_block_minmax(out, S, 2, 2), exp)
    out[1, 0, 0] = np.nan
    assert np.isnan(oracle.clamp_block_minmax(out, S, 2, 2)[1, 0, 0])


def test_clamp_block_minmax_keeps_in_range_estimates_and_is_idempotent():
    rng = np.random.default_rng(3)
    S = rng.random((7, 9, 11))
    out, _ = oracle.krige_volume(S, 3, 1, k_sub=3, model="spherical", nugget=0.0, sill=float(S.var()), range=8.0)
    c = oracle.clamp_block_minmax(out, S, 3, 3)
    assert np.array_equal(c[::3], S)
    assert np.array_equal(oracle.clamp_block_minmax(c, S, 3, 3), c)
    a = oracle.sub_blocks(7, 3)
    for b in range(3):
        blk = c[a[b] * 3:a[b + 1] * 3 + 1]
        assert blk.min() >= S[a[b]:a[b + 1] + 1].min() and blk.max() <= S[a[b]:a[b + 1] + 1].max()
