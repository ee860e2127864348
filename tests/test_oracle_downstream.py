"""Pins of the downstream oracle (oracle/downstream.py): the similarity metrics of Appendix D,
the shearlet transform of Appendix B, the edge orientation of Eq. 1 and the mean-median
deblurring of Algorithm 2.  CPU only."""
import os

import numpy as np
import pytest

from oracle import downstream as ds

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _img(text):
    return np.array([[float(v) for v in row.split()] for row in text.split("/")])


def _similarity_cases():
    out = []
    for line in open(os.path.join(GOLDEN, "similarity_values.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        metric, g, r, val = [p.strip() for p in line.split("|")]
        out.append((metric, _img(g), _img(r), float(val)))
    return out


@pytest.mark.parametrize("metric,G,R,val", _similarity_cases())
def test_metric_hand_worked_values(metric, G, R, val):
    fn = {"ssim": ds.ssim_global, "rmse": ds.rmse, "mi": ds.mutual_information, "ed": ds.entropy_difference}
    assert fn[metric](G, R) == pytest.approx(val, abs=1e-12)


def _phantom_slice(seed=3, H=48, W=40):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    g = 0.2 + 0.6 * (((x - W / 2) / 14.0) ** 2 + ((y - H / 2) / 18.0) ** 2 < 1.0)
    return g + 0.01 * rng.normal(size=g.shape)


def test_self_comparison_p13():
    """RMSE(G, G) = 0, SSIM(G, G) = 1, MI(G, G) = H(G), ED(G, G) = 0."""
    G = _phantom_slice()
    lo, hi = float(G.min()), float(G.max())
    assert ds.rmse(G, G) == 0.0
    assert ds.ssim_global(G, G) == pytest.approx(1.0, abs=1e-15)
    assert ds.ssim_windowed(G, G) == pytest.approx(1.0, abs=1e-15)
    assert ds.mutual_information(G, G) == pytest.approx(ds.entropy(G, lo, hi), abs=1e-12)
    assert ds.entropy_difference(G, G) == 0.0


def test_windowed_ssim_equals_global_on_one_window():
    rng = np.random.default_rng(4)
    G = rng.random((7, 7))
    R = G + 0.1 * rng.random((7, 7))
    assert ds.ssim_windowed(G, R, win=7) == pytest.approx(ds.ssim_global(G, R), abs=1e-14)


def test_mi_brute_force_over_value_pairs():
    """On images whose distinct values fall in distinct bins, MI is the plain definition over the
    distinct value pairs (counted with a dictionary here)."""
    rng = np.random.default_rng(5)
    G = rng.integers(0, 4, (9, 11)).astype(float)
    R = (G + rng.integers(0, 2, G.shape)) % 4
    pairs = {}
    for g, r in zip(G.ravel(), R.ravel()):
        pairs[(g, r)] = pairs.get((g, r), 0) + 1
    n = G.size
    pg = {v: np.sum(G == v) / n for v in np.unique(G)}
    pr = {v: np.sum(R == v) / n for v in np.unique(R)}
    mi = sum(c / n * np.log2((c / n) / (pg[g] * pr[r])) for (g, r), c in pairs.items())
    assert ds.mutual_information(G, R) == pytest.approx(mi, abs=1e-12)


def test_entropy_of_equal_levels():
    G = np.repeat(np.array([0.0, 1.0, 2.0, 3.0]), 25).reshape(10, 10)
    assert ds.entropy(G, 0.0, 3.0) == pytest.approx(2.0, abs=1e-15)
    assert ds.entropy(np.full((5, 5), 0.7), 0.0, 1.0) == 0.0


# --------------------------------------------------------------------------- shearlets

@pytest.mark.parametrize("H,W", [(64, 64), (48, 80), (33, 17)])
def test_shearlet_system_is_a_parseval_frame(H, W):
    """The squared responses of the low-pass and every shearlet sum to one at every frequency, so
    the coefficients keep the image's energy (Parseval) and the frame reconstructs it."""
    low, fl = ds.shearlet_system(H, W)
    tot = low ** 2 + sum(f["resp"] ** 2 for f in fl)
    assert np.abs(tot - 1.0).max() < 1e-12
    rng = np.random.default_rng(6)
    img = rng.normal(size=(H, W))
    lowc, co = ds.shearlet_transform(img, (low, fl))
    energy = np.sum(lowc ** 2) + np.sum(co ** 2)
    assert energy == pytest.approx(np.sum(img ** 2), rel=1e-12)
    rec = np.real(np.fft.ifft2(np.fft.fft2(lowc) * low))
    for c, f in zip(co, fl):
        rec += np.real(np.fft.ifft2(np.fft.fft2(c) * f["resp"]))
    assert np.abs(rec - img).max() < 1e-10


def test_shearlet_responses_are_sheared_copies():
    """Within a cone and dilation, the response of shear s at frequency (w1, w2) equals the response of
    shear 0 at (w1, w2 - s w1): the shearing matrix S_s of Appendix B, checked on exact grid points."""
    H = W = 64
    low, fl = ds.shearlet_system(H, W)
    by = {(f["scale"], f["cone"], f["k"]): f for f in fl}
    j, K = 2, 8
    a = 4.0 ** (-(j + 1))
    f0 = by[(j, "h", 0)]["resp"]
    for k in (1, 3, -2):
        fk = by[(j, "h", k)]["resp"]
        s = k * np.sqrt(a)
        for w1 in (8, 16, 24, -16):
            for w2 in range(-20, 21):
                w2s = w2 - s * w1
                if abs(w2) > abs(w1) or abs(w2s) > abs(w1) or abs(w2s - round(w2s)) > 1e-12:
                    continue
                assert fk[w2 % H, w1 % W] == pytest.approx(f0[int(round(w2s)) % H, w1 % W], abs=1e-14)


@pytest.mark.parametrize("phi0", [0.0, np.pi / 8, np.pi / 4, 3 * np.pi / 8, np.pi / 2, 5 * np.pi / 8, 3 * np.pi / 4,
                                  7 * np.pi / 8])
def test_orientation_of_a_straight_edge(phi0):
    """Eq. 1 on a straight step edge: at the edge, the largest shearlet coefficient of the finest
    dilation is the one whose frequency line is nearest the edge normal."""
    H = W = 64
    y, x = np.mgrid[0:H, 0:W].astype(float)
    d = (x - 31.5) * np.cos(phi0) + (y - 31.5) * np.sin(phi0)
    img = 1.0 / (1.0 + np.exp(-d / 0.7))  # a smooth step across the normal (cos phi0, sin phi0)
    system = ds.shearlet_system(H, W)
    _, co = ds.shearlet_transform(img, system)
    finest = max(f["scale"] for f in system[1])
    theta, angs = ds.edge_orientation(co, system[1], finest)
    near = (np.abs(d) <= 0.75) & ((x - 31.5) ** 2 + (y - 31.5) ** 2 < 12 ** 2)
    got = angs[np.bincount(theta[near].ravel()).argmax()]
    diff = abs((got - phi0 + np.pi / 2) % np.pi - np.pi / 2)
    step = np.max(np.diff(np.sort(angs)))
    assert diff <= step / 2 + 1e-9


# --------------------------------------------------------------------------- Algorithm 2

def _golden_orientations():
    rows = {}
    for line in open(os.path.join(GOLDEN, "mean_median_example.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, *vals = line.split()
            rows[k] = [int(v) for v in vals]
    return rows["in"], rows["out"]


def test_worked_orientation_example():
    seq_in, seq_out = _golden_orientations()
    assert ds.smooth_window(seq_in) == seq_out


def test_steady_orientations_are_kept():
    assert ds.smooth_window([2] * 16) == [2] * 16
    steps = [1] * 8 + [2] * 8
    assert ds.smooth_window(steps) == steps
    # alternating 3, 1 (eight of each): the tie goes to the smaller orientation index
    flip = [3, 1] * 8
    assert ds.smooth_window(flip) == [3] + [1] * 14 + [1]


def test_median_adjust_hand_worked():
    img = np.arange(25, dtype=float).reshape(5, 5)
    out = ds.median_adjust(img.copy(), 2, 2, along_y=True)
    exp = img.copy()
    exp[1:4, 1] = 11.0   # median of 6, 11, 16
    exp[1:4, 3] = 13.0   # median of 8, 13, 18
    assert np.array_equal(out, exp)
    out = ds.median_adjust(img.copy(), 2, 2, along_y=False)
    exp = img.copy()
    exp[1, 1:4] = 7.0    # median of 6, 7, 8
    exp[3, 1:4] = 17.0   # median of 16, 17, 18
    assert np.array_equal(out, exp)


def test_deblur_touches_only_pixels_next_to_edges():
    G = _phantom_slice(H=40, W=40)
    out, info = ds.mean_median_deblur(G)
    assert out.shape == G.shape and info["n_edge"] > 0
    changed = np.argwhere(out != G)
    assert len(changed) == 0 or info["changed"] > 0


# --------------------------------------------------------------------------- marching cubes (Appendix C)

def _edge_keys(tris):
    """Directed edges of a triangle soup with vertices identified by their rounded coordinates."""
    keys = np.round(np.asarray(tris), 9)
    out = []
    for t in keys:
        v = [tuple(p) for p in t]
        out += [(v[0], v[1]), (v[1], v[2]), (v[2], v[0])]
    return out


def _check_closed(tris):
    """Every edge of a closed, consistently oriented surface is used once in each direction;
    returns the Euler characteristic V - E + F."""
    d = _edge_keys(tris)
    cnt = {}
    for a, b in d:
        cnt[(a, b)] = cnt.get((a, b), 0) + 1
    for (a, b), c in cnt.items():
        assert c == 1 and cnt.get((b, a), 0) == 1
    verts = {a for a, _ in d}
    return len(verts) - len(d) // 2 + len(tris)


def test_mc_plane_closed_form():
    """v = x cut at 2.3: every vertex at x = 2.3 (0.3 of the way from x = 2, not 0.7), the area is
    (H-1)(D-1), normals along -x (out of the region x > 2.3)."""
    D, H, W = 5, 7, 6
    z, y, x = np.mgrid[0:D, 0:H, 0:W].astype(np.float32)
    iso = np.float32(2.3)
    tris = ds.marching_cubes(x, iso)
    assert np.all(tris[:, :, 0] == float(iso))
    assert ds.mesh_area(tris) == pytest.approx((H - 1) * (D - 1), abs=1e-12)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert np.all(n[:, 0] < 0) and np.allclose(n[:, 1:], 0.0)


def test_mc_sphere_is_closed_genus_zero_with_its_volume():
    z, y, x = np.mgrid[0:24, 0:26, 0:28].astype(np.float64)
    r = 8.0
    vol = (r - np.sqrt((x - 13.5) ** 2 + (y - 12.5) ** 2 + (z - 11.5) ** 2)).astype(np.float32)
    tris = ds.marching_cubes(vol, np.float32(0.0))
    assert _check_closed(tris) == 2
    assert ds.mesh_signed_volume(tris) == pytest.approx(4 / 3 * np.pi * r ** 3, rel=0.02)
    assert ds.mesh_area(tris) == pytest.approx(4 * np.pi * r * r, rel=0.02)


def test_mc_torus_has_euler_characteristic_zero():
    z, y, x = np.mgrid[0:16, 0:36, 0:36].astype(np.float64)
    R, a = 10.0, 3.5
    q = np.sqrt((x - 17.5) ** 2 + (y - 17.5) ** 2) - R
    vol = (a - np.sqrt(q ** 2 + (z - 7.5) ** 2)).astype(np.float32)
    tris = ds.marching_cubes(vol, np.float32(0.0))
    assert _check_closed(tris) == 0
    assert ds.mesh_signed_volume(tris) == pytest.approx(2 * np.pi ** 2 * R * a * a, rel=0.03)


def test_mc_random_field_is_watertight():
    """Random values (every corner configuration, ambiguous faces included) inside a border of
    zeros: the surfaces are closed and consistently oriented."""
    rng = np.random.default_rng(8)
    vol = np.zeros((12, 13, 14), dtype=np.float32)
    vol[1:-1, 1:-1, 1:-1] = rng.random((10, 11, 12)).astype(np.float32)
    tris = ds.marching_cubes(vol, np.float32(0.5))
    assert len(tris) > 500
    # closed and consistently oriented: every edge is used as often in one direction as in the
    # other (a fan diagonal that lies on a face shared by two cubes is used by both cubes)
    cnt = {}
    for a, b in _edge_keys(tris):
        cnt[(a, b)] = cnt.get((a, b), 0) + 1
    for (a, b), c in cnt.items():
        assert cnt.get((b, a), 0) == c
    assert ds.mesh_signed_volume(tris) > 0


def test_mc_case_triangles_basic_cases():
    corners = list(np.ndindex(2, 2, 2))
    assert ds.mc_case_triangles({c: False for c in corners}) == []
    assert ds.mc_case_triangles({c: True for c in corners}) == []
    for c0 in corners:
        tri = ds.mc_case_triangles({c: c == c0 for c in corners})
        assert len(tri) == 1  # one corner cut off: the triangle on its three edges
    for k in range(256):
        tri = ds.mc_case_triangles({c: bool((k >> i) & 1) for i, c in enumerate(corners)})
        assert len(tri) <= 5
