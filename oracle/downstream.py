"""FP64 numpy oracle of the stages after the kriging: the similarity metrics of
Appendix D, the shearlet transform of Appendix B, the edge orientation of Eq. 1
(Sec. 4.1.2) and the mean-median deblurring of Algorithm 2.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU legs may import this module.  It shares no code with the CUDA
library and imports nothing from it.  Everything here is plain numpy in
float64, written step by step from the paper's definitions; where the paper
leaves a choice open the reading taken is stated beside the function.

Metrics (Appendix D; readings where the text is silent):
  * RMSE = sqrt(1/(MN) sum (R - G)^2).
  * Histograms for MI and entropy: 256 equal-width bins over the joint value
    range [min(G, R), max(G, R)] of the two images (one binning for both, so
    that MI(G, G) = H(G)), a value's bin floor((x - lo) * 256 / (hi - lo)) with
    the scale 256 / (hi - lo) formed first; logarithms base 2 (bits).
  * MI = sum p_GR log(p_GR / (p_G p_R)) over the joint histogram.
  * ED = |H(G) - H(R)| / H(G), the relative entropy difference.
  * SSIM: the global formula as printed, with means, variances (the text's
    "standard deviation" beside sigma^2 read as the variance) and covariance over
    the whole image (population moments), c1 = (0.01 L)^2, c2 = (0.03 L)^2 and L
    the dynamic range max(G) - min(G) of the ground truth; beside it the usual
    windowed form, the mean over every 7 x 7 window of the same formula.
"""
import numpy as np

NBINS = 256
K1, K2 = 0.01, 0.03


# ---------------------------------------------------------------------------
# Appendix D: similarity metrics of two 2-D images G (ground truth) and R
# ---------------------------------------------------------------------------

def rmse(G, R):
    """Root mean square error: the square root of the mean of (R - G)^2 over the M x N pixels."""
    G = np.asarray(G, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return float(np.sqrt(np.mean((R - G) ** 2)))


def _bin_index(X, lo, hi, nbins=NBINS):
    """Bin of every value in [lo, hi] split into nbins equal bins (the maximum falls in the last):
    floor((x - lo) * s) with the bin scale s = nbins / (hi - lo) formed once, in float64."""
    X = np.asarray(X, dtype=np.float64)
    if hi <= lo:
        return np.zeros(X.shape, dtype=np.int64)
    scale = float(nbins) / (float(hi) - float(lo))
    b = np.floor((X - lo) * scale).astype(np.int64)
    return np.clip(b, 0, nbins - 1)


def joint_range(G, R):
    return float(min(np.min(G), np.min(R))), float(max(np.max(G), np.max(R)))


def entropy(X, lo, hi, nbins=NBINS):
    """Shannon entropy (bits) of the histogram of X over [lo, hi] in nbins equal bins."""
    b = _bin_index(X, lo, hi, nbins).ravel()
    p = np.bincount(b, minlength=nbins).astype(np.float64) / b.size
    p = p[p > 0]
    return float(-np.sum(p * np.log2(p)))


def mutual_information(G, R, nbins=NBINS):
    """MI = sum over bin pairs of p_GR log2(p_GR / (p_G p_R)), joint histogram of G and R with one
    binning over their joint range."""
    lo, hi = joint_range(G, R)
    bg = _bin_index(G, lo, hi, nbins).ravel()
    br = _bin_index(R, lo, hi, nbins).ravel()
    joint = np.zeros((nbins, nbins))
    np.add.at(joint, (bg, br), 1.0)
    joint /= bg.size
    pg = joint.sum(axis=1)
    pr = joint.sum(axis=0)
    mi = 0.0
    for i, j in zip(*np.nonzero(joint)):
        mi += joint[i, j] * np.log2(joint[i, j] / (pg[i] * pr[j]))
    return float(mi)


def entropy_difference(G, R, nbins=NBINS):
    """ED = |H(G) - H(R)| / H(G), both entropies over the joint range of G and R."""
    lo, hi = joint_range(G, R)
    hg = entropy(G, lo, hi, nbins)
    hr = entropy(R, lo, hi, nbins)
    return float(abs(hg - hr) / hg) if hg > 0 else float(abs(hg - hr))


def _ssim_formula(mx, my, vx, vy, cxy, L):
    c1 = (K1 * L) ** 2
    c2 = (K2 * L) ** 2
    return ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))


def ssim_global(G, R):
    """SSIM of Appendix D over the whole image: population means, variances and covariance."""
    G = np.asarray(G, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    L = float(G.max() - G.min())
    mx, my = G.mean(), R.mean()
    vx = np.mean((G - mx) ** 2)
    vy = np.mean((R - my) ** 2)
    cxy = np.mean((G - mx) * (R - my))
    return float(_ssim_formula(mx, my, vx, vy, cxy, L))


def ssim_windowed(G, R, win=7):
    """Mean over every win x win window (fully inside the image) of the SSIM formula computed on that
    window's population moments; L is the dynamic range of the whole ground-truth image."""
    G = np.asarray(G, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    L = float(G.max() - G.min())
    H, W = G.shape
    vals = []
    for y in range(H - win + 1):
        for x in range(W - win + 1):
            a = G[y:y + win, x:x + win]
            b = R[y:y + win, x:x + win]
            ma, mb = a.mean(), b.mean()
            vals.append(_ssim_formula(ma, mb, np.mean((a - ma) ** 2), np.mean((b - mb) ** 2),
                                      np.mean((a - ma) * (b - mb)), L))
    return float(np.mean(vals))


def metrics(G, R):
    """The four metrics of Appendix D for one ground-truth / reconstructed image pair."""
    return {"rmse": rmse(G, R), "mi": mutual_information(G, R), "mi_gg": mutual_information(G, G),
            "ed": entropy_difference(G, R), "ssim": ssim_global(G, R)}


def accuracy(m, value_range):
    """Accuracy of one pair as the mean of the four per-metric scores (the garbled formula after
    Table 1 read as: 1 - ED, MI(G, R) / MI(G, G), 1 - RMSE / range, SSIM)."""
    return float(np.mean([1.0 - m["ed"], m["mi"] / m["mi_gg"] if m["mi_gg"] > 0 else 1.0,
                          1.0 - m["rmse"] / value_range, m["ssim"]]))


# ---------------------------------------------------------------------------
# Appendix B: discrete shearlet transform of a 2-D image, by FFT
# ---------------------------------------------------------------------------
#
# The shearlet with dilation a, shear s and translation t has the Fourier
# transform  a^{3/4} psi1(a w1) psi2((w2 - s w1) / (sqrt(a) w1)) e^{-2 pi i w.t}
# (the frequency form printed in Appendix B, the transform of
# a^{-3/4} psi(A_a^{-1} S_s^{-1}(x - t))), and SH(f)(a, s, t) = <f, psi_{a,s,t}>
# is, by Plancherel, the inverse Fourier transform over t of
# f^(w) psi^_{a,s}(w).  The paper names neither psi1 nor psi2; the readings:
#   * frequencies w in cycles per image (integers, |w| <= N/2 on an N-point axis);
#   * psi1 a band-pass with psi1(u)^2 = phi(u/4)^2 - phi(u)^2 (phi: a smooth
#     low-pass, 1 for |u| <= 1/8, 0 for |u| >= 1/4, Meyer's transition), so the
#     squares over the dilations a_j = 4^{-(j+1)}, j = 0..J-1, sum with the
#     low-pass phi(a_0 |w|)^2 to one;
#   * psi2(v) = cos(pi/2 nu(|v|)) on [-1, 1] (Meyer's nu), whose integer
#     shifts have squares summing to one;
#   * shears s = k sqrt(a_j), |k| <= 2^{j+1}, in the horizontal cone |w2| <= |w1|
#     and the same with w1, w2 exchanged in the vertical cone |w2| > |w1| (each
#     shearlet restricted to its cone), so that every frequency is covered by the
#     low-pass and the shearlets with squares summing to one (a Parseval frame);
#   * on an even axis the Nyquist frequency stands for both +N/2 and -N/2, so the
#     squared response there is the mean of the two;
#   * the factor a^{3/4} is replaced by 1: the digital system is normalised as a
#     Parseval frame instead (the orientation argmax of Eq. 1 is taken over the
#     shears of one dilation, where a common factor does not matter).

def _meyer_nu(x):
    x = np.clip(x, 0.0, 1.0)
    return x ** 4 * (35.0 - 84.0 * x + 70.0 * x * x - 20.0 * x ** 3)


def _phi(u):
    """Low-pass window: 1 for |u| <= 1/8, 0 for |u| >= 1/4, Meyer transition between."""
    u = np.abs(u)
    return np.cos(0.5 * np.pi * _meyer_nu(8.0 * u - 1.0))


def _psi1(u):
    """Band-pass window with psi1(u)^2 = phi(u/4)^2 - phi(u)^2."""
    return np.sqrt(np.maximum(_phi(u / 4.0) ** 2 - _phi(u) ** 2, 0.0))


def _psi2(v):
    v = np.abs(v)
    return np.where(v <= 1.0, np.cos(0.5 * np.pi * _meyer_nu(v)), 0.0)


def shearlet_system(H, W, n_scales=None):
    """Frequency responses of the digital shearlet system on an H x W grid.

    Returns (low, filters): ``low`` the low-pass (H x W), ``filters`` a list of dicts with
    ``scale`` j (0 = coarsest), ``cone`` ("h" or "v"), ``k`` (shear index), ``a`` and ``s`` and
    ``resp`` (H x W real response, numpy FFT frequency order)."""
    w1 = np.fft.fftfreq(W) * W  # along x (columns), cycles per image
    w2 = np.fft.fftfreq(H) * H  # along y (rows)
    X1, X2 = np.meshgrid(w1, w2)  # (H, W)
    if n_scales is None:
        n_scales = max(1, int(np.ceil(np.log(max(H, W)) / np.log(4.0))))
    a0 = 0.25
    low = _phi(a0 * np.maximum(np.abs(X1), np.abs(X2)))
    horiz = np.abs(X2) <= np.abs(X1)
    filters = []
    with np.errstate(divide="ignore", invalid="ignore"):
        for j in range(n_scales):
            a = 4.0 ** (-(j + 1))
            sa = np.sqrt(a)
            K = 2 ** (j + 1)
            for cone, (P, Q, mask) in (("h", (X1, X2, horiz)), ("v", (X2, X1, ~horiz))):
                band = _psi1(a * P)
                for k in range(-K, K + 1):
                    s = k * sa
                    v = np.where(P != 0, (Q - s * P) / (sa * P), np.inf)
                    resp = np.where(mask & (P != 0), band * _psi2(v), 0.0)
                    # the Nyquist row / column of an even axis is its own mirror on the DFT grid:
                    # symmetrise |resp|^2 over w and -w there, so a real image gets real
                    # coefficients (elsewhere resp(w) = resp(-w) already; the sum of squares stays 1)
                    mirror = resp[(-np.arange(H)) % H][:, (-np.arange(W)) % W]
                    resp = np.sqrt(0.5 * (resp * resp + mirror * mirror))
                    filters.append({"scale": j, "cone": cone, "k": k, "a": a, "s": s, "resp": resp})
    return low, filters


def shearlet_transform(img, system=None):
    """SH(f)(a, s, t) for every shearlet of the system and every pixel t: the inverse FFT of
    f^ psi^_{a,s}.  Returns (low coefficients (H x W), array [n_filters, H, W]) (real parts:
    the responses are real and even, so the coefficients of a real image are real)."""
    f = np.asarray(img, dtype=np.float64)
    H, W = f.shape
    low, filters = system if system is not None else shearlet_system(H, W)
    F = np.fft.fft2(f)
    lowc = np.real(np.fft.ifft2(F * low))
    coeffs = np.stack([np.real(np.fft.ifft2(F * flt["resp"])) for flt in filters])
    return lowc, coeffs


def shearlet_normal_angle(flt):
    """Direction (radians in [0, pi)) of the frequency line the shearlet sits on, i.e. the normal of
    the image edges it responds to: w2 / w1 = s in the horizontal cone, w1 / w2 = s in the vertical."""
    if flt["cone"] == "h":
        ang = np.arctan(flt["s"])
    else:
        ang = np.pi / 2 - np.arctan(flt["s"])
    return float(np.mod(ang, np.pi))


def edge_orientation(coeffs, filters, scale):
    """Eq. 1: theta_j(e) = argmax_k |SH(I)(j, k, e)| for every pixel e, over the shears k (both cones)
    of dilation j.  Returns (index into the sorted orientations of that scale, their normal angles)."""
    sel = [i for i, f in enumerate(filters) if f["scale"] == scale]
    angs = np.array([shearlet_normal_angle(filters[i]) for i in sel])
    order = np.argsort(angs, kind="stable")
    sel = [sel[i] for i in order]
    mag = np.abs(coeffs[sel])
    return np.argmax(mag, axis=0), angs[order]


# ---------------------------------------------------------------------------
# Sec. 4.1.2 / Algorithm 2: edge points, clockwise walk, mean-median deblurring
# ---------------------------------------------------------------------------
#
# Readings where the text leaves the step open:
#   * edge points ("as in [29]"): pixels whose largest shearlet magnitude over the
#     shears of the finest dilation is at least `rel_threshold` of the image's
#     largest and not below its two neighbours along its edge normal (the normal
#     of its argmax shearlet, rounded to the 8-neighbour directions);
#   * clockwise walk: the edge points in order of their angle about their
#     centroid, increasing atan2(y - cy, x - cx) with y pointing down the rows
#     (clockwise as the image is displayed), windows of 16 consecutive points;
#   * "changes frequently back and forth": more changes of orientation between
#     consecutive points of the window than half the window length;
#   * "mean(theta)": the worked example (16 orientations, nine of them theta_1)
#     gives theta_1, which is the most frequent orientation, not the arithmetic
#     mean of the indices (1.5); the most frequent one is taken, ties to the
#     smaller orientation index; the first and last point keep theirs;
#   * step 5 "left" and "right": the text's case (the next point is e(x, y+1))
#     puts them at x - 1 and x + 1; when the walk moves mostly along x instead,
#     they are taken at y - 1 and y + 1 (across the walk in both cases).

def smooth_window(thetas):
    """Alg. 2 steps 3-4 on one window of consecutive edge orientations: if they flip back and forth,
    every point but the first and last takes the window's most frequent orientation."""
    th = list(int(t) for t in thetas)
    n = len(th)
    if n < 3:
        return th
    changes = sum(1 for i in range(1, n) if th[i] != th[i - 1])
    if changes * 2 <= n:
        return th
    vals, counts = np.unique(th, return_counts=True)
    rep = int(vals[np.argmax(counts)])  # np.unique sorts: the first maximum is the smallest index
    return [th[0]] + [rep] * (n - 2) + [th[-1]]


def median_adjust(img, x, y, along_y=True):
    """Alg. 2 step 5 at edge pixel (x, y): the three pixels on one side take their median, the three
    on the other side theirs (x - 1 / x + 1 columns when the walk runs along y, rows otherwise).
    Pixels outside the image are left out."""
    out = img
    H, W = out.shape
    for side in (-1, 1):
        if along_y:
            pts = [(x + side, y + d) for d in (-1, 0, 1)]
        else:
            pts = [(x + d, y + side) for d in (-1, 0, 1)]
        pts = [(px, py) for px, py in pts if 0 <= px < W and 0 <= py < H]
        if not pts:
            continue
        med = float(np.median([out[py, px] for px, py in pts]))
        for px, py in pts:
            out[py, px] = med
    return out


_DIRS8 = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]


def edge_points(coeffs, filters, scale, rel_threshold=0.25):
    """Edge pixels of one image: (y, x) arrays and their orientation index (Eq. 1) at `scale`."""
    theta, angs = edge_orientation(coeffs, filters, scale)
    sel = [i for i, f in enumerate(filters) if f["scale"] == scale]
    E = np.max(np.abs(coeffs[sel]), axis=0)
    H, W = E.shape
    ys, xs = np.nonzero(E >= rel_threshold * E.max())
    keep = []
    for y, x in zip(ys, xs):
        a = angs[theta[y, x]]
        d = _DIRS8[int(np.round(a / (np.pi / 4))) % 4]  # normal direction, in (dx, dy) with y down the rows
        ok = True
        for sgn in (-1, 1):
            xx, yy = x + sgn * d[0], y + sgn * d[1]
            if 0 <= xx < W and 0 <= yy < H and E[yy, xx] > E[y, x]:
                ok = False
        if ok:
            keep.append((y, x))
    if not keep:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64)
    ys = np.array([p[0] for p in keep])
    xs = np.array([p[1] for p in keep])
    return ys, xs, theta[ys, xs]


def clockwise(ys, xs):
    """Order of the points by angle about their centroid, clockwise as displayed (rows down)."""
    cy, cx = ys.mean(), xs.mean()
    return np.argsort(np.arctan2(ys - cy, xs - cx), kind="stable")


def mean_median_deblur(img, window=16, rel_threshold=0.25, system=None):
    """Algorithm 2 on one 2-D image (a YZ-plane image of the interpolated volume): shearlet transform
    (step 1), edge points and their orientation (step 2, Eq. 1), the clockwise walk in windows of
    `window` points (step 3), the representative orientation of a window that flips (step 4: each
    changed point moves to a neighbour of the previous point that has that orientation, if there is
    one) and the median adjustment around each newly selected edge pixel (step 5).

    Returns (adjusted image, dict with the edge points, orientations before and after)."""
    f = np.array(img, dtype=np.float64, copy=True)
    H, W = f.shape
    system = system if system is not None else shearlet_system(H, W)
    _, coeffs = shearlet_transform(f, system)
    finest = max(flt["scale"] for flt in system[1])
    theta, _ = edge_orientation(coeffs, system[1], finest)
    ys, xs, th = edge_points(coeffs, system[1], finest, rel_threshold)
    info = {"n_edge": int(len(ys)), "changed": 0}
    if len(ys) == 0:
        return f, info
    order = clockwise(ys, xs)
    ys, xs, th = ys[order], xs[order], th[order]
    new_th = th.copy()
    for w0 in range(0, len(th), window):
        seg = smooth_window(th[w0:w0 + window])
        for i, t in enumerate(seg):
            k = w0 + i
            if t == th[k] or i == 0:
                continue
            new_th[k] = t
            info["changed"] += 1
            # step 4: among the 8 neighbours of the previous edge point, one with orientation t
            py, px = ys[k - 1], xs[k - 1]
            for dx, dy in _DIRS8:
                qx, qy = px + dx, py + dy
                if 0 <= qx < W and 0 <= qy < H and theta[qy, qx] == t and (qy, qx) != (py, px):
                    ys[k], xs[k] = qy, qx
                    break
            # step 5 around the selected pixel, across the direction of the walk
            along_y = abs(int(ys[k]) - int(py)) >= abs(int(xs[k]) - int(px))
            median_adjust(f, int(xs[k]), int(ys[k]), along_y)
    info["theta_before"] = th
    info["theta_after"] = new_th
    return f, info


# ---------------------------------------------------------------------------
# Appendix C: marching cubes
# ---------------------------------------------------------------------------
#
# The paper describes the method (256 corner configurations of a cube, linear
# interpolation along the cut edges) but prints no table.  The reading taken,
# derived here from the cube's geometry for every configuration:
#   * a corner is inside when its value is above the iso level;
#   * on every face the cut edges are paired into segments: walking the face's
#     boundary counter-clockwise as seen from outside the cube, each edge where
#     the walk enters the inside is joined to the nearest edge after it where
#     the walk leaves the inside (so a face with two diagonal inside corners
#     cuts each of them off alone); the segment runs from the first to the second;
#   * the segments close into loops (every cut edge begins one segment and ends
#     another); each loop, started at its edge of smallest number, is cut into
#     a fan of triangles (loop[0], loop[i], loop[i+1]), whose normals (right-hand
#     rule) point out of the inside region;
#   * cube corners are the voxels (x+dx, y+dy, z+dz), dx, dy, dz in {0, 1};
#     edges are numbered by axis (x: 0-3, y: 4-7, z: 8-11) and, within an axis,
#     by the two other offsets (for x edges dy + 2 dz, for y edges dx + 2 dz, for
#     z edges dx + 2 dy); a vertex lies on its edge at the fraction
#     t = (iso - v_low) / (v_high - v_low) from the lower corner;
#   * cubes in memory order of the volume (x fastest), their triangles in loop
#     order.

def _mc_edges():
    """The 12 edges as (lower corner offset, axis) with the numbering above."""
    edges = []
    for axis in range(3):
        others = [a for a in range(3) if a != axis]
        for k in range(4):
            off = [0, 0, 0]
            off[others[0]] = k & 1
            off[others[1]] = k >> 1
            edges.append((tuple(off), axis))
    return edges


def _mc_faces():
    """Each face as its four corner offsets in counter-clockwise order seen from outside."""
    faces = []
    for axis in range(3):
        for side in (0, 1):
            n = np.zeros(3)
            n[axis] = 1.0 if side else -1.0
            corners = [c for c in np.ndindex(2, 2, 2) if c[axis] == side]
            centre = np.mean(np.array(corners, dtype=float), axis=0)
            u = np.zeros(3)
            u[(axis + 1) % 3] = 1.0
            v = np.cross(n, u)  # (u, v, n) right-handed: angles about n increase counter-clockwise
            ang = [np.arctan2(np.dot(np.array(c) - centre, v), np.dot(np.array(c) - centre, u)) for c in corners]
            faces.append([tuple(corners[i]) for i in np.argsort(ang)])
    return faces


_MC_CACHE = {}


def mc_case_triangles(inside):
    """Triangles (as triples of edge numbers) of one cube configuration; ``inside`` maps a corner
    offset (dx, dy, dz) to True when it lies above the iso level."""
    key = tuple(bool(inside[c]) for c in np.ndindex(2, 2, 2))
    if key in _MC_CACHE:
        return _MC_CACHE[key]
    edges = _mc_edges()
    eid = {}
    for i, (off, axis) in enumerate(edges):
        hi = list(off)
        hi[axis] = 1
        eid[frozenset([off, tuple(hi)])] = i
    nxt = {}
    for face in _mc_faces():
        crossings = []  # (edge, leaving) walking counter-clockwise
        for i in range(4):
            a, b = face[i], face[(i + 1) % 4]
            if inside[a] != inside[b]:
                crossings.append((eid[frozenset([a, b])], inside[a] and not inside[b]))
        for k, (e, leaving) in enumerate(crossings):
            if leaving:
                continue
            j = k + 1
            while not crossings[j % len(crossings)][1]:
                j += 1
            nxt[e] = crossings[j % len(crossings)][0]
    tris, seen = [], set()
    for e0 in sorted(nxt):
        if e0 in seen:
            continue
        loop, e = [], e0
        while e not in seen:
            seen.add(e)
            loop.append(e)
            e = nxt[e]
        tris += [(loop[0], loop[i], loop[i + 1]) for i in range(1, len(loop) - 1)]
    _MC_CACHE[key] = tris
    return tris


def marching_cubes(vol, iso):
    """Iso-surface triangles of a volume (D x H x W, z y x), as an array [n, 3, 3] of vertex (x, y, z)
    coordinates in voxel units, float64."""
    V = np.asarray(vol)
    D, H, W = V.shape
    edges = _mc_edges()
    inside_all = V > iso
    out = []
    for z in range(D - 1):
        for y in range(H - 1):
            block = inside_all[z:z + 2, y:y + 2, :]
            anyin = block.any(axis=(0, 1))
            allin = block.all(axis=(0, 1))
            act = anyin[:-1] | anyin[1:]
            full = allin[:-1] & allin[1:]
            for x in np.nonzero(act & ~full)[0]:
                inside = {(dx, dy, dz): bool(inside_all[z + dz, y + dy, x + dx]) for dx, dy, dz in np.ndindex(2, 2, 2)}
                for tri in mc_case_triangles(inside):
                    verts = []
                    for e in tri:
                        off, axis = edges[e]
                        va = float(V[z + off[2], y + off[1], x + off[0]])
                        hi = list(off)
                        hi[axis] = 1
                        vb = float(V[z + hi[2], y + hi[1], x + hi[0]])
                        t = (float(iso) - va) / (vb - va)
                        p = [x + off[0], y + off[1], z + off[2]]
                        p[axis] += t
                        verts.append(p)
                    out.append(verts)
    return np.array(out, dtype=np.float64).reshape(-1, 3, 3)


def mesh_signed_volume(tris):
    """Volume enclosed by a closed triangle mesh (divergence theorem, sum of signed tetrahedra)."""
    t = np.asarray(tris, dtype=np.float64)
    return float(np.sum(np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2]))) / 6.0)


def mesh_area(tris):
    t = np.asarray(tris, dtype=np.float64)
    return float(0.5 * np.sum(np.linalg.norm(np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]), axis=1)))
