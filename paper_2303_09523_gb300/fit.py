"""Fit the variogram of a slice stack: by gradient descent on the leave-one-slice-out loss,
or by weighted least squares on the empirical variogram.

The paper names kriging but fixes no variogram; the leave-one-slice-out loss
(each interior known slice predicted from its neighbours, ``binding.loo_loss``)
makes the choice a differentiable fit.  The ordinary-kriging weights are
0-homogeneous in (nugget, sill), so the sill is held fixed and the fit moves
log(range) and log(nugget / sill).  Loss and gradients come from the CUDA
kernels; the optimizer update is a two-element PyTorch step.

The classical alternative fits the model curve to the empirical variogram:
``variogram_bins`` pools the per-lag-vector sums of
``binding.empirical_variogram`` (computed on the GPU) into distance classes,
``fit_variogram_wls`` fits (nugget, partial sill, range) to them by weighted
least squares with Cressie's weights N(h) / gamma(h; theta)^2 (a three-parameter
fit over a few dozen classes, on the host).
"""
import json
import math
import os

from . import binding


def fit_log_append(path, record):
    """Append one step of a fit as a JSON line (flushed and synced, so a crash leaves at most a
    partial last line)."""
    with open(path, "a") as f:
        f.write(json.dumps(record) + "\n")
        f.flush()
        os.fsync(f.fileno())


def fit_log_last(path):
    """The last complete record of a fit log, or None (no file, or no complete line)."""
    if not os.path.exists(path):
        return None
    last = None
    with open(path) as f:
        for line in f:
            if not line.endswith("\n"):
                break  # a partial last line: the step it describes did not finish
            try:
                last = json.loads(line)
            except ValueError:
                break
    return last


def fit_variogram_loo(slices, zfactor, half_w, n_sub_blocks, model, sill, init_range=8.0, init_ratio=0.05,
                      steps=50, lr=0.1, log_path=None, resume=False):
    """Adam on (log range, log nugget/sill).  ``slices``: CUDA tensor (n, H, W), float32 or float64.

    With ``log_path`` every step is appended there as a JSON line (step, theta, loss, the two
    parameters and Adam's state); with ``resume=True`` the fit continues after the last complete
    record of that log, with the same parameters and optimizer state, so an interrupted fit ends
    where an uninterrupted one would.

    Returns dict: ``theta`` (nugget, sill, range) at the end, ``loss`` there, ``losses`` per step and
    ``trajectory`` of theta per step (the steps run by this call).
    """
    import torch

    dev = slices.device
    p = torch.tensor([math.log(init_range), math.log(max(init_ratio, 1e-8))], dtype=torch.float64, device=dev,
                     requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr)
    losses, traj = [], []
    first = 0
    if resume and log_path is not None:
        rec = fit_log_last(log_path)
        if rec is not None:
            with torch.no_grad():
                p.copy_(torch.tensor(rec["p"], dtype=torch.float64, device=dev))
            st = opt.state[p]
            st["step"] = torch.tensor(float(rec["adam"]["step"]), dtype=torch.float32)
            st["exp_avg"] = torch.tensor(rec["adam"]["exp_avg"], dtype=torch.float64, device=dev)
            st["exp_avg_sq"] = torch.tensor(rec["adam"]["exp_avg_sq"], dtype=torch.float64, device=dev)
            first = int(rec["step"]) + 1

    def theta_of(q):
        return torch.stack([torch.exp(q[1]) * sill, torch.ones((), dtype=torch.float64, device=dev) * sill,
                            torch.exp(q[0])])

    for it in range(first, steps):
        opt.zero_grad()
        th = theta_of(p)
        loss = binding.loo_loss(slices, th, zfactor, half_w, n_sub_blocks, model)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        traj.append([float(x) for x in th.detach()])
        if log_path is not None:
            st = opt.state[p]
            fit_log_append(log_path, {"step": it, "theta": traj[-1], "loss": losses[-1],
                                      "p": [float(x) for x in p.detach()],
                                      "adam": {"step": float(st["step"]),
                                               "exp_avg": [float(x) for x in st["exp_avg"]],
                                               "exp_avg_sq": [float(x) for x in st["exp_avg_sq"]]}})
    with torch.no_grad():
        th = theta_of(p)
        final = float(binding.loo_loss(slices, th, zfactor, half_w, n_sub_blocks, model))
    return {"theta": [float(x) for x in th], "loss": final, "losses": losses, "trajectory": traj}


def variogram_bins(sums, counts, zfactor):
    """Distance classes of the empirical variogram.

    ``sums``, ``counts``: arrays [2, 2L+1, 2L+1] of ``binding.empirical_variogram`` (squared-increment
    sums and pair counts per lag vector (s, dy, dx)).  The lag vector's length in output-voxel units is
    sqrt(dx^2 + dy^2 + (s zfactor)^2); vectors are pooled by that length rounded to the nearest integer
    (the zero lag left out).  Returns (h, gamma, n): the pair-weighted mean length, gamma = pooled sum /
    (2 pooled count) and the pooled count per class, classes with pairs only, by increasing h.
    """
    import numpy as np
    sums = np.asarray(sums, dtype=np.float64)
    counts = np.asarray(counts, dtype=np.int64)
    L = (sums.shape[-1] - 1) // 2
    acc = {}
    for s in (0, 1):
        for dy in range(-L, L + 1):
            for dx in range(-L, L + 1):
                c = int(counts[s, dy + L, dx + L])
                if c <= 0 or (s == 0 and dx == 0 and dy == 0):
                    continue
                h = math.sqrt(dx * dx + dy * dy + (s * zfactor) ** 2)
                b = int(round(h))
                t = acc.setdefault(b, [0.0, 0, 0.0])
                t[0] += float(sums[s, dy + L, dx + L])
                t[1] += c
                t[2] += h * c
    keys = sorted(acc)
    n = np.array([acc[b][1] for b in keys], dtype=np.float64)
    gamma = np.array([acc[b][0] for b in keys]) / (2.0 * n)
    h = np.array([acc[b][2] for b in keys]) / n
    return h, gamma, n


def variogram_model(h, model, nugget, sill, rng):
    """gamma(h) for h > 0: nugget plus the partial sill times the spherical or exponential shape."""
    import numpy as np
    h = np.asarray(h, dtype=np.float64)
    if model == "spherical":
        q = np.minimum(h / rng, 1.0)
        return nugget + sill * (1.5 * q - 0.5 * q ** 3)
    return nugget + sill * (1.0 - np.exp(-3.0 * h / rng))


def fit_variogram_wls(h, gamma, n, model, init=None, max_range=None):
    """Weighted least squares: minimise sum_b n_b (gamma_b / gamma(h_b; theta) - 1)^2 over
    theta = (nugget >= 0, partial sill > 0, 0 < range <= max_range).  The data say nothing about a
    range far beyond the longest lag class, where the models are all but linear in h (a fit that
    runs off there trades range for sill along a ridge), so the range is bounded by default at three
    times the longest class.  Returns dict ``theta`` (nugget, sill, range), ``cost`` and
    ``range_at_bound`` (True when the bound holds the range: no sill within the observed lags)."""
    import numpy as np
    from scipy.optimize import least_squares
    h = np.asarray(h, dtype=np.float64)
    gamma = np.asarray(gamma, dtype=np.float64)
    w = np.sqrt(np.asarray(n, dtype=np.float64))
    if max_range is None:
        max_range = 3.0 * float(h.max())
    if init is None:
        init = (0.1 * gamma[0], max(gamma.max() - 0.1 * gamma[0], 1e-12), min(max(h.max() / 2.0, 1.0), max_range))

    def res(p):
        return w * (gamma / variogram_model(h, model, p[0], p[1], p[2]) - 1.0)

    r = least_squares(res, np.asarray(init, dtype=np.float64),
                      bounds=([0.0, 1e-12, 1e-6], [np.inf, np.inf, float(max_range)]),
                      x_scale="jac", xtol=1e-12, ftol=1e-12, gtol=1e-12, max_nfev=2000)
    return {"theta": (float(r.x[0]), float(r.x[1]), float(r.x[2])), "cost": float(r.cost),
            "range_at_bound": bool(r.x[2] >= 0.999 * float(max_range))}

