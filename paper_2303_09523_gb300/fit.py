"""Fit the variogram of a slice stack by gradient descent on the leave-one-slice-out loss.

The paper names kriging but fixes no variogram; the leave-one-slice-out loss
(each interior known slice predicted from its neighbours, ``binding.loo_loss``)
makes the choice a differentiable fit.  The ordinary-kriging weights are
0-homogeneous in (nugget, sill), so the sill is held fixed and the fit moves
log(range) and log(nugget / sill).  Loss and gradients come from the CUDA
kernels; the optimizer update is a two-element PyTorch step.
"""
import math

from . import binding


def fit_variogram_loo(slices, zfactor, half_w, n_sub_blocks, model, sill, init_range=8.0, init_ratio=0.05,
                      steps=50, lr=0.1):
    """Adam on (log range, log nugget/sill).  ``slices``: CUDA tensor (n, H, W), float32 or float64.

    Returns dict: ``theta`` (nugget, sill, range) at the end, ``loss`` there, ``losses`` per step and
    ``trajectory`` of theta per step.
    """
    import torch

    dev = slices.device
    p = torch.tensor([math.log(init_range), math.log(max(init_ratio, 1e-8))], dtype=torch.float64, device=dev,
                     requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr)
    losses, traj = [], []

    def theta_of(q):
        return torch.stack([torch.exp(q[1]) * sill, torch.ones((), dtype=torch.float64, device=dev) * sill,
                            torch.exp(q[0])])

    for _ in range(steps):
        opt.zero_grad()
        th = theta_of(p)
        loss = binding.loo_loss(slices, th, zfactor, half_w, n_sub_blocks, model)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        traj.append([float(x) for x in th.detach()])
    with torch.no_grad():
        th = theta_of(p)
        final = float(binding.loo_loss(slices, th, zfactor, half_w, n_sub_blocks, model))
    return {"theta": [float(x) for x in th], "loss": final, "losses": losses, "trajectory": traj}
