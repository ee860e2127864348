"""GPU leave-one-slice-out loss and adjoint against the FP64 oracle.

Tolerances: loss and predictions within 1e-5 (relative / normwise), gradients
w.r.t. the variogram parameters and the slice intensities within 1e-4 normwise
(max |gpu - oracle| <= 1e-4 * max |oracle| per tensor).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu


def _run(vol, theta, dtype=None, want=True):
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    if dtype is not None and t.dtype != torch.uint16:
        t = t.to(dtype)
    code = binding.dtype_code(t.dtype)
    d = binding.desc_for(tuple(t.shape), vol.zfactor, vol.half_w, vol.n_sub_blocks, code, vol.in_scale)
    plan = binding.Plan([d], form="DS", flags=binding.FLAG_LOO)
    params = binding.variogram_tensor([theta])
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    pred = torch.empty((vol.n - 2, vol.H, vol.W), dtype=torch.float32, device="cuda")
    plan.loo_forward([t], params, loss, [pred])
    out = {"loss": float(loss.item()), "pred": pred.double().cpu().numpy()}
    if want:
        gl = torch.ones(1, dtype=torch.float64, device="cuda")
        gs = torch.empty(t.shape, dtype=torch.float32, device="cuda")
        gp = torch.empty(3, dtype=torch.float64, device="cuda")
        plan.backward([t], params, gl, [gs], gp)
        out["grad_slices"] = gs.double().cpu().numpy()
        out["grad_theta"] = gp.cpu().numpy()
    plan.device_status()
    plan.close()
    vals = t.double().cpu().numpy() if t.dtype != torch.uint16 else vol.values_f64()
    return out, vals


def _nw(a, b):
    """Normwise error; a reference that is exactly zero (e.g. the symmetric 2-point LOO weights do
    not depend on theta at all) is compared absolutely."""
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / scale) if scale > 1e-12 else float(np.abs(a - b).max() * 1e8)


CASES = [
    ("spherical", 1, None),
    ("exponential", 2, None),
    ("spherical", 1, torch.float64),
    ("exponential", 0, None),
]


@pytest.mark.parametrize("model,r,dtype", CASES)
def test_loo_matches_oracle(model, r, dtype):
    vol = phantoms.random_stack(6, 37, 45, 3, r, k=2, seed=50, model=model)
    theta = dict(model=model, nugget=0.02, sill=vol.sill, range=6.0)
    got, vals = _run(vol, theta, dtype)
    ref = oracle.loo(vals, vol.zfactor, r, want_pred=True, want_grad_theta=True, want_grad_slices=True, **theta)
    assert got["loss"] == pytest.approx(ref["loss"], rel=1e-5)
    assert _nw(got["pred"], ref["pred"]) <= 1e-5
    assert _nw(got["grad_theta"], ref["grad_theta"]) <= 1e-4
    assert _nw(got["grad_slices"], ref["grad_slices"]) <= 1e-4


def test_loo_uint16_spine_small():
    vol = phantoms.spine(n=7, H=40, W=64, g=4, k=2)
    theta = dict(model="spherical", nugget=0.0, sill=vol.sill, range=8.0)
    got, vals = _run(vol, theta)
    ref = oracle.loo(vals, vol.zfactor, vol.half_w, want_grad_theta=True, want_grad_slices=True, **theta)
    assert got["loss"] == pytest.approx(ref["loss"], rel=1e-5)
    assert _nw(got["grad_slices"], ref["grad_slices"]) <= 1e-4
    # at zero nugget the weights do not depend on the sill, so dL/dsill = 0
    assert abs(got["grad_theta"][1]) <= 1e-6 * np.abs(got["grad_theta"]).max()
    assert _nw(got["grad_theta"][[0, 2]], ref["grad_theta"][[0, 2]]) <= 1e-4


def test_loo_homogeneity_and_fd():
    """nugget dL/dnugget + sill dL/dsill = 0; central differences (h = 1e-3) of the GPU loss in theta.

    The GPU loss forms residuals in FP32, so its central difference carries about 1 % noise at this
    step; the tight check is against the FP64 oracle gradient (itself pinned by central differences).
    """
    vol = phantoms.random_stack(5, 32, 40, 2, 1, k=1, seed=51)
    theta = dict(model="spherical", nugget=0.05, sill=0.8, range=5.0)
    got, vals = _run(vol, theta, torch.float64)
    g = got["grad_theta"]
    assert abs(theta["nugget"] * g[0] + theta["sill"] * g[1]) <= 1e-4 * np.abs(g).max()
    ref = oracle.loo(vals, vol.zfactor, vol.half_w, want_grad_theta=True, **theta)
    assert _nw(g, ref["grad_theta"]) <= 1e-4
    for p, key in ((0, "nugget"), (2, "range")):
        h = 1e-3
        hi = dict(theta); hi[key] += h
        lo = dict(theta); lo[key] -= h
        fd = (_run(vol, hi, torch.float64, want=False)[0]["loss"] - _run(vol, lo, torch.float64, want=False)[0]["loss"]) / (2 * h)
        assert g[p] == pytest.approx(fd, rel=2e-2, abs=1e-9)


def test_backward_accumulate():
    vol = phantoms.random_stack(5, 20, 24, 3, 1, k=1, seed=52)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    d = binding.desc_for(tuple(t.shape), 3, 1, 1, binding.F32)
    plan = binding.Plan([d], form="DS", flags=binding.FLAG_LOO)
    params = binding.variogram_tensor([dict(model="spherical", nugget=0.01, sill=0.5, range=4.0)])
    gl = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")
    gs = torch.zeros(t.shape, dtype=torch.float32, device="cuda")
    gp = torch.zeros(3, dtype=torch.float64, device="cuda")
    plan.backward([t], params, gl, [gs], gp)
    gs1, gp1 = gs.clone(), gp.clone()
    plan.backward([t], params, gl, [gs], gp, accumulate=True)
    assert torch.allclose(gs, 2 * gs1, rtol=1e-6, atol=0)
    assert torch.allclose(gp, 2 * gp1, rtol=1e-6, atol=0)
    plan.close()


def test_autograd_function_matches_oracle():
    vol = phantoms.random_stack(6, 30, 34, 2, 1, k=2, seed=53)
    s = torch.from_numpy(vol.slices.astype(np.float32)).cuda().requires_grad_(True)
    theta = torch.tensor([0.03, 0.7, 5.5], dtype=torch.float64, device="cuda", requires_grad=True)
    loss = binding.loo_loss(s, theta, 2, 1, 2, "exponential")
    loss.backward()
    ref = oracle.loo(vol.slices.astype(np.float64), 2, 1, want_grad_theta=True, want_grad_slices=True,
                     model="exponential", nugget=0.03, sill=0.7, range=5.5)
    assert float(loss.detach()) == pytest.approx(ref["loss"], rel=1e-5)
    assert _nw(theta.grad.cpu().numpy(), ref["grad_theta"]) <= 1e-4
    assert _nw(s.grad.double().cpu().numpy(), ref["grad_slices"]) <= 1e-4


def test_fit_reaches_grid_minimum():
    """50 Adam steps on log-range and the nugget/sill ratio (sill fixed: weights are 0-homogeneous in
    (nugget, sill)) reach a loss within 1 % of the best of a brute-force grid."""
    vol = phantoms.spine(n=10, H=64, W=64, g=4, k=3)
    s = torch.from_numpy(vol.values_f64().astype(np.float32)).cuda()
    sill = vol.sill
    from paper_2303_09523_gb300 import fit
    res = fit.fit_variogram_loo(s, vol.zfactor, vol.half_w, vol.n_sub_blocks, "spherical", sill,
                                init_range=3.0, init_ratio=0.1, steps=50, lr=0.1)
    losses = res["losses"]
    assert losses[-1] < losses[0]
    best = np.inf
    for a in np.linspace(1.5, 30.0, 40):
        for ratio in (0.0, 0.01, 0.03, 0.1, 0.3):
            th = torch.tensor([ratio * sill, sill, a], dtype=torch.float64, device="cuda")
            best = min(best, float(binding.loo_loss(s, th, vol.zfactor, vol.half_w, vol.n_sub_blocks, "spherical")))
    assert res["loss"] <= best * 1.01


def test_loo_full_size_spine():
    """24 known 256x256 uint16 slices, g 4, 18 points: loss and gradients against the oracle."""
    vol = phantoms.spine()
    theta = dict(model="spherical", nugget=0.005, sill=vol.sill, range=8.0)
    got, vals = _run(vol, theta)
    ref = oracle.loo(vals, vol.zfactor, vol.half_w, want_grad_theta=True, want_grad_slices=True, **theta)
    assert got["loss"] == pytest.approx(ref["loss"], rel=1e-5)
    assert _nw(got["grad_theta"], ref["grad_theta"]) <= 1e-4
    assert _nw(got["grad_slices"], ref["grad_slices"]) <= 1e-4


def test_loo_batched_volumes_mixed_r():
    """One plan over three volumes with r = 0, 1, 2 (one launch per r in each pass), mixed
    dtypes and variogram models: every volume's loss, predictions and gradients match the oracle;
    repeated forward passes give the same bits (the forward's block ticket resets itself); the
    backward pass with only dL/dtheta or only dL/dS asked for gives the same values as with both."""
    vols = [phantoms.random_stack(5, 33, 40, 2, 0, k=1, seed=60, model="spherical"),
            phantoms.random_stack(7, 29, 52, 3, 1, k=2, seed=61, model="exponential"),
            phantoms.random_stack(6, 41, 36, 2, 2, k=1, seed=62, model="spherical")]
    thetas = [dict(model=v.variogram()["model"], nugget=0.03, sill=v.sill, range=5.0 + i) for i, v in enumerate(vols)]
    ts = [torch.from_numpy(np.ascontiguousarray(v.slices)).cuda() for v in vols]
    ts[1] = ts[1].double()
    descs = [binding.desc_for(tuple(t.shape), v.zfactor, v.half_w, v.n_sub_blocks, binding.dtype_code(t.dtype))
             for v, t in zip(vols, ts)]
    plan = binding.Plan(descs, form="DS", flags=binding.FLAG_LOO)
    params = binding.variogram_tensor(thetas)
    nv = len(vols)
    loss = torch.empty(nv, dtype=torch.float64, device="cuda")
    preds = [torch.empty((v.n - 2, v.H, v.W), dtype=torch.float32, device="cuda") for v in vols]
    plan.loo_forward(ts, params, loss, preds)
    first = loss.clone()
    plan.loo_forward(ts, params, loss, preds)
    assert torch.equal(loss, first)
    gl = torch.ones(nv, dtype=torch.float64, device="cuda")
    gs = [torch.empty(t.shape, dtype=torch.float32, device="cuda") for t in ts]
    gp = torch.empty(3 * nv, dtype=torch.float64, device="cuda")
    plan.backward(ts, params, gl, gs, gp)
    gp_only = torch.empty(3 * nv, dtype=torch.float64, device="cuda")
    plan.backward(ts, params, gl, None, gp_only)
    gs_only = [torch.empty_like(g) for g in gs]
    plan.backward(ts, params, gl, gs_only, None)
    plan.device_status()
    plan.close()
    # the per-block partial sums of dL/dw meet in atomics in any order (FP32 within a block), so the
    # two calls agree up to FP32 rounding (r = 0 has dL/dtheta = 0 exactly: the two weights are 1/2
    # whatever theta, so its entries are rounding noise)
    assert torch.allclose(gp_only, gp, rtol=1e-6, atol=1e-9 * gp.abs().max().item())
    for a, b in zip(gs_only, gs):
        assert torch.equal(a, b)
    for i, (v, t, th) in enumerate(zip(vols, ts, thetas)):
        ref = oracle.loo(t.double().cpu().numpy(), v.zfactor, v.half_w, want_pred=True, want_grad_theta=True,
                         want_grad_slices=True, **th)
        assert loss[i].item() == pytest.approx(ref["loss"], rel=1e-5), i
        assert _nw(preds[i].double().cpu().numpy(), ref["pred"]) <= 1e-5, i
        assert _nw(gp[3 * i:3 * i + 3].cpu().numpy(), ref["grad_theta"]) <= 1e-4, i
        assert _nw(gs[i].double().cpu().numpy(), ref["grad_slices"]) <= 1e-4, i


@pytest.mark.parametrize("n,H,W,g,r,model", [
    (3, 3, 5, 2, 2, "spherical"),        # one target slice; window wider than the slice: no interior class
    (4, 2, 9, 3, 1, "exponential"),      # two rows: every pixel is a border pixel
    (3, 17, 6, 4, 0, "spherical"),       # r = 0 (two-point midpoint); width not a multiple of 4
    (5, 70, 131, 2, 2, "exponential"),   # several tiles with ragged right and bottom tails
])
def test_loo_edge_geometries(n, H, W, g, r, model):
    vol = phantoms.random_stack(n, H, W, g, r, k=1, seed=70 + n + H, model=model)
    theta = dict(model=model, nugget=0.03, sill=vol.sill, range=4.0)
    got, vals = _run(vol, theta)
    ref = oracle.loo(vals, g, r, want_pred=True, want_grad_theta=True, want_grad_slices=True, **theta)
    assert got["loss"] == pytest.approx(ref["loss"], rel=1e-5)
    assert _nw(got["pred"], ref["pred"]) <= 1e-5
    assert _nw(got["grad_theta"], ref["grad_theta"]) <= 1e-4
    assert _nw(got["grad_slices"], ref["grad_slices"]) <= 1e-4
