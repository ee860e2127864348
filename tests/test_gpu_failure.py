"""Failure detection on the GPU without a fault: the stencil kernel's bounded device
waits give up and report KRIG_ETIMEOUT, and the context stays usable."""
import numpy as np
import pytest
import torch

from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu

FLAG_FAULT_TIMEOUT = 0x100


def _spec(vol, t):
    return dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                variogram=vol.variogram(), in_scale=vol.in_scale)


def test_bounded_wait_times_out_and_context_survives():
    vol = phantoms.random_stack(5, 64, 64, 3, 1, k=2, seed=40)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    with pytest.raises(binding.KrigError) as ei:
        binding.krige([_spec(vol, t)], form="DS", flags=FLAG_FAULT_TIMEOUT)
    assert ei.value.status == binding.KRIG_ETIMEOUT
    # the device is still healthy: a normal call afterwards succeeds and is correct
    outs, _ = binding.krige([_spec(vol, t)], form="DS")
    torch.cuda.synchronize()
    assert torch.isfinite(outs[0]).all()
    assert torch.equal(outs[0][::vol.zfactor], t)


def test_status_is_cleared_after_report():
    vol = phantoms.random_stack(3, 32, 32, 2, 1, k=1, seed=41)
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).cuda()
    plan = binding.Plan([binding.desc_for(tuple(t.shape), 2, 1, 1, binding.F32)], form="DS")
    bad = binding.variogram_tensor([dict(model="spherical", nugget=0.0, sill=0.0, range=8.0)])
    good = binding.variogram_tensor([vol.variogram()])
    out = torch.empty((vol.n_out, 32, 32), dtype=torch.float32, device="cuda")
    plan.interpolate([t], [out], bad)
    with pytest.raises(binding.KrigError):
        plan.device_status()
    plan.interpolate([t], [out], good)
    plan.device_status()  # cleared: no error now
    plan.close()
