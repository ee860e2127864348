"""Batched uneven workload in one launch, the schedule autotuner and CUDA-graph replay.

16 seeded spine/brain float32 volumes (sides 128..512, 12-40 slices, g 2-6, 18 or 50
points).  Parity with the FP64 oracle on sampled voxels of every volume (normwise
1e-5, known slices bit-exact); one launch over all volumes is bit-identical to one
launch per volume, to every autotuned schedule and to a replayed CUDA graph.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2303_09523_gb300 import binding, phantoms

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup(vols):
    ts = [torch.from_numpy(np.ascontiguousarray(v.slices)).cuda() for v in vols]
    descs = [binding.desc_for(tuple(t.shape), v.zfactor, v.half_w, v.n_sub_blocks, binding.dtype_code(t.dtype),
                              v.in_scale) for v, t in zip(vols, ts)]
    outs = [torch.empty((v.n_out, v.H, v.W), dtype=torch.float32, device="cuda") for v in vols]
    params = binding.variogram_tensor([v.variogram() for v in vols])
    return ts, descs, outs, params


@pytest.fixture(scope="module")
def mix():
    return phantoms.batch_mix()


def test_batch_mix_parity_and_single_launch_equality(mix):
    ts, descs, outs, params = _setup(mix)
    plan = binding.Plan(descs, form="DS")
    plan.interpolate(ts, outs, params)
    plan.device_status()
    rng = np.random.default_rng(5)
    for i, (v, t, o) in enumerate(zip(mix, ts, outs)):
        got = o.double().cpu().numpy()
        vals = v.values_f64()
        assert np.array_equal(got[::v.zfactor], vals)
        idx = np.stack([rng.integers(0, v.n_out, 1500), rng.integers(0, v.H, 1500), rng.integers(0, v.W, 1500)], 1)
        border = np.array([[1, 0, 0], [1, v.H - 1, v.W - 1], [v.n_out - 2, 1, v.W - 2], [1, v.H // 2, 0]])
        idx = np.concatenate([idx, border]).astype(np.int64)
        est, _ = oracle.krige_voxels(vals, v.zfactor, v.half_w, idx, **v.variogram())
        scale = max(np.abs(est).max(), np.abs(vals).max())
        assert np.abs(got[idx[:, 0], idx[:, 1], idx[:, 2]] - est).max() <= TOL * scale, v.name
        # the same volume alone in its own launch gives the same bits
        single = binding.Plan([descs[i]], form="DS")
        so = torch.empty_like(o)
        single.interpolate([t], [so], binding.variogram_tensor([v.variogram()]))
        assert torch.equal(so, o), v.name
        single.close()
    plan.close()


def test_autotune_keeps_results_bit_identical(mix):
    sub = mix[:6]
    ts, descs, outs, params = _setup(sub)
    plan = binding.Plan(descs, form="DS")
    plan.interpolate(ts, outs, params)
    ref = [o.clone() for o in outs]
    chunk = plan.autotune(ts, outs, params, iters=2)
    assert chunk >= 1
    c2, bps = plan.schedule()
    assert c2 == min(chunk, max((v.n - 1 + v.n_sub_blocks - 1) // v.n_sub_blocks for v in sub[:1])) and bps in (0, 1)
    for sched in ((chunk, bps), (1, 1), (3, 0)):  # the tuned one, then fixed schedules and launch shapes
        plan.set_schedule(*sched)
        for o in outs:
            o.zero_()
        plan.interpolate(ts, outs, params)
        plan.device_status()
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)
    plan.close()


def test_graph_replay_matches_eager_and_follows_new_parameters(mix):
    sub = mix[6:10]
    ts, descs, outs, params = _setup(sub)
    plan = binding.Plan(descs, form="DS")
    g = plan.capture(ts, outs, params)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    eager = [torch.empty_like(o) for o in outs]
    plan.interpolate(ts, eager, params)
    plan.device_status()
    for a, b in zip(outs, eager):
        assert torch.equal(a, b)
    # new variogram values in the same device buffer are picked up by the next replay
    new = binding.variogram_tensor([dict(v.variogram(), range=5.0, nugget=0.01) for v in sub])
    params.copy_(new)
    g.replay()
    torch.cuda.synchronize()
    plan.interpolate(ts, eager, params)
    plan.device_status()
    for a, b in zip(outs, eager):
        assert torch.equal(a, b)
    plan.close()


def test_variance_class_table_reproduces_the_variance_volume():
    """krig_plan_variance_table: the variance volume rebuilt from the class table and the class
    maps equals, bit for bit, the one krig_interpolate writes (both volumes of a two-volume plan)."""
    vols = [phantoms.random_stack(5, 37, 45, 3, 2, k=2, seed=91, model="exponential"),
            phantoms.random_stack(4, 20, 64, 5, 1, k=1, seed=92)]
    ts = [torch.from_numpy(np.ascontiguousarray(v.slices)).cuda() for v in vols]
    descs = [binding.desc_for(tuple(t.shape), v.zfactor, v.half_w, v.n_sub_blocks, binding.F32)
             for v, t in zip(vols, ts)]
    plan = binding.Plan(descs, form="DS")
    outs = [torch.empty((v.n_out, v.H, v.W), dtype=torch.float32, device="cuda") for v in vols]
    var = [torch.empty_like(o) for o in outs]
    params = binding.variogram_tensor([v.variogram() for v in vols])
    plan.interpolate(ts, outs, params, var)
    plan.device_status()
    for i, v in enumerate(vols):
        table, cx, cy = plan.variance_table(i)
        rebuilt = np.zeros((v.n_out, v.H, v.W), dtype=np.float32)
        for z in range(v.n_out):
            t = z % v.zfactor
            if t:
                rebuilt[z] = table[cy[:, None], cx[None, :], t - 1]
        assert np.array_equal(rebuilt, var[i].cpu().numpy())
    plan.close()
