"""Benchmark: kriged (interpolated) voxels per second on one GB300.

One step = one pass of the kriging path over one synthetic slice stack: the
geometry-class solve and the stencil apply of the DS form (sub-block
partition and class enumeration are planned once, on the host).  The headline
workload is the spine-like stack: 24 known 256x256 uint16 slices, Z factor 4
(93 output slices), 4 Z sub-blocks, 18-point window, spherical variogram.

Prints one JSON line (rank 0).  See ``--help`` for options.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kriged voxels/s on 1 GB300, mixed/batched vs plain FP64 at stated err; fwd+bwd vox/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel, from the ncu capture summarised in profiles/ (None until captured, and again
# whenever the kernel changes).  Under ncu replay part of the output is still in L2 when
# the launch ends, so these read below the algorithmic bytes.
NCU_TRAFFIC = {
    "spine": 3590656 + 25088,
    "brain": 34455040 + 139843840,
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(name):
    from paper_2303_09523_gb300 import phantoms
    if name == "spine":
        return phantoms.spine()
    if name == "brain":
        return phantoms.brain()
    if name == "tiny":
        return phantoms.tiny_ellipsoids()
    raise SystemExit("unknown workload %s" % name)


def algorithmic_bytes(vol):
    """Bytes a launch of the stencil must move: read every known slice once, write every output slice once."""
    esz_in = vol.slices.dtype.itemsize
    esz_out = 8 if vol.slices.dtype == np.float64 else 4
    return vol.n * vol.H * vol.W * esz_in + vol.n_out * vol.H * vol.W * esz_out


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=5.0):
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        t0, t1 = getattr(self, "window", (-1e30, 1e30))
        inside = [ln for (t, ln) in self.lines if t0 <= t <= t1 + 0.05]
        lines = inside if inside else [ln for (_, ln) in self.lines]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_timed_region": len(inside)}


def cpu_oracle_rate(vol, target_s=12.0, threads=0, seed=0):
    """Time the FP64 oracle on a bounded random sample of missing voxels of the workload."""
    import oracle
    vals = vol.values_f64()
    g = vol.zfactor
    rng = np.random.default_rng(seed)

    def sample(count):
        j = rng.integers(0, vol.n - 1, count)
        t = rng.integers(1, g, count)
        return np.stack([j * g + t, rng.integers(0, vol.H, count), rng.integers(0, vol.W, count)], 1)

    probe = sample(2000 if threads != 1 else 300)
    t0 = time.perf_counter()
    oracle.krige_voxels(vals, g, vol.half_w, probe, threads=threads, **vol.variogram())
    dt = time.perf_counter() - t0
    count = int(max(1000, min(5_000_000, len(probe) * target_s / max(dt, 1e-6))))
    idx = sample(count)
    t0 = time.perf_counter()
    oracle.krige_voxels(vals, g, vol.half_w, idx, threads=threads, **vol.variogram())
    dt = time.perf_counter() - t0
    used = threads if threads > 0 else oracle.max_threads()
    return count / dt, count, dt, used


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step krige a bounded random sample of the workload."""
    if rank != 0:
        return
    vol = workload(args.workload)
    rates = []
    for _ in range(args.warmup):
        cpu_oracle_rate(vol, target_s=args.ref_step_s / 4)
    t_all = 0.0
    vox = 0
    for s in range(args.steps):
        rate, count, dt, used = cpu_oracle_rate(vol, target_s=args.ref_step_s, seed=s + 1)
        rates.append(rate)
        t_all += dt
        vox += count
    value = vox / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": vol.name, "form": "oracle FP64 per voxel (Gaussian elimination)"},
        "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": used, "kind": "oracle",
                         "sample": "%d random missing voxels per step of %s" % (vox // args.steps, vol.name)},
        "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line, args)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="spine", choices=["spine", "brain", "tiny"])
    ap.add_argument("--forms-steps", type=int, default=3, help="steps for the per-voxel forms comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip form comparison and at-scale lines")
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--no-fit", action="store_true", help="use the default variogram instead of the LOO fit")
    ap.add_argument("--no-loo", action="store_true", help="skip the leave-one-slice-out fwd+bwd timing")
    ap.add_argument("--no-batch", action="store_true", help="skip the 16-volume batched graph-replay timing")
    ap.add_argument("--no-variogram", action="store_true", help="skip the empirical-variogram timing")
    ap.add_argument("--results", default=None, help="also append the JSON line to this JSON-lines file")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mine":
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_2303_09523_gb300 import binding

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl", device_id=dev)
        dist = dist_

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    vol = workload(args.workload)
    s_host = torch.from_numpy(np.ascontiguousarray(vol.slices))
    s_dev = s_host.to(dev)
    variogram_fit = None
    if args.workload == "spine" and not args.no_fit:
        # the spine configuration uses a spherical variogram fitted to the slice data: fit it by gradient
        # descent on the leave-one-slice-out loss (CUDA kernels), before anything is timed
        from paper_2303_09523_gb300 import fit
        vals = torch.from_numpy(vol.values_f64().astype(np.float32)).to(dev)
        res = fit.fit_variogram_loo(vals, vol.zfactor, vol.half_w, vol.n_sub_blocks, "spherical", vol.sill,
                                    init_range=8.0, init_ratio=0.05, steps=50, lr=0.1)
        vol.nugget, vol.sill, vol.range = res["theta"]
        variogram_fit = {"method": "leave-one-slice-out loss, Adam 50 steps on log range and log nugget/sill",
                         "loss_first": res["losses"][0], "loss_final": res["loss"]}
    code = binding.dtype_code(s_dev.dtype)
    desc = binding.desc_for(tuple(s_dev.shape), vol.zfactor, vol.half_w, vol.n_sub_blocks, code, vol.in_scale)
    out_dt = binding.out_dtype(code)
    out = torch.empty((vol.n_out, vol.H, vol.W), dtype=out_dt, device=dev)
    params = binding.variogram_tensor([vol.variogram()], device=dev)
    plan = binding.Plan([desc], form="DS", device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.interpolate([s_dev], [out], params, None, stream)

    for _ in range(args.warmup):
        step()
    plan.device_status(stream)

    # ---------------- timed region (device time, L2 flushed before every step)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        clk.wait_first()
        t_wall = time.perf_counter()
        t_start = t_wall
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
        clk.mark(t_start, t_start + t_wall)
    plan.device_status(stream)
    # per-kernel durations (for the roofline), measured in a separate pass: the
    # library's events between the two kernels would serialise their overlap
    plan.set_timing(True)
    plan.get_timing()
    for i in range(min(args.steps, 200)):
        flush.zero_()
        step()
    plan.set_timing(False)
    kms, klaunch = plan.get_timing()
    plan.device_status(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    vox_step = vol.n_missing
    value = whole_job_rate(vox_step, args.steps, world, total_ms)

    # dominant kernel (stencil apply) roofline
    peak, peak_kind = _peaks()
    apply_ms = kms[1] / max(klaunch[1], 1)
    solve_ms = kms[0] / max(klaunch[0], 1)
    abytes = algorithmic_bytes(vol)
    achieved = abytes / (apply_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": NCU_TRAFFIC.get(args.workload), "kernel": "k_ds_apply",
                "algorithmic_bytes": abytes, "avg_launch_ms": apply_ms, "peak_source": peak_kind + " hbm_gbs",
                "class_solve_avg_ms": solve_ms}

    # ---------------- end to end through the public API with host buffers
    s_pin = s_host.pin_memory()
    out_pin = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
    s_stage = torch.empty_like(s_dev)

    def e2e_step():
        s_stage.copy_(s_pin, non_blocking=True)
        plan.interpolate([s_stage], [out], params, None, stream)
        out_pin.copy_(out, non_blocking=True)

    for _ in range(3):
        e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    e2e = {"value": whole_job_rate(vox_step, args.steps, world, e2e_ms), "unit": "voxels/s",
           "h2d_bytes_per_step": int(s_pin.numel() * s_pin.element_size()),
           "d2h_bytes_per_step": int(out_pin.numel() * out_pin.element_size())}

    extra = {}
    if not args.no_extra and rank == 0:
        peaks = {"fp32_fma_gflops": binding.measure_fma_peak(False), "fp64_fma_gflops": binding.measure_fma_peak(True)}
        extra = compare_forms(args, vol, s_dev, desc, params, out, dev, stream, peaks)
        extra["alu_peaks_measured"] = peaks
    if rank == 0 and not args.no_loo:
        extra["fwd_bwd"] = time_loo(args, vol, s_dev, desc, params, dev, stream, flush)
    if rank == 0 and not args.no_batch:
        extra["batched"] = time_batch(args, dev, stream, flush)
    if rank == 0 and not args.no_variogram:
        extra["empirical_variogram"] = time_variogram(args, vol, s_dev, stream, flush,
                                                      extra.get("alu_peaks_measured"))
    if variogram_fit is not None:
        extra["variogram_fit"] = variogram_fit

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        rate, count, dt, used = cpu_oracle_rate(vol, target_s=12.0)
        rate1, count1, dt1, _ = cpu_oracle_rate(vol, target_s=4.0, threads=1)
        cpu = {"value": rate, "unit": "voxels/s", "cores": used, "kind": "oracle",
               "sample": "%d random missing voxels of %s (%.1f s); single-core: %.4g voxels/s on %d voxels"
                         % (count, vol.name, dt, rate1, count1)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 stencil / f64-refined f32 solve",
            "data": "synthetic",
            "config": {"workload": vol.name, "form": "DS", "n_known": vol.n, "H": vol.H, "W": vol.W,
                       "zfactor": vol.zfactor, "half_w": vol.half_w, "n_sub_blocks": vol.n_sub_blocks,
                       "variogram": vol.variogram(), "interpolated_voxels_per_step": vox_step,
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": "replicas"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
            "wall_s_timed_region": t_wall,
        }
        line.update(extra)
        emit(line, args)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


def time_loo(args, vol, s_dev, desc, params, dev, stream, flush):
    """Leave-one-slice-out forward + backward (gradients w.r.t. every slice voxel and the variogram)."""
    import torch
    from paper_2303_09523_gb300 import binding
    plan = binding.Plan([desc], form="DS", flags=binding.FLAG_LOO, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gl = torch.ones(1, dtype=torch.float64, device=dev)
    gs = torch.empty(s_dev.shape, dtype=torch.float32, device=dev)
    gp = torch.empty(3, dtype=torch.float64, device=dev)

    def step(st):
        plan.loo_forward([s_dev], params, loss, None, st)
        plan.backward([s_dev], params, gl, [gs], gp, False, st)

    for _ in range(max(3, args.warmup)):
        step(stream)
    plan.device_status(stream)
    # the forward + backward pair replayed as one CUDA graph (the calls only
    # launch kernels and memsets on the stream they are given)
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        step(cap)
    stream.wait_stream(cap)
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    plan.close()
    nvox = (vol.n - 2) * vol.H * vol.W
    return {"value": nvox / (ms * 1e-3), "unit": "LOO-predicted voxels/s (forward + backward)", "ms_per_step": ms,
            "replay": "CUDA graph of loo_forward + backward",
            "voxels_per_step": nvox, "loss": float(loss.item()),
            "grad_theta": [float(x) for x in gp.cpu()]}


def emit(line, args):
    """The run's one JSON line on stdout, and appended to ``--results`` (JSON lines) if given."""
    text = json.dumps(line)
    print(text, flush=True)
    if getattr(args, "results", None):
        with open(args.results, "a") as f:
            f.write(text + "\n")


def max_over_ranks(x, dist, device):
    """The slowest rank's value (the job ends with it): an all-reduce (max) across the process
    group, or x itself when there is one process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, world, ms):
    """Units per second of the whole job: every rank processes units_per_step per step (weak
    scaling, independent replicas), all done when the slowest rank's ms have passed."""
    return units_per_step * steps * world / (ms * 1e-3)


def time_variogram(args, vol, s_dev, stream, flush, peaks, max_lag=8):
    """Method-of-moments variogram data of the workload's known slices (krig_empirical_variogram):
    squared-increment sums for every lag vector |dx|, |dy| <= 8 within a slice and to the next slice.
    FP32-pipe bound: a subtract and a fused multiply-add per voxel pair."""
    import torch
    from paper_2303_09523_gb300 import binding
    for _ in range(max(3, args.warmup)):
        sums, counts = binding.empirical_variogram(s_dev, max_lag, in_scale=vol.in_scale, stream=stream)
    evs = []
    steps = min(args.steps, 50)
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        binding.empirical_variogram(s_dev, max_lag, in_scale=vol.in_scale, stream=stream)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    pairs = int(counts.sum())
    out = {"value": pairs / (ms * 1e-3), "unit": "voxel pairs/s", "ms_per_call": ms, "max_lag": max_lag,
           "lag_vectors": int(counts.size), "pairs_per_call": pairs}
    out["fit"] = variogram_fits(sums.cpu().numpy(), counts, vol)
    if peaks:
        peak = peaks["fp32_fma_gflops"] * 1e9 / 2 / 2  # FP32 instructions/s, two per pair
        out["roofline"] = {"bound": "alu", "achieved": pairs / (ms * 1e-3), "peak": peak, "unit": "pairs/s",
                           "frac": pairs / (ms * 1e-3) / peak,
                           "peak_source": "measured FP32 FMA rate / 2 instructions per pair"}
    return out


def variogram_fits(sums, counts, vol):
    """Weighted least-squares fit of the workload's model to the empirical variogram (distance
    classes of the per-lag-vector sums), beside the variogram the benchmark interpolates with."""
    from paper_2303_09523_gb300 import fit
    res = {"model": vol.model, "used": {"nugget": vol.nugget, "sill": vol.sill, "range": vol.range}}
    try:
        h, gamma, n = fit.variogram_bins(sums, counts, vol.zfactor)
        r = fit.fit_variogram_wls(h, gamma, n, vol.model)
    except Exception as e:  # scipy missing, or no fit: the line reports it instead of failing the run
        res["wls"] = "unavailable: %s" % e
        return res
    nug, sill, rng = r["theta"]
    res["wls"] = {"nugget": nug, "sill": sill, "range": rng, "classes": int(len(h)), "max_lag_length": float(h.max())}
    return res


def time_batch(args, dev, stream, flush):
    """16 uneven spine/brain volumes in one DS call: autotuned schedule, captured in a CUDA graph, replayed."""
    import torch
    from paper_2303_09523_gb300 import binding, phantoms
    vols = phantoms.batch_mix()
    ts = [torch.from_numpy(np.ascontiguousarray(v.slices)).to(dev) for v in vols]
    descs = [binding.desc_for(tuple(t.shape), v.zfactor, v.half_w, v.n_sub_blocks, binding.dtype_code(t.dtype),
                              v.in_scale) for v, t in zip(vols, ts)]
    outs = [torch.empty((v.n_out, v.H, v.W), dtype=torch.float32, device=dev) for v in vols]
    params = binding.variogram_tensor([v.variogram() for v in vols], device=dev)
    plan = binding.Plan(descs, form="DS", device=dev)
    chunk = plan.autotune(ts, outs, params, iters=3, stream=stream)
    g = plan.capture(ts, outs, params)
    torch.cuda.synchronize()
    steps = max(10, args.steps // 10)
    for _ in range(3):
        g.replay()
    evs = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    plan.device_status()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    nvox = sum(v.n_missing for v in vols)
    abytes = sum(algorithmic_bytes(v) for v in vols)
    peak, kind = _peaks()
    plan.close()
    return {"value": nvox / (ms * 1e-3), "unit": "voxels/s", "ms_per_step": ms, "volumes": len(vols),
            "interpolated_voxels_per_step": nvox, "autotuned_gaps_per_item": chunk,
            "step_bytes_per_s": abytes / (ms * 1e-3), "frac_of_hbm_peak": abytes / (ms * 1e-3) / (peak * 1e9),
            "replay": "CUDA graph (class solve + stencil, programmatic dependent launch)"}


def p64_flops_per_voxel(vol):
    """FP64 flops of one interior voxel's P64 solve: Cholesky K^3/3, four triangular sweeps 4K^2, combine 6K."""
    K = 2 * (2 * vol.half_w + 1) ** 2
    return K ** 3 / 3.0 + 4.0 * K * K + 6.0 * K


def compare_forms(args, vol, s_dev, desc, params, out_ds, dev, stream, peaks):
    """Plain FP64 per-voxel form (P64) and the mixed per-voxel form (PMX) on the same workload."""
    import torch
    from paper_2303_09523_gb300 import binding
    res = {}
    ref = None
    for form in ("P64", "PMX"):
        plan = binding.Plan([desc], form=form, device=dev)
        o = torch.empty_like(out_ds)
        plan.interpolate([s_dev], [o], params, None, stream)
        plan.device_status(stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.forms_steps):
            plan.interpolate([s_dev], [o], params, None, stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.forms_steps
        res[form] = {"value": vol.n_missing / (ms * 1e-3), "unit": "voxels/s", "ms_per_step": ms}
        if form == "P64":
            ref = o.double()
            gfl = p64_flops_per_voxel(vol) * vol.n_missing / (ms * 1e-3) / 1e9
            res[form]["fp64_roofline"] = {"bound": "fp64", "achieved": gfl, "peak": peaks["fp64_fma_gflops"],
                                          "unit": "GFLOP/s", "frac": gfl / peaks["fp64_fma_gflops"],
                                          "flops_per_voxel": p64_flops_per_voxel(vol),
                                          "peak_source": "krig_measure_fma_peak (FP64 FMA microbenchmark)"}
        else:
            res[form]["max_rel_err_vs_P64"] = float((o.double() - ref).abs().max() / ref.abs().max())
        plan.close()
    res["DS_max_rel_err_vs_P64"] = float((out_ds.double() - ref).abs().max() / ref.abs().max())
    return {"forms": res}


if __name__ == "__main__":
    main()
