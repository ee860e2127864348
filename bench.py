"""Benchmark: kriged (interpolated) voxels per second on one GB300.

One step = one pass of the kriging path over one batch of synthetic slice
stacks: the geometry-class solve and the stencil apply of the DS form for every
volume of the batch, replayed as one CUDA graph (sub-block partition, class
enumeration and the schedule autotune happen once, on the host, before timing).

The headline workload is the mixed batch: 16 seeded spine/brain float32 stacks
of 128^2..512^2 pixels, 12-40 known slices, Z factors 2-6, 18- or 50-point
windows, all in one persistent launch (about 8.8e7 interpolated voxels per
step).  Beside it the line carries the brain stack (32 x 512^2 float32, g 6,
50 points, exponential) and the spine stack (24 x 256^2 uint16, g 4, 18 points,
spherical variogram fitted to the slices) as full second measurements, the
plain FP64 and mixed per-voxel forms on the headline batch, the leave-one-
slice-out forward + backward on the spine stack, and the error of every output
and gradient against the FP64 oracle.

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
TOL_INTENSITY = 1e-5        # normwise, per volume
TOL_GRAD = 1e-4             # normwise, per tensor

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel, from the ncu capture summarised in profiles/ (None until captured, and again
# whenever the kernel changes).
NCU_TRAFFIC = {
    "batch": 611489280,  # schedule 16 gaps per item, 2 blocks per SM (the autotuner's choice may differ)
    "brain": 183497472,  # part of the output is still in L2 when the captured launch ends
    "spine": None,
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


_ALU = {}


def _alu_peak(fp64):
    """FP32 / FP64 FMA throughput of this GPU in GFLOP/s (the library's FMA microbenchmark), once."""
    from paper_2303_09523_gb300 import binding
    if fp64 not in _ALU:
        _ALU[fp64] = binding.measure_fma_peak(fp64)
    return _ALU[fp64]


def workload(name):
    """The volumes of a workload (a list) and its name."""
    from paper_2303_09523_gb300 import phantoms
    if name == "batch":
        vols = phantoms.batch_mix()
        return vols, "batch16_mixed_128-512_g2-6_r1-2_f32"
    if name == "spine":
        v = phantoms.spine()
        return [v], v.name
    if name == "brain":
        v = phantoms.brain()
        return [v], v.name
    if name == "tiny":
        v = phantoms.tiny_ellipsoids()
        return [v], v.name
    raise SystemExit("unknown workload %s" % name)


def algorithmic_bytes(vol):
    """Bytes a launch of the stencil must move: read every known slice once, write every output slice once."""
    esz_in = vol.slices.dtype.itemsize
    esz_out = 8 if vol.slices.dtype == np.float64 else 4
    return vol.n * vol.H * vol.W * esz_in + vol.n_out * vol.H * vol.W * esz_out


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while a timed region runs (query only)."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.windows = []

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

    def mark(self, name, t0, t1):
        self.windows.append((name, t0, t1))

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @classmethod
    def _parse(cls, lines):
        sm, smax, power, reasons = [], [], [], set()
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < len(cls.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            try:
                power.append(float(parts[2]))
            except ValueError:
                pass
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return sm, smax, power, reasons

    def summary(self):
        """Median SM clock, maximum clock and active throttle reasons over the marked windows (the
        timed steps and the clock pass that replays the same step for at least a second)."""
        per = {}
        all_in = []
        for name, t0, t1 in self.windows:
            inside = [ln for (t, ln) in self.lines if t0 <= t <= t1 + 0.05]
            per[name] = len(inside)
            all_in += inside
        sm, smax, power, reasons = self._parse(all_in)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "samples_per_window": per}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "power_w_max": float(max(power)) if power else None, "samples": len(sm),
                "samples_per_window": per}


# ---------------------------------------------------------------------------
# the FP64 oracle on a bounded sample (CPU baseline and error reference)
# ---------------------------------------------------------------------------

def _sample_missing(vol, count, rng):
    g = vol.zfactor
    j = rng.integers(0, vol.n - 1, count)
    t = rng.integers(1, g, count)
    return np.stack([j * g + t, rng.integers(0, vol.H, count), rng.integers(0, vol.W, count)], 1)


def oracle_sample(vols, target_s=10.0, threads=0, seed=0, with_values=True):
    """Krige a seeded random sample of the missing voxels of the workload with the FP64 oracle, the
    sample split over the volumes in proportion to their missing voxels.  The size is set from a
    short probe so the oracle works for about ``target_s`` seconds.

    Returns dict: ``rate`` (voxels/s over the oracle calls), ``count``, ``seconds``, ``threads``
    (host threads used) and, with ``with_values``, per volume ``idx`` (M x 3 output z, y, x),
    ``est`` and ``var``."""
    import oracle
    rng = np.random.default_rng(seed)
    nmiss = np.array([v.n_missing for v in vols], dtype=np.float64)
    share = nmiss / nmiss.sum()
    vals = [v.values_f64() for v in vols]

    def run(total):
        counts = np.maximum(1, np.round(share * total)).astype(np.int64)
        res, secs = [], 0.0
        for v, s, c in zip(vols, vals, counts):
            idx = _sample_missing(v, int(c), rng)
            t0 = time.perf_counter()
            est, var = oracle.krige_voxels(s, v.zfactor, v.half_w, idx, threads=threads, **v.variogram())
            secs += time.perf_counter() - t0
            res.append({"idx": idx, "est": est, "var": var})
        return res, int(counts.sum()), secs

    _, pc, pt = run(3000 if threads != 1 else 400)
    total = int(max(len(vols), min(20_000_000, pc * target_s / max(pt, 1e-6))))
    res, count, secs = run(total)
    used = threads if threads > 0 else oracle.max_threads()
    out = {"rate": count / secs, "count": count, "seconds": secs, "threads": used}
    if with_values:
        out["per_volume"] = res
    return out


def _gather(t, idx):
    import torch
    ii = torch.from_numpy(idx).to(t.device)
    return t[ii[:, 0], ii[:, 1], ii[:, 2]].double().cpu().numpy()


def err_vs_oracle(outs, variances, sample):
    """Max abs and normwise relative error (max |gpu - oracle| / max |oracle|, per volume, the
    largest over the volumes) of the estimates and variances at the oracle's sample voxels."""
    res = {}
    for key, tens in (("estimate", outs), ("variance", variances)):
        if tens is None:
            continue
        mabs, mrel = 0.0, 0.0
        for t, pv in zip(tens, sample["per_volume"]):
            got = _gather(t, pv["idx"])
            ref = pv["est"] if key == "estimate" else pv["var"]
            d = float(np.abs(got - ref).max())
            mabs = max(mabs, d)
            mrel = max(mrel, d / max(float(np.abs(ref).max()), 1e-300))
        res[key] = {"max_abs": mabs, "max_rel_normwise": mrel, "tolerance": TOL_INTENSITY,
                    "within": mrel <= TOL_INTENSITY}
    res["voxels"] = sample["count"]
    return res


# ---------------------------------------------------------------------------
# the DS path on one workload: graph replay, roofline, clocks, e2e
# ---------------------------------------------------------------------------

class DsHarness:
    """Device buffers, plan (autotuned for batches) and the captured CUDA graph of one workload."""

    def __init__(self, vols, dev, stream, autotune, schedule=None):
        import torch
        from paper_2303_09523_gb300 import binding
        self.vols = vols
        self.dev = dev
        self.stream = stream
        self.host = [torch.from_numpy(np.ascontiguousarray(v.slices)) for v in vols]
        self.ts = [h.to(dev) for h in self.host]
        codes = [binding.dtype_code(t.dtype) for t in self.ts]
        self.descs = [binding.desc_for(tuple(t.shape), v.zfactor, v.half_w, v.n_sub_blocks, c, v.in_scale)
                      for v, t, c in zip(vols, self.ts, codes)]
        self.outs = [torch.empty((v.n_out, v.H, v.W), dtype=binding.out_dtype(c), device=dev)
                     for v, c in zip(vols, codes)]
        self.params = binding.variogram_tensor([v.variogram() for v in vols], device=dev)
        self.plan = binding.Plan(self.descs, form="DS", device=dev)
        self.chunk = None
        if schedule is not None:
            self.plan.set_schedule(*schedule)
            self.chunk = schedule[0]
        elif autotune:
            self.chunk = self.plan.autotune(self.ts, self.outs, self.params, iters=3, stream=stream)
        self.graph = self.plan.capture(self.ts, self.outs, self.params)
        self.n_missing = sum(v.n_missing for v in vols)
        self.abytes = sum(algorithmic_bytes(v) for v in vols)

    def replay(self):
        self.graph.replay()

    def time_steps(self, steps, flush):
        import torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(self.stream)
            self.replay()
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    def kernel_ms(self, iters, flush):
        """Average CUDA-event duration of the class solve and of the stencil per launch, each launch
        bracketed by the library's own events on the launching stream (separate pass: events between
        the two kernels serialise their overlap)."""
        self.plan.set_timing(True)
        self.plan.get_timing()
        for _ in range(iters):
            flush.zero_()
            self.plan.interpolate(self.ts, self.outs, self.params, None, self.stream)
        self.plan.set_timing(False)
        kms, kl = self.plan.get_timing()
        self.plan.device_status(self.stream)
        return kms[0] / max(kl[0], 1), kms[1] / max(kl[1], 1)

    def variances(self):
        import torch
        var = [torch.empty_like(o, dtype=torch.float32) for o in self.outs]
        self.plan.interpolate(self.ts, self.outs, self.params, var, self.stream)
        self.plan.device_status(self.stream)
        return var

    def known_slices_bit_exact(self):
        import torch
        ok = True
        for v, t, o in zip(self.vols, self.ts, self.outs):
            if t.dtype == torch.uint16:
                exp = t.to(torch.float32) * torch.tensor(v.in_scale, dtype=torch.float32, device=t.device)
            else:
                exp = t
            ok = ok and bool(torch.equal(o[::v.zfactor], exp.to(o.dtype)))
        return ok

    def e2e(self, steps):
        """Same step through the public API with the slices in pinned host memory and the output read
        back to pinned host memory every step (copies inside the timed region).  Steps are pipelined
        over two sets of device buffers, each with its own captured graph of the one plan: step i+1's
        slices go up (copy stream) while step i is interpolated (compute stream, the graphs run one
        after the other, never overlapping on the plan's workspace) and step i-1's volumes come down
        (second copy stream).  Returns (ms for the steps, H2D bytes per step, D2H bytes per step,
        pure-copy ms per step measured alone), medians of three interleaved repetitions."""
        import torch
        pin_in = [h.pin_memory() for h in self.host]
        pin_out = [[torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in self.outs] for _ in range(2)]
        ins = [self.ts, [torch.empty_like(t) for t in self.ts]]
        outs = [self.outs, [torch.empty_like(o) for o in self.outs]]
        graphs = [self.graph, self.plan.capture(ins[1], outs[1], self.params)]
        s_in, s_comp, s_out = (torch.cuda.Stream(device=self.dev) for _ in range(3))
        ev = lambda: torch.cuda.Event()  # noqa: E731
        ev_in, ev_comp, ev_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        for b in range(2):  # every buffer starts free
            for e in (ev_comp[b], ev_out[b]):
                e.record(self.stream)

        def step(i):
            b = i % 2
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_comp[b])  # the graph that last read these inputs is done
                for d, h in zip(ins[b], pin_in):
                    d.copy_(h, non_blocking=True)
                ev_in[b].record(s_in)
            with torch.cuda.stream(s_comp):
                s_comp.wait_event(ev_in[b])
                s_comp.wait_event(ev_out[b])  # the outputs of this buffer have been read back
                graphs[b].replay()
                ev_comp[b].record(s_comp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_comp[b])
                for h, o in zip(pin_out[b], outs[b]):
                    h.copy_(o, non_blocking=True)
                ev_out[b].record(s_out)

        def run(n):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            for st in (s_in, s_comp, s_out):
                st.wait_event(e0)
            for i in range(n):
                step(i)
            for st in (s_in, s_comp, s_out):
                self.stream.wait_stream(st)
            e1.record(self.stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        def copies(n):
            # the copies alone (both directions concurrently, same buffers), for the copy bound
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(self.stream)
            for st in (s_in, s_out):
                st.wait_event(c0)
            for i in range(n):
                with torch.cuda.stream(s_in):
                    for d, h in zip(ins[i % 2], pin_in):
                        d.copy_(h, non_blocking=True)
                with torch.cuda.stream(s_out):
                    for h, o in zip(pin_out[i % 2], outs[i % 2]):
                        h.copy_(o, non_blocking=True)
            for st in (s_in, s_out):
                self.stream.wait_stream(st)
            c1.record(self.stream)
            torch.cuda.synchronize()
            return c0.elapsed_time(c1)

        run(3)
        # host-link bandwidth varies on a shared machine: three pipelined runs and three copy-only
        # runs, interleaved; the medians are reported
        e_runs, c_runs = [], []
        for _ in range(3):
            e_runs.append(run(steps))
            c_runs.append(copies(steps) / steps)
        ms = sorted(e_runs)[1]
        bi = sum(h.numel() * h.element_size() for h in pin_in)
        bo = sum(h.numel() * h.element_size() for h in pin_out[0])
        # the second buffer set's outputs must equal the first's (same slices, same plan)
        for a, b_ in zip(outs[0], outs[1]):
            if not torch.equal(a, b_):
                raise RuntimeError("pipelined e2e: the two buffer sets disagree")
        return ms, bi, bo, sorted(c_runs)[1]

    def close(self):
        self.plan.close()


def roofline_of(h, apply_ms, solve_ms, wl_key):
    peak, kind = _peaks()
    achieved = h.abytes / (apply_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": NCU_TRAFFIC.get(wl_key), "kernel": "k_ds_apply", "algorithmic_bytes": h.abytes,
            "avg_launch_ms": apply_ms, "peak_source": kind + " hbm_gbs (burst: the kernel is timed alone)",
            "class_solve_avg_ms": solve_ms}


def measure_workload(wl_key, vols, wl_name, args, dev, stream, flush, world, dist, clk=None, cpu=True,
                     e2e=True, steps=None):
    """Full measurement of the DS path on one workload: timed graph replays, per-kernel roofline,
    clock pass, e2e, error against the FP64 oracle on a seeded sample, the oracle's CPU rate."""
    import torch
    steps = args.steps if steps is None else steps
    h = DsHarness(vols, dev, stream, autotune=len(vols) > 1, schedule=getattr(args, "schedule_tuple", None))
    for _ in range(args.warmup):
        h.replay()
    h.plan.device_status(stream)
    barrier(dist)
    t0 = time.perf_counter()
    step_ms = h.time_steps(steps, flush)
    t1 = time.perf_counter()
    barrier(dist)
    if clk is not None:
        clk.mark(wl_key + ":timed", t0, t1)
    h.plan.device_status(stream)
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    res = {"value": whole_job_rate(h.n_missing, steps, world, total_ms), "unit": "voxels/s",
           "ms_per_step": total_ms / steps, "interpolated_voxels_per_step": h.n_missing,
           "volumes": len(vols), "workload": wl_name}
    if h.chunk is not None:
        res["autotuned_gaps_per_item"], res["autotuned_stencil_blocks_per_sm"] = h.plan.schedule()
    solve_ms, apply_ms = h.kernel_ms(min(max(steps, 20), 200), flush)
    res["roofline"] = roofline_of(h, apply_ms, solve_ms, wl_key)
    if clk is not None:
        # clock pass: the same step replayed for at least a second, so the sampled clocks cover it
        n = max(1, int(1.0 / max(total_ms / steps * 1e-3, 1e-6)))
        c0 = time.perf_counter()
        while time.perf_counter() - c0 < 1.0:
            for _ in range(min(n, 500)):
                h.replay()
            torch.cuda.synchronize()
        clk.mark(wl_key + ":clock_pass", c0, time.perf_counter())
    if e2e:
        ne = max(3, min(steps, 50))
        e_ms, bi, bo, copy_ms = h.e2e(ne)
        e_ms = max_over_ranks(e_ms, dist, dev)
        res["e2e"] = {"value": whole_job_rate(h.n_missing, ne, world, e_ms), "unit": "voxels/s",
                      "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo), "ms_per_step": e_ms / ne,
                      "copy_only_ms_per_step": copy_ms, "frac_of_copy_bound": copy_ms / (e_ms / ne),
                      "pipeline": "two buffer sets: H2D of step i+1, interpolation of step i and D2H of step "
                                  "i-1 on three streams; medians of three runs interleaved with three copy-only runs"}
    if cpu and not args.no_cpu:
        sample = oracle_sample(vols, target_s=args.cpu_s, seed=11)
        var = h.variances()
        torch.cuda.synchronize()
        res["err_vs_oracle"] = err_vs_oracle(h.outs, var, sample)
        res["err_vs_oracle"]["known_slices_bit_exact"] = h.known_slices_bit_exact()
        del var
        single = oracle_sample(vols, target_s=args.cpu_s / 3, threads=1, seed=12, with_values=False)
        res["cpu_baseline"] = {
            "value": sample["rate"], "unit": "voxels/s", "cores": sample["threads"], "kind": "oracle",
            "sample": "%d seeded random missing voxels of %s, split over its volumes by their missing voxels "
                      "(%.1f s on %d threads); single-core: %.4g voxels/s on %d voxels"
                      % (sample["count"], wl_name, sample["seconds"], sample["threads"], single["rate"],
                         single["count"]),
            "single_core": single["rate"]}
        res["_sample"] = sample
    res["_harness"] = h
    return res


def barrier(dist):
    import torch
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step krige a bounded random sample of the workload."""
    if rank != 0:
        return
    vols, name = workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample(vols, target_s=args.ref_step_s / 4, with_values=False)
    t_all, vox, used = 0.0, 0, 1
    for s in range(args.steps):
        r = oracle_sample(vols, target_s=args.ref_step_s, seed=s + 1, with_values=False)
        t_all += r["seconds"]
        vox += r["count"]
        used = r["threads"]
    value = vox / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "form": "oracle FP64 per voxel (Gaussian elimination)"},
        "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": used, "kind": "oracle",
                         "sample": "%d seeded random missing voxels per step of %s" % (vox // args.steps, name)},
        "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line, args)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "brain", "spine", "tiny"])
    ap.add_argument("--forms-steps", type=int, default=1, help="timed calls of each per-voxel form")
    ap.add_argument("--cpu-s", type=float, default=8.0, help="seconds of oracle work per CPU sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline and error sample")
    ap.add_argument("--no-extra", action="store_true", help="skip every line beside the headline")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-voxel P64 / PMX forms")
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--no-fit", action="store_true", help="use the default spine variogram instead of the LOO fit")
    ap.add_argument("--no-loo", action="store_true", help="skip the leave-one-slice-out fwd+bwd timing")
    ap.add_argument("--no-variogram", action="store_true", help="skip the empirical-variogram timing")
    ap.add_argument("--no-downstream", action="store_true",
                    help="skip universal kriging, marching cubes and the similarity metrics")
    ap.add_argument("--results", default=None, help="also append the JSON line to this JSON-lines file")
    ap.add_argument("--schedule", default=None,
                    help="CHUNK,BLOCKS_PER_SM: set the DS schedule instead of autotuning (profiling one fixed launch)")
    ap.add_argument("--loo-workload", default="spine", choices=["spine", "brain"],
                    help="stack of the --section loo measurement")
    ap.add_argument("--section", default=None, choices=["uk", "mc", "sim", "loo", "variogram"],
                    help="run only one of the lines beside the headline and print it (a profiling mode; "
                         "not the benchmark's result line)")
    args = ap.parse_args()
    args.schedule_tuple = tuple(int(x) for x in args.schedule.split(",")) if args.schedule else None
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
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    extra = {}
    if args.section:
        fn = {"uk": time_uk, "mc": time_mc, "sim": similarity_table,
              "loo": lambda a, d, s_, f, with_oracle: time_loo(a, d, s_, f, None, with_oracle=with_oracle,
                                                                workload=a.loo_workload),
              "variogram": lambda a, d, s_, f, with_oracle: time_variogram(a, d, s_, f)}[args.section]
        print(json.dumps({"section": args.section, "result": fn(args, dev, stream, flush, with_oracle=not args.no_cpu)}))
        return
    lead = rank == 0 and world == 1

    # the spine configuration's variogram is fitted to its slices: gradient descent on the
    # leave-one-slice-out loss (CUDA kernels), before anything is timed
    spine_fit = None
    if not args.no_fit and (args.workload == "spine" or (not args.no_extra)):
        from paper_2303_09523_gb300 import fit, phantoms
        sp = phantoms.spine()
        vals = torch.from_numpy(sp.values_f64().astype(np.float32)).to(dev)
        r = fit.fit_variogram_loo(vals, sp.zfactor, sp.half_w, sp.n_sub_blocks, "spherical", sp.sill,
                                  init_range=8.0, init_ratio=0.05, steps=50, lr=0.1)
        spine_fit = {"theta": r["theta"], "loss_first": r["losses"][0], "loss_final": r["loss"],
                     "method": "leave-one-slice-out loss, Adam 50 steps on log range and log nugget/sill"}
        del vals

    def fitted(vols, key):
        if key == "spine" and spine_fit is not None:
            vols[0].nugget, vols[0].sill, vols[0].range = spine_fit["theta"]
        return vols

    vols, wl_name = workload(args.workload)
    vols = fitted(vols, args.workload)
    with ClockSampler(local) as clk:
        clk.wait_first()
        head = measure_workload(args.workload, vols, wl_name, args, dev, stream, flush, world, dist, clk=clk,
                                cpu=rank == 0)
        h = head.pop("_harness")
        sample = head.pop("_sample", None)
        clocks = clk.summary()

    if lead and not args.no_extra:
        if not args.no_forms:
            extra["forms"] = compare_forms(args, h, sample)
            extra["forms"]["DS"] = {"value": head["value"], "unit": "voxels/s", "ms_per_step": head["ms_per_step"],
                                    "err_vs_oracle": (head.get("err_vs_oracle") or {}).get("estimate")}
            extra["forms"]["DS_vs_P64_speedup"] = head["value"] / extra["forms"]["P64"]["value"]
            extra["forms"]["PMX_vs_P64_speedup"] = extra["forms"]["PMX"]["value"] / extra["forms"]["P64"]["value"]
        for key in ("brain", "spine"):
            if key == args.workload:
                continue
            v2, n2 = workload(key)
            v2 = fitted(v2, key)
            r2 = measure_workload(key, v2, n2, args, dev, stream, flush, world, None, cpu=True, e2e=True)
            r2.pop("_harness").close()
            r2.pop("_sample", None)
            r2["config"] = workload_config(v2)
            extra[key] = r2
        if not args.no_loo:
            extra["fwd_bwd"] = time_loo(args, dev, stream, flush, spine_fit, with_oracle=not args.no_cpu)
            extra["fwd_bwd_brain"] = time_loo(args, dev, stream, flush, None, with_oracle=False, workload="brain")
        if not args.no_variogram:
            extra["empirical_variogram"] = time_variogram(args, dev, stream, flush)
        if not args.no_downstream:
            extra["universal_kriging"] = time_uk(args, dev, stream, flush, with_oracle=not args.no_cpu)
            extra["marching_cubes"] = time_mc(args, dev, stream, flush, with_oracle=not args.no_cpu)
            extra["similarity_table1_analogue"] = similarity_table(args, dev, stream, flush,
                                                                   with_oracle=not args.no_cpu)
        peaks = {"fp32_fma_gflops": binding.measure_fma_peak(False), "fp64_fma_gflops": binding.measure_fma_peak(True)}
        extra["alu_peaks_measured"] = peaks
        if "forms" in extra and "P64" in extra["forms"]:
            p = extra["forms"]["P64"]
            p["fp64_roofline"]["peak"] = peaks["fp64_fma_gflops"]
            p["fp64_roofline"]["frac"] = p["fp64_roofline"]["achieved"] / peaks["fp64_fma_gflops"]
    if spine_fit is not None:
        extra["variogram_fit"] = spine_fit

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 stencil / f64-refined f32 solve",
            "data": "synthetic",
            "config": dict(workload_config(vols), workload=wl_name,
                           l2="flushed (512 MB write) before every timed step; inputs + outputs exceed L2",
                           step="one CUDA-graph replay: class solve + persistent stencil over every volume",
                           parallelism="replicas"),
            "roofline": head["roofline"],
            "cpu_baseline": head.get("cpu_baseline"),
            "e2e": head.get("e2e"),
            "err_vs_oracle": head.get("err_vs_oracle"),
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        for k in ("autotuned_gaps_per_item", "autotuned_stencil_blocks_per_sm", "interpolated_voxels_per_step"):
            if k in head:
                line["config"][k] = head[k]
        line.update(extra)
        emit(line, args)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


def workload_config(vols):
    if len(vols) == 1:
        v = vols[0]
        return {"n_known": v.n, "H": v.H, "W": v.W, "zfactor": v.zfactor, "half_w": v.half_w,
                "n_sub_blocks": v.n_sub_blocks, "dtype": str(v.slices.dtype), "variogram": v.variogram(),
                "form": "DS"}
    return {"form": "DS", "volumes": [{"name": v.name, "n_known": v.n, "H": v.H, "W": v.W, "zfactor": v.zfactor,
                                       "half_w": v.half_w, "n_sub_blocks": v.n_sub_blocks,
                                       "model": v.model} for v in vols]}


def time_loo(args, dev, stream, flush, spine_fit, with_oracle=True, workload="spine"):
    """Leave-one-slice-out forward + backward on the spine (or brain) stack (gradients w.r.t. every slice
    voxel and the variogram), replayed as a CUDA graph; gradients compared with the FP64 oracle's."""
    import torch
    from paper_2303_09523_gb300 import binding, phantoms
    vol = phantoms.brain() if workload == "brain" else phantoms.spine()
    theta = dict(model="spherical", nugget=0.0, sill=vol.sill, range=8.0)
    if spine_fit is not None:
        theta.update(nugget=spine_fit["theta"][0], sill=spine_fit["theta"][1], range=spine_fit["theta"][2])
    s_dev = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dev)
    desc = binding.desc_for(tuple(s_dev.shape), vol.zfactor, vol.half_w, vol.n_sub_blocks,
                            binding.dtype_code(s_dev.dtype), vol.in_scale)
    params = binding.variogram_tensor([theta], device=dev)
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
    # launch kernels on the stream they are given)
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
    plan.device_status(stream)
    plan.close()
    nvox = (vol.n - 2) * vol.H * vol.W
    # algorithmic bytes of one forward + backward: the slices read by both passes, the
    # residuals written and read back, dL/dS written
    plane = vol.H * vol.W
    abytes = (2 * vol.n * plane * s_dev.element_size() + 2 * (vol.n - 2) * plane * 4 + vol.n * plane * 4)
    peak, kind = _peaks()
    out = {"value": nvox / (ms * 1e-3), "unit": "LOO-predicted voxels/s (forward + backward)", "ms_per_step": ms,
           "roofline": {"bound": "hbm", "achieved": abytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": abytes / (ms * 1e-3) / 1e9 / peak, "traffic": None, "algorithmic_bytes": abytes,
                        "scope": "whole forward + backward step (six launches)",
                        "peak_source": kind + " hbm_gbs"},
           "replay": "CUDA graph of loo_forward + backward", "workload": vol.name + " (leave-one-slice-out)",
           "voxels_per_step": nvox, "variogram": theta, "loss": float(loss.item()),
           "grad_theta": [float(x) for x in gp.cpu()]}
    if with_oracle:
        import oracle
        ref = oracle.loo(vol.values_f64(), vol.zfactor, vol.half_w, want_grad_theta=True, want_grad_slices=True,
                         **theta)
        g_t = gp.cpu().numpy()
        g_s = gs.double().cpu().numpy()
        et = float(np.abs(g_t - ref["grad_theta"]).max())
        es = float(np.abs(g_s - ref["grad_slices"]).max())
        out["err_vs_oracle"] = {
            "loss": {"max_abs": abs(float(loss.item()) - ref["loss"]),
                     "max_rel": abs(float(loss.item()) - ref["loss"]) / abs(ref["loss"])},
            "grad_theta": {"max_abs": et, "max_rel_normwise": et / float(np.abs(ref["grad_theta"]).max()),
                           "tolerance": TOL_GRAD},
            "grad_slices": {"max_abs": es, "max_rel_normwise": es / float(np.abs(ref["grad_slices"]).max()),
                            "tolerance": TOL_GRAD},
        }
        for k in ("grad_theta", "grad_slices"):
            out["err_vs_oracle"][k]["within"] = out["err_vs_oracle"][k]["max_rel_normwise"] <= TOL_GRAD
    return out


def _graph_time(fn, steps, flush, stream):
    """Average CUDA-event ms of fn() (launches on `stream`) over `steps` calls, L2 flushed before each."""
    import torch
    evs = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def time_uk(args, dev, stream, flush, with_oracle=True):
    """Universal kriging (drift {1, x, y, z}, four known slices) on the spine and brain stacks:
    class solve + stencil replayed as a CUDA graph, error against orc_uk_voxels on a sample."""
    import torch
    from paper_2303_09523_gb300 import binding, phantoms
    res = {}
    for name, vol, count in (("spine", phantoms.spine(), 1500), ("brain", phantoms.brain(), 300)):
        t = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dev)
        code = binding.dtype_code(t.dtype)
        d = binding.desc_for(tuple(t.shape), vol.zfactor, vol.half_w, vol.n_sub_blocks, code, vol.in_scale)
        out = torch.empty((vol.n_out, vol.H, vol.W), dtype=binding.out_dtype(code), device=dev)
        params = binding.variogram_tensor([vol.variogram()], device=dev)
        plan = binding.Plan([d], form="DS", flags=binding.FLAG_DRIFT_XYZ | binding.FLAG_SLABS4, device=dev)
        g = plan.capture([t], [out], params)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        plan.device_status()
        ms = _graph_time(g.replay, max(5, min(args.steps, 50)), flush, stream)
        pts = 4 * (2 * vol.half_w + 1) ** 2
        flops = 2.0 * pts * vol.n_missing  # the weighted sums over the 4-slab neighbourhood
        abytes = vol.n * vol.H * vol.W * t.element_size() + vol.n_out * vol.H * vol.W * out.element_size()
        peak = _alu_peak(False)
        hbm, kind = _peaks()
        r = {"value": vol.n_missing / (ms * 1e-3), "unit": "voxels/s", "ms_per_step": ms, "workload": vol.name,
             "drift": "1, x, y, z", "slabs": 4, "points_per_voxel": pts,
             "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GFLOP/s",
                          "frac": flops / (ms * 1e-3) / 1e9 / peak, "traffic": None,
                          "scope": "whole step (class solve + stencil); 2 flops per point and interpolated voxel",
                          "peak_source": "krig_measure_fma_peak (FP32 FMA microbenchmark)",
                          "hbm_frac": abytes / (ms * 1e-3) / 1e9 / hbm, "algorithmic_bytes": abytes}}
        if with_oracle:
            import oracle
            rng = np.random.default_rng(21)
            idx = _sample_missing(vol, count, rng)
            est, _ = oracle.uk_voxels(vol.values_f64(), vol.zfactor, vol.half_w, idx, slabs=4, drift="xyz",
                                      **vol.variogram())
            got = _gather(out, idx)
            r["err_vs_oracle"] = {"max_abs": float(np.abs(got - est).max()),
                                  "max_rel_normwise": float(np.abs(got - est).max() / np.abs(est).max()),
                                  "voxels": count, "tolerance": TOL_INTENSITY}
        res[name] = r
        plan.close()
    return res


def time_mc(args, dev, stream, flush, with_oracle=True):
    """Marching cubes (Appendix C) on the kriged brain stack (187 x 512 x 512) at iso 0.5: the three
    kernels per call, triangles per call, the volume read once and the triangles written as the
    algorithmic bytes; the triangles of a cropped sub-volume against the oracle."""
    import torch
    from paper_2303_09523_gb300 import binding, phantoms
    vol = phantoms.brain()
    t = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dev)
    outs, _ = binding.krige([dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w, n_sub_blocks=vol.n_sub_blocks,
                                  variogram=vol.variogram())])
    v = outs[0]
    iso = 0.5
    tri, n = binding.marching_cubes(v, iso)
    D, H, W = v.shape
    L = binding.lib()
    work = torch.empty(int(L.krig_marching_cubes_workspace_bytes(D, H, W)), dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    import ctypes

    def call():
        binding._check(L.krig_marching_cubes(ctypes.c_void_p(v.data_ptr()), D, H, W, iso, ctypes.c_void_p(tri.data_ptr()),
                                             tri.shape[0], ctypes.c_void_p(cnt.data_ptr()),
                                             ctypes.c_void_p(work.data_ptr()), work.numel(),
                                             ctypes.c_void_p(stream.cuda_stream)))

    for _ in range(3):
        call()
    ms = _graph_time(call, max(5, min(args.steps, 30)), flush, stream)
    cubes = (D - 1) * (H - 1) * (W - 1)
    abytes = D * H * W * 4 + n * 36
    peak, kind = _peaks()
    r = {"value": cubes / (ms * 1e-3), "unit": "cubes/s", "ms_per_call": ms, "triangles": n, "iso": iso,
         "workload": vol.name + " kriged output",
         "roofline": {"bound": "hbm", "achieved": abytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                      "frac": abytes / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes": abytes,
                      "peak_source": kind + " hbm_gbs"}}
    if with_oracle:
        from oracle import downstream
        # a crop around a vertex of the surface (x, y, z of the middle triangle)
        cx_, cy_, cz_ = (int(c) for c in tri[n // 2, 0].tolist()) if n else (W // 2, H // 2, D // 2)
        z0, y0, x0 = (max(0, min(c - 16, m - 32)) for c, m in ((cz_, D), (cy_, H), (cx_, W)))
        sub = v[z0:z0 + 32, y0:y0 + 32, x0:x0 + 32].contiguous()
        exp = downstream.marching_cubes(sub.cpu().numpy(), np.float32(iso))
        got, m = binding.marching_cubes(sub, iso)
        gh = got.double().cpu().numpy()
        r["crop_vs_oracle"] = {"triangles": m, "oracle_triangles": int(len(exp)),
                               "max_abs_vertex_err": float(np.abs(gh - exp).max()) if len(exp) == m and m else None}
    return r


def similarity_table(args, dev, stream, flush, with_oracle=True):
    """The analogue of the paper's Table 1 on the phantoms: RMSE, MI, ED and SSIM (Appendix D) of every
    interpolated slice (DS kriging on the GPU) against the phantom's noise-free slice at that z,
    computed by krig_similarity, averaged; a few slices checked against the oracle's metrics."""
    import torch
    from paper_2303_09523_gb300 import binding, phantoms
    res = {}
    for name, mk in (("spine", phantoms.spine), ("brain", phantoms.brain)):
        vol = mk(with_truth=True)
        t = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dev)
        outs, _ = binding.krige([dict(slices=t, zfactor=vol.zfactor, half_w=vol.half_w,
                                      n_sub_blocks=vol.n_sub_blocks, variogram=vol.variogram(),
                                      in_scale=vol.in_scale)])
        miss = [z for z in range(vol.n_out) if z % vol.zfactor]
        R = outs[0][miss].contiguous()
        G = torch.from_numpy(vol.truth[miss].astype(np.float32)).to(dev)
        m = binding.similarity(G, R)
        ms = _graph_time(lambda: binding.similarity(G, R, stream=stream), 5, flush, stream)
        mh = m.cpu().numpy()
        varied = G.reshape(len(miss), -1).std(dim=1).cpu().numpy() > 0
        # the pixel pairs are read by the moments pass and again by the histogram pass (4 + 4 bytes each)
        sbytes = 2 * 2 * G.numel() * 4
        hbm, kind = _peaks()
        row = {"images": len(miss), "ms_per_call": ms, "workload": vol.name,
               "roofline": {"bound": "hbm", "achieved": sbytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                            "frac": sbytes / (ms * 1e-3) / 1e9 / hbm, "traffic": None, "algorithmic_bytes": sbytes,
                            "scope": "the four similarity kernels (FP64-pipe bound: sums and logarithms in FP64)",
                            "peak_source": kind + " hbm_gbs"},
               "mean_rmse": float(mh[:, 0].mean()), "mean_mi": float(mh[:, 1].mean()),
               "mean_mi_gg": float(mh[:, 2].mean()), "mean_ed": float(mh[:, 3].mean()),
               "mean_ssim_anatomy_slices": float(mh[varied, 4].mean()) if varied.any() else None}
        if with_oracle:
            from oracle import downstream
            errs = []
            for i in (0, len(miss) // 2, len(miss) - 1):
                Gi = G[i].double().cpu().numpy()
                Ri = R[i].double().cpu().numpy()
                lo, hi = downstream.joint_range(Gi, Ri)
                exp = [downstream.rmse(Gi, Ri), downstream.mutual_information(Gi, Ri),
                       downstream.mutual_information(Gi, Gi), downstream.entropy_difference(Gi, Ri),
                       downstream.ssim_global(Gi, Ri)]
                errs += [abs(mh[i, k] - exp[k]) / max(abs(exp[k]), 1e-12) for k in range(5) if np.isfinite(exp[k])]
            row["max_rel_err_vs_oracle"] = float(max(errs))
        res[name] = row
    return res


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


def time_variogram(args, dev, stream, flush, max_lag=8):
    """Method-of-moments variogram data of the spine stack's known slices (krig_empirical_variogram):
    squared-increment sums for every lag vector |dx|, |dy| <= 8 within a slice and to the next slice.
    FP32-pipe bound: a subtract and a fused multiply-add per voxel pair."""
    import torch
    from paper_2303_09523_gb300 import binding, phantoms
    vol = phantoms.spine()
    s_dev = torch.from_numpy(np.ascontiguousarray(vol.slices)).to(dev)
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
    peak = _alu_peak(False)
    gf = 2.0 * pairs / (ms * 1e-3) / 1e9  # a subtract and a fused multiply-add per voxel pair
    out = {"value": pairs / (ms * 1e-3), "unit": "voxel pairs/s", "ms_per_call": ms, "max_lag": max_lag,
           "lag_vectors": int(counts.size), "pairs_per_call": pairs, "workload": vol.name,
           "roofline": {"bound": "alu", "achieved": gf, "peak": peak, "unit": "GFLOP/s", "frac": gf / peak,
                        "traffic": None, "scope": "k_emp_variogram; 2 flops per voxel pair",
                        "peak_source": "krig_measure_fma_peak (FP32 FMA microbenchmark)"}}
    # the fit uses the widest lags the kernel stages (16 pixels: distance classes to about 23 voxels)
    sums16, counts16 = binding.empirical_variogram(s_dev, 16, in_scale=vol.in_scale, stream=stream)
    out["fit"] = variogram_fits(sums16.cpu().numpy(), counts16, vol)
    return out


def variogram_fits(sums, counts, vol):
    """Weighted least-squares fit of the workload's model to the empirical variogram (distance
    classes of the per-lag-vector sums)."""
    from paper_2303_09523_gb300 import fit
    res = {"model": vol.model}
    try:
        h, gamma, n = fit.variogram_bins(sums, counts, vol.zfactor)
        r = fit.fit_variogram_wls(h, gamma, n, vol.model)
    except Exception as e:  # scipy missing, or no fit: the line reports it instead of failing the run
        res["wls"] = "unavailable: %s" % e
        return res
    nug, sill, rng = r["theta"]
    res["wls"] = {"nugget": nug, "sill": sill, "range": rng, "classes": int(len(h)), "max_lag_length": float(h.max()),
                  "range_at_bound": r["range_at_bound"], "max_lag": 16}
    return res


def p64_flops_per_voxel(vol):
    """FP64 flops of one interior voxel's P64 solve: Cholesky K^3/3, four triangular sweeps 4K^2, combine 6K."""
    K = 2 * (2 * vol.half_w + 1) ** 2
    return K ** 3 / 3.0 + 4.0 * K * K + 6.0 * K


def compare_forms(args, h, sample):
    """Plain FP64 per-voxel form (P64) and the mixed per-voxel form (PMX) on the headline workload, each
    against the FP64 oracle at the sample voxels; DS against P64 over every output voxel."""
    import torch
    from paper_2303_09523_gb300 import binding
    res = {}
    ref = None
    for form in ("P64", "PMX"):
        plan = binding.Plan(h.descs, form=form, device=h.dev)
        o = [torch.empty_like(x) for x in h.outs]
        plan.interpolate(h.ts, o, h.params, None, h.stream)
        plan.device_status(h.stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(h.stream)
        for _ in range(args.forms_steps):
            plan.interpolate(h.ts, o, h.params, None, h.stream)
        b.record(h.stream)
        torch.cuda.synchronize()
        plan.device_status(h.stream)
        ms = a.elapsed_time(b) / args.forms_steps
        res[form] = {"value": h.n_missing / (ms * 1e-3), "unit": "voxels/s", "ms_per_step": ms}
        if sample is not None:
            res[form]["err_vs_oracle"] = err_vs_oracle(o, None, sample)["estimate"]
        if form == "P64":
            ref = o
            fl = sum(p64_flops_per_voxel(v) * v.n_missing for v in h.vols)
            gfl = fl / (ms * 1e-3) / 1e9
            res[form]["fp64_roofline"] = {"bound": "fp64", "achieved": gfl, "peak": None, "unit": "GFLOP/s",
                                          "frac": None, "flops_per_step": fl,
                                          "peak_source": "krig_measure_fma_peak (FP64 FMA microbenchmark)"}
        else:
            res[form]["max_rel_err_vs_P64"] = max(float((x.double() - y.double()).abs().max() / y.double().abs().max())
                                                  for x, y in zip(o, ref))
        plan.close()
        del o
    res["DS_max_rel_err_vs_P64"] = max(float((x.double() - y.double()).abs().max() / y.double().abs().max())
                                       for x, y in zip(h.outs, ref))
    return res


if __name__ == "__main__":
    main()
