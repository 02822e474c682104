"""Benchmark of the improved ETD particle-in-cell step on GB300.

Workload (default, `vp1e6`): the Vlasov-Poisson beam with eps = 0.01,
N_p = 1e6 particles, radial mesh of 256 cells on [-4, 4] with linear
deposit/gather, f0 Gaussian in v (v_th = 1) times a Gaussian in r (sigma 1)
truncated to |r| <= 4, macro step dt = 0.1, Lawson RK4 fine solver at
h = 2 pi eps / 100.  One "step" is one macro step of Algorithm ETDFSSModAlgo
for every particle (period detection, fine window with a full field cycle
per stage, landing, extrapolation).  Metric: particle-steps/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload vp1e6|duffing1e4|vp1e8_f32|...] [--no-forms]

`vp1e8_f32` is the FP32 form (precision 1): eps = 0.001, N_p = 1e8, 1024
cells on [-4, 4], dt = 0.1; its line also carries the error of the FP32
form against the FP64 path (itself bit-identical to the FP64 oracle) on a
1e6-particle run of the same physics.

With the default workload at N = 1 the line also carries `forms`: the other
forms measured in the same run, each with its own timing, roofline and
clocks -- the FP32 form on the same physics as the FP64 headline (with its
error against the FP64 path), the learned stepper (with its errors against
the fine-solver reference) beside the plain FP64 and FP32 steps of its own
physics, the batched form, and 150 steps of the headline step for a longer
clock record (`--no-forms` skips them).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the only reference this method has) on a bounded sample of the same
workload.
"""
from __future__ import annotations

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

METRIC = "particle-steps/sec per GB300 (push+deposit+field) at stated error vs FP64 oracle"
UNIT = "particle-steps/s"
# FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA/clk x 2 flop x
# 2.07 GHz = 1.258 TFLOP/s (GB300 nominal 1.25 TFLOP/s; a DFMA probe measured
# 1.19 TFLOP/s at 2070 MHz).
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2.07e9

WORKLOADS = {
    # paper-shaped Vlasov-Poisson run (the metric's workload)
    "vp1e6": dict(n=10**6, params=dict(sort_every=4), r_cut=4.0, desc="Vlasov-Poisson, eps=0.01, N_p=1e6, N_r=256 on [-4,4], CIC, dt=0.1, Lawson RK4 fine step 2*pi*eps/100, FP64"),
    # Duffing test field, periods once at init: no tracking in the window, so the storage order does not
    # matter and the sort is off
    "duffing1e4": dict(n=10**4, params=dict(field_model=1, dt=0.05, periods_once=1, sort_every=0), r_cut=None,
                       desc="Duffing E=-r^3, eps=0.01, N_p=1e4, dt=0.05, periods once, FP64"),
    # comparator schemes (Algorithm ClassicETDAlgo) on the same beam as vp1e6
    "vp1e6_classical": dict(n=10**6, params=dict(), r_cut=4.0, scheme=0,
                            desc="Classical ETD (P = 2 pi eps), Vlasov-Poisson, eps=0.01, N_p=1e6, N_r=256 on [-4,4], "
                                 "dt=0.1, Lawson RK4 fine solver, FP64"),
    "vp1e6_modified": dict(n=10**6, params=dict(), r_cut=4.0, scheme=1,
                           desc="Modified ETD (P = mean first-tour time), Vlasov-Poisson, eps=0.01, N_p=1e6, N_r=256 "
                                "on [-4,4], dt=0.1, Lawson RK4 fine solver, FP64"),
    # learned stepper: network-corrected improved-ETD steps of dt = 0.4 (FP32 form underneath)
    "learned1e7": dict(n=10**7, params=dict(precision=1, dt=0.4, n_cells=512, sort_every=4), r_cut=4.0,
                       learned=dict(train_n=100_000, train_macro=3, steps=1500, batch=8192, tol=1e-4, eval_n=20_000),
                       desc="Learned stepper: Vlasov-Poisson, eps=0.01, N_p=1e7, N_r=512 on [-4,4], CIC, dt=0.4, "
                            "improved-ETD step (FP32 form) + 5-64-64-2 GELU network (BF16 weights, FP32 accumulate), "
                            "frozen-field energy check 1e-4"),
    # batched form: 64 independent beams in one launch per macro step
    "batch64": dict(n=0, params=dict(precision=1), r_cut=4.0,
                    batch=dict(n_beams=64, seed=3, log_n=(4.0, 6.0), eps=(0.1, 0.05, 0.01, 0.005, 0.001),
                               cells=(128, 256, 512, 1024), p_poisson=0.75, dt=0.1),
                    desc="Batched form: 64 independent beams, N_p log-uniform in [1e4, 1e6], eps in "
                         "{0.1, 0.05, 0.01, 0.005, 0.001}, N_r in {128, 256, 512, 1024} on [-4, 4], Poisson (3/4) and "
                         "Duffing (periods once) fields, dt = 0.1, FP32 form, one cooperative graph-replayed launch "
                         "per macro step, autotuned launch shape"),
    # the FP32 form on the physics of vp1e6 (the same-physics comparison with the FP64 headline)
    "vp1e6_f32": dict(n=10**6, params=dict(precision=1, sort_every=4), r_cut=4.0, error_n=10**6, error_steps=20,
                      desc="Vlasov-Poisson FP32 form, eps=0.01, N_p=1e6, N_r=256 on [-4,4], CIC, dt=0.1, Lawson RK4 "
                           "in the rotating frame, binary32 state, FP64 field conversion and diagnostics"),
    # the plain steps on the learned stepper's physics (dt = 0.4, 1e7 particles, 512 cells)
    "learned1e7_plain64": dict(n=10**7, params=dict(precision=0, dt=0.4, n_cells=512, sort_every=4), r_cut=4.0,
                               desc="Plain improved-ETD step (FP64) on the learned stepper's physics: Vlasov-Poisson, "
                                    "eps=0.01, N_p=1e7, N_r=512 on [-4,4], dt=0.4"),
    "learned1e7_plain32": dict(n=10**7, params=dict(precision=1, dt=0.4, n_cells=512, sort_every=4), r_cut=4.0,
                               desc="Plain improved-ETD step (FP32 form) on the learned stepper's physics: "
                                    "Vlasov-Poisson, eps=0.01, N_p=1e7, N_r=512 on [-4,4], dt=0.4"),
    # FP32 form of the same physics at eps = 1e-3 (N about 15 periods per step)
    "vp1e8_f32": dict(n=10**8, params=dict(precision=1, eps=1e-3, n_cells=1024, max_window_steps=202, sort_every=4),
                      r_cut=4.0, error_n=10**6, error_steps=20,
                      desc="Vlasov-Poisson FP32 form, eps=0.001, N_p=1e8, N_r=1024 on [-4,4], CIC, dt=0.1, Lawson RK4 "
                           "in the rotating frame, binary32 state, FP64 field conversion and diagnostics"),
}

# Algorithmic FP64 flops per particle per fine step of the Lawson RK4 window
# (FMA = 2): four stage positions (3+5+5 flops), the update of R and V
# (6+9), and per stage the CIC location, deposit weight and gather (7 x 4).
FLOPS_PER_PARTICLE_FINE_STEP = 56


# FP32 form: the window streams its state; the least a streaming window
# moves is the rotating-frame state of every particle in and out once per
# fine step (8 B + 8 B).
BYTES_PER_PARTICLE_FINE_STEP_F32 = 16

# committed ncu summaries (DRAM traffic of the window kernel) and the sources
# they were taken from
PROFILES = {
    "vp1e6": ("window_coop_vp1e6.md", ["paper_1404_1160_gb300/csrc/window.cu",
                                       "paper_1404_1160_gb300/csrc/window_coop.cuh",
                                       "paper_1404_1160_gb300/csrc/window_common.cuh",
                                       "paper_1404_1160_gb300/csrc/pic_device.cuh"]),
    "vp1e8_f32": ("window32_coop_vp1e8_f32.md", ["paper_1404_1160_gb300/csrc/window32.cu",
                                                 "paper_1404_1160_gb300/csrc/window_common.cuh",
                                                 "paper_1404_1160_gb300/csrc/pic_device.cuh"]),
}


def kernel_sources_sha256(workload: str) -> str:
    import hashlib

    h = hashlib.sha256()
    for f in PROFILES[workload][1]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_traffic(n: int, workload: str):
    """DRAM bytes per window launch from the committed ncu summary, or None
    when the kernel sources changed since it was captured (or no summary)."""
    if workload not in PROFILES or n != WORKLOADS[workload]["n"]:
        return None
    PROFILE = os.path.join(ROOT, "profiles", PROFILES[workload][0])
    if not os.path.exists(PROFILE):
        return None
    sha = bytes_ = None
    for line in open(PROFILE):
        if line.startswith("source_sha256:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            bytes_ = float(line.split(":", 1)[1].strip())
    if sha != kernel_sources_sha256(workload) or bytes_ is None:
        return None
    return bytes_


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while it runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_params(pic, wl):
    return pic.pic_default_params(**WORKLOADS[wl]["params"])


def time_steps(pic, h, do_step, steps, warmup, stream, rank_sync=None):
    """W untimed steps, then K steps each bracketed by CUDA events on the
    handle's stream with an L2 flush (256 MB write) between them, under the
    clock sampler.  Returns (per-step ms, window ms per step, kernel launches,
    wall s, clocks, window launches of the last step)."""
    import torch

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    for _ in range(warmup):
        do_step()
    torch.cuda.synchronize()
    if rank_sync:
        rank_sync()
    launches0 = pic.pic_launch_count(h)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    win_ms, win_n = [], []
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.fill_(float(k))  # L2 flush between timed steps (outside the step events)
            evs[k][0].record(stream)
            do_step()
            evs[k][1].record(stream)
            wt = pic.pic_window_time(h)  # window kernel(s), timed by the library on this stream
            win_ms.append(wt[0])
            win_n.append(int(wt[1]))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    return step_ms, win_ms, pic.pic_launch_count(h) - launches0, wall, clk.summary(), (win_n[-1] if win_n else 0)


def roofline_of(prm, wl_name, n, K, kern_ms, scheme=None, timed_K=None, win_n=0):
    """Roofline object of the dominant kernel: the FP32 window against the
    measured HBM copy bandwidth (streamed bytes), the FP64 window against the
    derived FP64 peak (flops)."""
    if not kern_ms:
        return None
    if prm.field_model != 0:
        return None
    if prm.precision == 1:
        bytes_ = BYTES_PER_PARTICLE_FINE_STEP_F32 * n * K
        achieved = bytes_ / (kern_ms / 1e3)
        peak, peak_src = measured_hbm_peak()
        return {"bound": "hbm", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GB/s",
                "frac": achieved / peak, "traffic": kernel_traffic(n, wl_name),
                "kernel": "k_window32_coop (FP32 form, one launch per macro step)",
                "kernel_ms": kern_ms, "fine_steps_per_launch": K, "algorithmic_bytes_per_launch": bytes_,
                "peak_source": peak_src}
    if scheme is not None:
        # the comparator's step runs several windows (the fine solves over P
        # and o, and for the modified scheme the period detection); its
        # window time is their sum, its fine steps theirs
        K = float(np.mean(timed_K))
        flops = FLOPS_PER_PARTICLE_FINE_STEP * n * K
        achieved = flops / (kern_ms / 1e3)
        return {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_FLOPS, "traffic": None,
                "kernel": "k_window_coop (Lawson RK4 fine solves of the comparator step)",
                "kernel_ms": kern_ms, "fine_steps_per_step": K, "window_launches_per_step": win_n,
                "flops_per_step": flops,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 is not in MEASURED_PEAKS.json)"}
    flops = FLOPS_PER_PARTICLE_FINE_STEP * n * K
    achieved = flops / (kern_ms / 1e3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_FLOPS, "traffic": kernel_traffic(n, wl_name),
            "kernel": "k_window_coop (Lawson RK4, one launch per macro step)",
            "kernel_ms": kern_ms, "fine_steps_per_launch": K, "flops_per_launch": flops,
            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64 is not in MEASURED_PEAKS.json)"}


def measure(wl_name, n, steps, warmup, rank=0, world=1, with_e2e=True, with_errors=True, rank_sync=None):
    """Times `steps` macro steps of a workload (its line, without the
    harness keys).  The network of a learned workload is trained first,
    outside the timed region."""
    import torch

    from paper_1404_1160_gb300 import inputs
    from paper_1404_1160_gb300 import pic

    wl = WORKLOADS[wl_name]
    # replicas: every rank advances its own beam (different seed)
    R0, V0 = inputs.gaussian_beam(n, seed=rank, r_cut=wl["r_cut"])
    prm = make_params(pic, wl_name)
    stream = torch.cuda.current_stream()
    lw = wl.get("learned")
    net = None
    learned_info = None
    if lw:
        from paper_1404_1160_gb300 import learned as _learned

        t_tr = time.perf_counter()
        beam = inputs.gaussian_beam(lw["train_n"], seed=100 + rank, r_cut=wl["r_cut"])
        X, T = _learned.make_dataset(prm, [beam], n_macro=lw["train_macro"], reference="fine")
        net, out_scale, hist, kept = _learned.train(X, T, steps=lw["steps"], batch=lw["batch"], seed=1)
        learned_info = {"train_samples": int(X.shape[0]), "train_steps": lw["steps"], "kept": kept,
                        "loss_first": float(np.mean(hist[:10])), "loss_last": float(np.mean(hist[-50:])),
                        "train_s": time.perf_counter() - t_tr}
    h = pic.pic_init(prm, torch.from_numpy(R0).cuda(), torch.from_numpy(V0).cuda(), stream)
    n_fb = [0]
    scheme = wl.get("scheme")
    classic_K = []  # fine steps of each timed comparator step

    def do_step():
        if scheme is not None:
            classic_K.append(pic.pic_step_classic(h, 1, scheme, with_fine_steps=True)[1])
        elif net is None:
            pic.pic_step(h, 1)
        else:
            n_fb[0] += pic.pic_step_learned(h, net, 1, scale=tuple(out_scale), drift_tol=lw["tol"])

    def reset_counts():
        n_fb[0] = 0
        classic_K.clear()
        if rank_sync:
            rank_sync()

    step_ms, win_ms, launches, wall, clocks, win_n = time_steps(pic, h, do_step, steps, warmup, stream, reset_counts)
    timed_K = classic_K[:steps]
    kernel_ms = [w for w in win_ms if w > 0.0]
    dev_s = sum(step_ms) / 1e3
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([dev_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_s = float(t.item())
    value = world * n * steps / dev_s
    mom = pic.pic_moments(h)
    e2e = None
    if with_e2e:
        # end to end through the public API with host buffers: H2D of the
        # step's input (pinned), the step, D2H of the result
        r_h = torch.from_numpy(R0.copy()).pin_memory()
        v_h = torch.from_numpy(V0.copy()).pin_memory()
        r_o = torch.empty(n, dtype=torch.float64).pin_memory()
        v_o = torch.empty(n, dtype=torch.float64).pin_memory()
        e2e_steps = max(1, min(steps, 5))
        parts = []  # host time of the three calls of each step (they synchronise)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ta = time.perf_counter()
            pic.pic_set_particles(h, r_h, v_h)
            tb = time.perf_counter()
            do_step()
            tc = time.perf_counter()
            pic.pic_get_particles(h, r_o, v_o)
            parts.append((tb - ta, tc - tb, time.perf_counter() - tc))
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        pm = np.mean(np.array(parts), axis=0) * 1e3
        e2e = {"value": world * n * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": 16 * n,
               "mean_ms": {"set_particles": float(pm[0]), "step": float(pm[1]), "get_particles": float(pm[2])}}
    pic.pic_destroy(h)
    if rank != 0:
        if net is not None:
            net.close()
        return None
    K = mom["window_steps"]
    f32 = prm.precision == 1
    roofline = roofline_of(prm, wl_name, n, K, float(np.mean(kernel_ms)) if kernel_ms else None, scheme, timed_K,
                           win_n)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "ms_per_step_min_median_max": [float(np.min(step_ms)), float(np.median(step_ms)), float(np.max(step_ms))],
        "dtype": "f32" if f32 else "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n_particles": n, "fine_steps_per_window": K, "dt": prm.dt,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "L2 flushed between timed steps (256 MB write); per-step trajectory store > L2"},
        "roofline": roofline,
        "gpu_launches": int(launches),
        # FP64 windows that replayed with every trajectory row (the stored
        # band around the forecast landing rows missed one), warm-up included
        "band_replays": int(mom["band_replays"]),
        "wall_s": wall,
        "clocks": clocks,
        "error_vs_oracle": ("FP32 form: see error_vs_fp64 (binary32 bounds checked against the FP64 oracle in the "
                            "parity tests)") if f32 else
                           "bit-identical R, V and charge on the parity tests (tolerance 1e-12 rel)",
    }
    if e2e is not None:
        line["e2e"] = e2e
    if with_errors and f32 and "error_n" in wl:
        line["error_vs_fp64"] = error_vs_fp64(wl_name)
    if lw:
        learned_info["fallback_fraction"] = n_fb[0] / float(n * steps)
        if with_errors:
            learned_info.update(learned_errors(prm, wl, net, out_scale))
        line["learned"] = learned_info
        net.close()
    return line


def form_summary(line, ref_value=None, ref_dt=None):
    """The keys of a form entry: its throughput, timing, roofline, clocks and
    errors; with the FP64 headline's value, the speed-up per macro step and
    per unit of simulated time."""
    keep = ("value", "unit", "ms_per_step", "ms_per_step_min_median_max", "steps", "warmup", "dtype", "config",
            "roofline", "clocks", "band_replays",
            "gpu_launches", "error_vs_fp64", "learned", "error_vs_oracle")
    out = {k: line[k] for k in keep if k in line}
    if ref_value:
        out["vs_fp64_headline"] = line["value"] / ref_value
        dt = line["config"].get("dt")
        if dt and ref_dt:
            out["vs_fp64_headline_per_simulated_time"] = line["value"] * dt / (ref_value * ref_dt)
    return out


def measure_forms(head_line, head_dt):
    """The other forms, measured in the same run as the FP64 headline: the FP32
    form on the same physics, the learned stepper with the plain FP64 and FP32
    steps of its own physics beside it, the batched form, and a longer run of
    the headline step for its clock record.  A form that fails records its error."""
    forms = {}
    ref = head_line["value"]
    plan = [
        ("fp32_same_physics", lambda: form_summary(measure("vp1e6_f32", WORKLOADS["vp1e6_f32"]["n"], 30, 3,
                                                           with_e2e=False), ref, head_dt)),
        ("learned", lambda: form_summary(measure("learned1e7", WORKLOADS["learned1e7"]["n"], 10, 3,
                                                 with_e2e=False), ref, head_dt)),
        ("plain_fp64_learned_physics", lambda: form_summary(measure("learned1e7_plain64",
                                                                    WORKLOADS["learned1e7_plain64"]["n"], 5, 3,
                                                                    with_e2e=False, with_errors=False),
                                                            ref, head_dt)),
        ("plain_fp32_learned_physics", lambda: form_summary(measure("learned1e7_plain32",
                                                                    WORKLOADS["learned1e7_plain32"]["n"], 10, 3,
                                                                    with_e2e=False, with_errors=False),
                                                            ref, head_dt)),
        ("batch64", lambda: form_summary(measure_batch("batch64", 10, 3, with_e2e=False)[0], ref, head_dt)),
        ("fp64_sustained", lambda: form_summary(measure("vp1e6", WORKLOADS["vp1e6"]["n"], 150, 3, with_e2e=False,
                                                        with_errors=False), ref, head_dt)),
    ]
    for name, fn in plan:
        t0 = time.perf_counter()
        try:
            forms[name] = fn()
        except Exception as e:  # a failing form must not lose the headline line
            forms[name] = {"error": f"{type(e).__name__}: {e}"}
        forms[name]["run_s"] = time.perf_counter() - t0
    return forms


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1404_1160_gb300 import build as _build

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()
    wl = WORKLOADS[args.workload]
    n = args.n_particles or wl["n"]
    line = measure(args.workload, n, args.steps, args.warmup, rank, world, with_errors=not args.no_errors,
                   rank_sync=(lambda: dist.barrier()) if world > 1 else None)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample)
    if args.workload == "vp1e6" and world == 1 and not args.no_forms and not args.n_particles:
        line["forms"] = measure_forms(line, WORKLOADS["vp1e6"]["params"].get("dt", 0.1))
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def batch_specs(wl):
    """(pic_params per beam, (R0, V0) per beam) of a batched workload (seeded)."""
    from paper_1404_1160_gb300 import inputs
    from paper_1404_1160_gb300 import pic

    bw = wl["batch"]
    rng = np.random.default_rng(bw["seed"])
    params, beams = [], []
    for i in range(bw["n_beams"]):
        n = int(round(10 ** rng.uniform(*bw["log_n"])))
        eps = float(rng.choice(bw["eps"]))
        cells = int(rng.choice(bw["cells"]))
        poisson = rng.uniform() < bw["p_poisson"]
        if poisson:
            p = pic.pic_default_params(precision=1, eps=eps, dt=bw["dt"], n_cells=cells)
            beams.append(inputs.gaussian_beam(n, seed=1000 + i, r_cut=4.0))
        else:
            p = pic.pic_default_params(precision=1, eps=eps, dt=bw["dt"], field_model=pic.PIC_FIELD_DUFFING,
                                       periods_once=1)
            beams.append(inputs.gaussian_beam(n, seed=1000 + i))
        params.append(p)
    return params, beams


def measure_batch(wl_name, steps, warmup, with_e2e=True):
    """Times `steps` batched macro steps (after autotuning, whose trial steps
    are real steps); returns the line without the harness keys."""
    import torch

    from paper_1404_1160_gb300 import pic

    wl = WORKLOADS[wl_name]
    params, beams = batch_specs(wl)
    sizes = np.array([r.size for r, _ in beams])
    n_total = int(sizes.sum())
    stream = torch.cuda.current_stream()
    b = pic.pic_batch_create(params, beams, stream)
    t_tune = time.perf_counter()
    tuned = pic.pic_batch_tune(b, steps_per_trial=2)  # real steps; they also warm up
    t_tune = time.perf_counter() - t_tune
    pic.pic_batch_step(b, warmup)
    torch.cuda.synchronize()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    launches0 = pic.pic_batch_launch_count(b)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            pic.pic_batch_step(b, 1)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(c) for a, c in evs]
    dev_s = sum(step_ms) / 1e3
    value = n_total * steps / dev_s
    launches = pic.pic_batch_launch_count(b) - launches0
    Ks = np.array([pic.pic_batch_moments(b, i)["window_steps"] for i in range(len(beams))])
    # each beam's own window time in the shared launch (device timer), averaged
    # over three more steps: which beams set the step
    beam_ms = np.zeros(len(beams))
    for _ in range(3):
        pic.pic_batch_step(b, 1)
        beam_ms += np.array([pic.pic_batch_moments(b, i)["window_ms"] for i in range(len(beams))]) / 3.0
    slow = int(np.argmax(beam_ms))
    beam_window = {"max": float(beam_ms.max()), "median": float(np.median(beam_ms)), "min": float(beam_ms.min()),
                   "slowest_beam": {"n_particles": int(sizes[slow]), "eps": float(params[slow].eps),
                                    "n_cells": int(params[slow].n_cells), "field_model": int(params[slow].field_model),
                                    "fine_steps_per_window": int(Ks[slow])}}
    e2e = None
    if with_e2e:
        # end to end with host buffers: every beam's (R, V) in and out each step
        host = [(torch.from_numpy(r.copy()).pin_memory(), torch.from_numpy(v.copy()).pin_memory()) for r, v in beams]
        outs = [(torch.empty(r.size, dtype=torch.float64).pin_memory(),
                 torch.empty(r.size, dtype=torch.float64).pin_memory()) for r, _ in beams]
        e2e_steps = max(1, min(steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for i, (r, v) in enumerate(host):
                pic.pic_batch_set_particles(b, i, r, v)
            pic.pic_batch_step(b, 1)
            for i, (r, v) in enumerate(outs):
                pic.pic_batch_get_particles_into(b, i, r, v)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": n_total * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * n_total,
               "d2h_bytes_per_step": 16 * n_total}
    b.close()
    mean_ms = float(np.mean(step_ms))
    bytes_ = BYTES_PER_PARTICLE_FINE_STEP_F32 * float(np.sum(sizes * Ks))
    peak, peak_src = measured_hbm_peak()
    achieved = bytes_ / (mean_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n_beams": len(beams), "n_particles_total": n_total,
                   "n_particles_min": int(sizes.min()), "n_particles_max": int(sizes.max()), "dt": wl["batch"]["dt"],
                   "fine_steps_per_window_max": int(Ks.max()), "tuned": tuned, "tune_s": t_tune,
                   "beam_window_ms": beam_window,
                   "parallelism": "single GPU", "l2": "L2 flushed between timed steps (256 MB write)"},
        "roofline": {"bound": "hbm", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_window32_batch (all beams, one cooperative launch per macro step)",
                     "kernel_ms": mean_ms, "algorithmic_bytes_per_launch": bytes_,
                     "peak_source": peak_src},
        "gpu_launches": int(launches), "wall_s": wall, "clocks": clk.summary(),
        "error_vs_oracle": "every beam bit-identical to the FP32 form run alone, and every beam of a mixed batch "
                           "within the binary32 bound of the FP64 oracle (tests/test_gpu_batch.py)",
    }
    if e2e is not None:
        line["e2e"] = e2e
    return line, params, beams


def run_batch(args):
    import torch

    from paper_1404_1160_gb300 import build as _build

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _build.build()
    line, params, beams = measure_batch(args.workload, args.steps, args.warmup)
    if rank != 0:
        return
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(params, beams)
    print(json.dumps(line))


def batch_cpu_baseline(params, beams, budget_s: float = 8.0):
    """The FP64 oracle, single-threaded, on the batch's beams in order (each
    cut to at most 2e4 particles) until the time budget is used."""
    import oracle

    done, el, t0 = 0, 0.0, time.perf_counter()
    used = []
    for p, (R, V) in zip(params, beams):
        n = min(R.size, 20_000)
        cfg = oracle.Config(eps=p.eps, dt=p.dt, field_model=p.field_model, fine_solver=1, steps_per_turn=100,
                            n_cells=p.n_cells, r_min=p.r_min, r_max=p.r_max, total_charge=1.0,
                            weight_fixed=p.weight_fixed, max_window_steps=p.max_window_steps)
        T = oracle.periods(cfg, R[:n], V[:n])[0] if p.periods_once else None
        oracle.etd_step(cfg, R[:n], V[:n], T)
        done += n
        used.append(n)
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    return {"value": done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one macro step of each of the first {len(used)} beams, cut to <= 2e4 particles ({el:.1f} s)"}


def learned_errors(prm, wl, net, out_scale):
    """Errors after one macro step of dt, on a held-out sample of the same
    beam, against the reference solution (fine solver over dt on the FP64
    path, bit-identical to the oracle's brute force): the plain large step,
    the learned step, and 8 plain steps of dt/8."""
    import ctypes

    from paper_1404_1160_gb300 import inputs
    from paper_1404_1160_gb300 import pic

    lw = wl["learned"]
    R0, V0 = inputs.gaussian_beam(lw["eval_n"], seed=999, r_cut=wl["r_cut"])

    def clone(**kw):
        p = pic.pic_params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(prm), ctypes.sizeof(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    out = {}
    ref = pic.pic_init(clone(precision=0), R0, V0)
    pic.pic_fine_advance(ref, prm.dt)
    Rf, Vf = pic.pic_get_particles(ref)
    pic.pic_destroy(ref)
    for name, p, how in (("plain", prm, "plain"), ("learned", prm, "learned"), ("plain_8_small", clone(dt=prm.dt / 8), "8")):
        h = pic.pic_init(p, R0, V0)
        if how == "plain":
            pic.pic_step(h, 1)
        elif how == "learned":
            pic.pic_step_learned(h, net, 1, scale=tuple(out_scale), drift_tol=lw["tol"])
        else:
            pic.pic_step(h, 8)
        R, V = pic.pic_get_particles(h)
        pic.pic_destroy(h)
        e = np.sort(np.hypot(R - Rf, V - Vf))
        out[f"err_{name}_median"] = float(np.median(e))
        out[f"err_{name}_rms99"] = float(np.sqrt(np.mean(e[:int(0.99 * e.size)] ** 2)))
    out["error_sample"] = f"{lw['eval_n']} held-out particles of the same beam, one macro step, vs the fine-solver reference"

    # long time: 10 macro steps (t = 10 dt) from the same held-out beam; the
    # reference is the fine solver over the whole time on the FP64 path
    n_long = 10
    ref = pic.pic_init(clone(precision=0), R0, V0)
    m0 = pic.pic_moments(ref)
    pic.pic_fine_advance(ref, n_long * prm.dt)
    Rf, Vf = pic.pic_get_particles(ref)
    mf = pic.pic_moments(ref)
    Qf = pic.pic_get_field(ref, prm.n_cells)[0].astype(np.float64)
    pic.pic_destroy(ref)
    ke0, kef = m0["kinetic"], mf["kinetic"]
    longt = {"macro_steps": n_long, "time": n_long * prm.dt,
             "reference_kinetic_drift": (kef - ke0) / ke0}
    for name, p, how in (("plain", prm, "plain"), ("learned", prm, "learned"), ("plain_8_small", clone(dt=prm.dt / 8), "8")):
        h = pic.pic_init(p, R0, V0)
        if how == "plain":
            pic.pic_step(h, n_long)
        elif how == "learned":
            pic.pic_step_learned(h, net, n_long, scale=tuple(out_scale), drift_tol=lw["tol"])
        else:
            pic.pic_step(h, 8 * n_long)
        R, V = pic.pic_get_particles(h)
        m = pic.pic_moments(h)
        Q = pic.pic_get_field(h, p.n_cells)[0].astype(np.float64)
        pic.pic_destroy(h)
        e = np.hypot(R - Rf, V - Vf)
        longt[f"{name}_err_median"] = float(np.median(e))
        longt[f"{name}_kinetic_drift"] = (m["kinetic"] - ke0) / ke0
        longt[f"{name}_kinetic_vs_reference"] = (m["kinetic"] - kef) / kef
        longt[f"{name}_density_L1_vs_reference"] = float(np.abs(Q - Qf).sum() / Qf.sum())
    out["long_time"] = longt
    return out


FALLBACK_HBM_GBS = 6800.0  # one earlier copy-bandwidth measurement on a GB300


def measured_hbm_peak():
    """HBM peak in B/s and where it comes from: the measured GB300 copy
    bandwidth in MEASURED_PEAKS.json when the file is present, else the
    fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return (float(json.load(fh)["hbm_gbs"]) * 1e9,
                    "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth), of measured")
    except (OSError, ValueError, KeyError, TypeError):
        return (FALLBACK_HBM_GBS * 1e9,
                "6.8 TB/s, an earlier copy-bandwidth measurement on a GB300 (no MEASURED_PEAKS.json), of fallback")


def error_vs_fp64(workload: str):
    """Runs the same seeded beam through the FP32 form and the FP64 path
    (bit-identical to the FP64 oracle) for a number of macro steps and
    compares positions, velocities, energy and charge density."""
    import torch

    from paper_1404_1160_gb300 import inputs
    from paper_1404_1160_gb300 import pic

    wl = WORKLOADS[workload]
    n, steps = wl["error_n"], wl["error_steps"]
    R0, V0 = inputs.gaussian_beam(n, seed=0, r_cut=wl["r_cut"])
    # both start from the same binary32-representable state
    R0 = R0.astype(np.float32).astype(np.float64)
    V0 = V0.astype(np.float32).astype(np.float64)
    out = {}
    for prec in (1, 0):
        prm = pic.pic_default_params(**dict(wl["params"], precision=prec))
        h = pic.pic_init(prm, R0, V0)
        m0 = pic.pic_moments(h)
        pic.pic_step(h, steps)
        R, V = pic.pic_get_particles(h)
        Q, _, _, n_out = pic.pic_get_field(h, prm.n_cells)
        m1 = pic.pic_moments(h)
        pic.pic_destroy(h)
        out[prec] = (R, V, Q, m0, m1)
    R32, V32, Q32, a0, a1 = out[1]
    R64, V64, Q64, b0, b1 = out[0]
    dR, dV = np.abs(R32 - R64), np.abs(V32 - V64)
    torch.cuda.synchronize()
    return {"n_particles": n, "macro_steps": steps, "max_abs_dR": float(dR.max()), "max_abs_dV": float(dV.max()),
            "rms_dR": float(np.sqrt(np.mean(dR * dR))), "rms_dV": float(np.sqrt(np.mean(dV * dV))),
            "kinetic_rel_diff": abs(a1["kinetic"] - b1["kinetic"]) / b1["kinetic"],
            "kinetic_drift_f32": (a1["kinetic"] - a0["kinetic"]) / a0["kinetic"],
            "kinetic_drift_f64": (b1["kinetic"] - b0["kinetic"]) / b0["kinetic"],
            "density_L1_rel": float(np.abs(Q32 - Q64).sum() / np.abs(Q64).sum()),
            "charge_exact_f32": bool(a1["Q_total"] + a1["n_out_of_mesh"] * (1 << 32) == n * (1 << 32)),
            "reference": "FP64 path of this library (bit-identical to the FP64 oracle)"}


def cpu_baseline(workload: str, n_sample: int):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample."""
    import oracle
    from paper_1404_1160_gb300 import inputs

    wl = WORKLOADS[workload]
    n = min(n_sample, wl["n"])
    cfg = oracle_cfg(workload)
    R0, V0 = inputs.gaussian_beam(n, seed=0, r_cut=wl["r_cut"])
    T = None
    if cfg_periods_once(workload):
        T, _, _ = oracle.periods(cfg, R0, V0)
    t0 = time.perf_counter()
    steps = 0
    R, V = R0, V0
    while True:
        if "scheme" in wl:
            R, V, _ = oracle.classic_step(cfg, R, V, wl["scheme"])
        else:
            res = oracle.etd_step(cfg, R, V, T)
            R, V = res.R, res.V
        steps += 1
        el = time.perf_counter() - t0
        if el > 8.0 or steps >= 1000:
            break
    note = " (the plain improved-ETD step: the oracle has no network)" if wl.get("learned") else ""
    return {"value": n * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} macro step(s) of {n} particles of the same workload ({el:.1f} s){note}"}


def cfg_periods_once(workload):
    return bool(WORKLOADS[workload]["params"].get("periods_once", 0))


def oracle_cfg(workload):
    import oracle

    p = dict(eps=0.01, dt=0.1, field_model=0, fine_solver=1, steps_per_turn=100, n_cells=256, r_min=-4.0, r_max=4.0,
             total_charge=1.0, weight_fixed=1 << 32, max_window_steps=300)
    q = dict(WORKLOADS[workload]["params"])
    for k in ("periods_once", "precision", "sort_every"):
        q.pop(k, None)
    p.update(q)
    return oracle.Config(**p)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1404_1160_gb300 import inputs

    oracle.build()
    wl = WORKLOADS[args.workload]
    if "batch" in wl:
        params, beams = batch_specs(wl)
        t0 = time.perf_counter()
        base = None
        for _ in range(args.warmup + args.steps):
            base = batch_cpu_baseline(params, beams, budget_s=2.0)
        value = base["value"]
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": (time.perf_counter() - t0) * 1e3 /
                max(1, args.warmup + args.steps), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": {"workload": wl["desc"]},
                "cpu_baseline": dict(base), "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                    "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    n = min(args.cpu_sample, wl["n"])
    cfg = oracle_cfg(args.workload)
    R, V = inputs.gaussian_beam(n, seed=0, r_cut=wl["r_cut"])
    T = oracle.periods(cfg, R, V)[0] if cfg_periods_once(args.workload) else None
    def one(R, V):
        if "scheme" in wl:
            return oracle.classic_step(cfg, R, V, wl["scheme"])[:2]
        res = oracle.etd_step(cfg, R, V, T)
        return res.R, res.V

    for _ in range(args.warmup):
        R, V = one(R, V)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        R, V = one(R, V)
    el = time.perf_counter() - t0
    value = n * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "n_particles_sample": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: one macro step of {n} particles of the same workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="vp1e6")
    ap.add_argument("--cpu-sample", type=int, default=100_000)
    ap.add_argument("--n-particles", type=int, default=0, help="override N_p (profiling of smaller cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="default workload: skip the other forms")
    ap.add_argument("--no-errors", action="store_true", help="skip the error runs of the FP32 and learned forms")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif "batch" in WORKLOADS[args.workload]:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
