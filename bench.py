#!/usr/bin/env python3
"""Benchmark: FSE / EPI seconds at 27,525,120 isochromats on one GB300,
grouped vs plain GPU forms, signal rel-L2 against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mrsim|reference]

One step = one grouped FP32 simulation of the 2-D FSE workload (512 x 512 x
105 isochromats, ETL 16, 256 phase encodes, 3 ms sinc pulses at 1 us) on a
phantom resident in HBM: combined-transition precompute, the fused
isochromat pass, the group-signal pass and the signal read-back.  Grouping
(classification + group build + layout) is prepared once per phantom and is
reported separately (`prep_s`), and again inside the end-to-end figure,
which runs the whole public API from pinned host buffers every step.

Also reported on the same GPU: grouped EPI, plain (per-isochromat) FSE and
EPI, plain+cache FSE, per-kernel device times, the roofline of the dominant
kernel, and the FP64 oracle timed on this host's cores on a sample.

`--impl reference` times the FP64 CPU oracle (the reference arm of this
build) on a bounded isochromat sample of the same workload and prints the
same JSON line with "impl": "reference".
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FSE/EPI seconds @27.5M isochromats, grouped vs plain GPU, rel-L2≤1e-4 vs FP64"
WORKLOAD = ("fse_27m: 2-D FSE, 512x512 in-plane x 105 z-subvoxels = 27,525,120 isochromats, "
            "8-ellipse phantom (seed 1002), 3 ms Hamming-sinc 90x/180y at 1 us, ETL 16, "
            "256 phase encodes in 16 shots, 256 samples at 4 us, ESP 8 ms, TR 3 s")
GOLDEN = os.path.join(ROOT, "tests", "golden")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    try:
                        rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                    except ValueError:
                        pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        power = [r[2] for r in rows]
        thr = 0.5 * max(power)
        load = [r for r in rows if r[2] >= thr] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load)}


# The source a fused kernel is compiled from: whole files, or (file, first
# line's text, text of the line that ends the part) for the part of a shared
# header that holds the kernel's argument and event records.
FUSED_SOURCES = {"fused_cell": ("k_cell.cu", "common.cuh",
                                ("internal.h", "// Cell mode of the fused kernel",
                                 "struct CellKey {")),
                 "fused_grouped": ("k_grouped.cu", "common.cuh")}


def kernel_source_sha(kind):
    import hashlib
    h = hashlib.sha256()
    for src in FUSED_SOURCES[kind]:
        name, first, stop = (src, None, None) if isinstance(src, str) else src
        with open(os.path.join(ROOT, "paper_2508_03960_gb300", "csrc", name), "rb") as f:
            data = f.read()
        if first is not None:
            i = data.index(first.encode())
            data = data[i:data.index(stop.encode(), i)]
        h.update(data)
    return h.hexdigest()


def fused_traffic(K, kind="fused_cell"):
    """DRAM bytes per fused-kernel launch from the committed ncu summary,
    scaled by K; None once the kernel source differs from the profiled one."""
    path = os.path.join(ROOT, "profiles", f"{kind}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if kernel_source_sha(kind) != rec.get("source_sha256"):
        return None
    return int(rec["dram_bytes_per_isochromat"] * K)


def cell_event_work(seq, mrsim, hs):
    """Events of the cell form of the fused kernel for a sequence whose
    with-ADC windows are Gx-only and with-RF subsequences Gz-only (primary
    axis x, secondary z, free axis y), and which of them rotate by the
    free-axis phasor (nonzero y moment since the state time, Eqs. 4-5):
    returns (RF + END events, those with the y phasor, ADC windows, those
    with the y phasor)."""
    info = mrsim.mrsim_seq_info(hs)
    gy = seq.gy.astype(np.float64) * seq.dt * seq.repeat
    my = 0.0
    rf = rf_q = adc = adc_q = 0
    for t, b, e in zip(info["type"], info["seg_begin"], info["seg_end"]):
        if t == 0:  # with-RF
            rf += 1
            rf_q += my != 0.0
            my = 0.0
        elif t == 1:  # with-ADC
            adc += 1
            adc_q += my != 0.0
            my += float(gy[b:e].sum())
        else:
            my += float(gy[b:e].sum())
    return rf + 1, rf_q + (my != 0.0), adc, adc_q


def batch_workload(ctx, mrsim, torch, steps, warmup, mixed=False):
    """64 independent jobs of uneven size (4k-2M isochromats, log-uniform),
    round-robin SE / GRE / FSE(ETL 8), in one batched graph launch per step,
    against the same jobs run one after the other.  mixed: 32 jobs (4k-500k)
    of which a quarter each start from a given state, receive with two coils
    or have subsequences without a gradient type (configs.batch_job_mixed)."""
    from mrsim_inputs import configs
    sizes = configs.batch_sizes(32, kmax=500_000) if mixed else configs.batch_sizes()
    make = configs.batch_job_mixed if mixed else configs.batch_job
    hps, hss, hgs, sigs = [], [], [], []
    K_total = 0
    for i, K in enumerate(sizes):
        ph, seq = make(i, K)
        hp = ctx.phantom(ph)
        hs = ctx.sequence(seq)
        hgs.append(ctx.group(hp, hs))
        hps.append(hp)
        hss.append(hs)
        n_coils = 0 if ph.coils is None else ph.coils.shape[0]
        sigs.append(np.zeros(2 * max(seq.n_samples, 1) * max(n_coils, 1)))
        K_total += ph.K
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        mrsim.mrsim_run_batch(ctx.h, hps, hss, hgs, sigs)
    torch.cuda.synchronize()
    n0 = mrsim.mrsim_launch_count(ctx.h)
    e0.record(stream)
    for _ in range(steps):
        mrsim.mrsim_run_batch(ctx.h, hps, hss, hgs, sigs)
    e1.record(stream)
    torch.cuda.synchronize()
    batched = e0.elapsed_time(e1) / steps / 1e3
    batch_sigs = [x.copy() for x in sigs]

    def one_by_one():
        for hp, hs, hg, sg in zip(hps, hss, hgs, sigs):
            mrsim.mrsim_run(ctx.h, hp, hs, hg, mrsim.GROUPED, mrsim.FP32, sg)

    one_by_one()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        one_by_one()
    e1.record(stream)
    torch.cuda.synchronize()
    sequential = e0.elapsed_time(e1) / steps / 1e3
    worst = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
                for a, b in zip(batch_sigs, sigs))
    return {"jobs": len(sizes), "isochromats": int(K_total), "batched_s": round(batched, 6),
            "one_by_one_s": round(sequential, 6), "speedup": round(sequential / batched, 2),
            "max_rel_l2_batched_vs_single": worst, "graph_launches_per_batched_step": 1}


SUR_LO = [-0.010, -80.0, 0.8, 0.3, 0.04]  # z (m), dB0 (Hz), b1, T1 (s), T2 (s)
SUR_HI = [0.010, 80.0, 1.2, 1.5, 0.2]


def surrogate_workload(ctx, mrsim, torch):
    """Learned with-RF transitions: train on 4M draws of the FSE pulses with
    2 ms sinc at 10 us, then simulate that FSE on a 27.5M-isochromat phantom
    with per-isochromat dB0 ~ N(0, 20 Hz) and b1 ~ U[0.8, 1.2] (so nearly
    every isochromat is its own group), exact preparation vs the network."""
    from mrsim_inputs import configs
    from mrsim_inputs.phantom import continuous_phantom
    _, seq = configs.surrogate_fse()
    hs = ctx.sequence(seq)
    t0 = time.perf_counter()
    # batch 4096: twice the optimizer steps of 8192 over the same 300 epochs
    # (two trainings each: 51-75 % of the gate's cells served, against 38-58 %)
    sur = mrsim.mrsim_surrogate_train(ctx.h, hs, SUR_LO, SUR_HI, n_train=1 << 22, epochs=300,
                                      batch=4096, lr=1e-2, seed=1005, bound=1e-3)
    train_s = time.perf_counter() - t0
    st = mrsim.mrsim_surrogate_stats(sur)
    ph = continuous_phantom(512, 512, 105, 8, seed=1005)
    hp = ctx.phantom(ph)
    # launch parameters tuned on the FSE (945 pulse groups) do not carry over to
    # 27.5M pulse groups: the preparation step uses its size heuristic here
    lanes_tuned = mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES, 0)
    t0 = time.perf_counter()
    hg = ctx.group(hp, hs)
    group_s = time.perf_counter() - t0
    sig = torch.zeros(2 * seq.n_samples, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(mode, reps=2):
        mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps / 1e3
        # per-kernel split of one more run (CUDA events around each launch)
        mrsim.mrsim_profile_reset(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, True)
        mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)
        torch.cuda.synchronize()
        prof = {k: round(v[1], 3) for k, v in mrsim.mrsim_profile_get(ctx.h).items() if v[0]}
        mrsim.mrsim_profile_enable(ctx.h, False)
        return t, sig.cpu().numpy().view(np.complex128).copy(), prof

    t_exact, s_exact, k_exact = timed(mrsim.GROUPED)
    mrsim.mrsim_surrogate_use(ctx.h, sur)
    t_sur, s_sur, k_sur = timed(mrsim.SURROGATE)
    run = mrsim.mrsim_surrogate_stats(sur, ctx.h)
    mrsim.mrsim_surrogate_use(ctx.h, None)
    n_served, n_exact = run["groups_served"], run["groups_exact"]
    # the gate's bound on this run's own groups: every served transition
    # against its exact FP64 counterpart
    run_err, run_served = mrsim.mrsim_surrogate_check(ctx.h, sur, hs, hg)
    out = {"K": ph.K, "groups_z": mrsim.mrsim_group_info(hg, mrsim.G_Z)[0],
           "train": {"samples_per_pulse": 1 << 22, "epochs": 300, "batch": 4096,
                     "seconds": round(train_s, 2),
                     "final_mse_per_entry": st["train_loss"],
                     "validation_max_error": st["val_max_err"],
                     "cells_served": st["cells_served"],
                     "served_max_error": st["val_served_max_err"], "bound": 1e-3,
                     "gate_margin": 0.5},
           "served_max_error_on_run": run_err, "served_pairs_checked": run_served,
           "grouping_s": round(group_s, 3), "exact_s": round(t_exact, 4),
           "surrogate_s": round(t_sur, 4), "speedup": round(t_exact / t_sur, 3),
           "kernels_ms_exact": k_exact, "kernels_ms_surrogate": k_sur,
           "preparation_ms": {"exact": k_exact.get("precompute_f32", 0.0),
                              "surrogate": round(sum(k_sur.get(n, 0.0) for n in
                                                     ("precompute_f32", "sur_gate",
                                                      "sur_infer")), 3)},
           "groups_served_fraction": round(n_served / max(n_served + n_exact, 1), 4),
           # the counters add up every run since mrsim_surrogate_use: timed() makes
           # 1 + reps + 1 = 4 runs
           "groups_served_per_run": int(n_served) // 4, "sur_infer_ms": k_sur.get("sur_infer"),
           "signal_rel_l2_vs_exact": float(np.linalg.norm(s_sur - s_exact) / np.linalg.norm(s_exact))}
    ctx.free("grp", hg)
    ctx.free("ph", hp)
    mrsim.mrsim_free_surrogate(sur)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES, lanes_tuned)
    out["precompute_lanes"] = "size heuristic"
    return out


def multicoil_workload(ctx, mrsim, torch, ph, seq, hp_single, hg_single, steps, n_coils=8):
    """The grouped FSE received by n_coils coils (Eq. 6 with P coils): one
    preparation step, then fused passes of up to four coils each (the cell
    form shares the state evolution between them).  Coil maps from
    mrsim_inputs.coil_maps on a second handle of the same phantom."""
    from mrsim_inputs import coil_maps
    t0 = time.perf_counter()
    S = coil_maps(ph, n_coils, seed=1006)
    maps_s = time.perf_counter() - t0
    hp = ctx.phantom(ph)
    mrsim.mrsim_coils(ctx.h, hp, S)
    del S
    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    ns = seq.n_samples
    sig = torch.zeros(n_coils * 2 * ns, dtype=torch.float64, device="cuda")
    run = lambda: mrsim.mrsim_run(ctx.h, hp, hs, hg, mrsim.GROUPED, mrsim.FP32, sig, None,
                                  mrsim.OUT_DEVICE)
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / steps / 1e3
    out = {"coils": n_coils, "fse_grouped_s": round(t, 5),
           "per_coil_ms": round(t / n_coils * 1e3, 3), "coil_maps_host_s": round(maps_s, 2),
           "note": "one preparation step and fused passes of up to 4 coils; coil signals "
                   "checked against the FP64 oracle in tests/test_gpu_coils.py"}
    ctx.free("grp", hg)
    ctx.free("seq", hs)
    ctx.free("ph", hp)
    return out


def radial_workload(ctx, mrsim, torch, hp, K, steps):
    """Radial readouts at 27.5M isochromats: 62 of the 64 spokes read on Gx and
    Gy together (two-axis with-ADC windows, the open problem of Sec. 5).  The
    same GPU runs them grouped on both positions, with two-axis typing off
    (those windows per isochromat, the conventional fallback) and fully per
    isochromat (plain)."""
    from mrsim_inputs import configs
    seq = configs.radial_sequence()
    stream = torch.cuda.current_stream()
    sig = torch.zeros(2 * seq.n_samples, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(hs, hg, mode, reps, warm=True):
        if warm:
            mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)
        mrsim.mrsim_profile_reset(ctx.h)
        mrsim.mrsim_profile_enable(ctx.h, True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = {k: round(v[1] / reps, 3) for k, v in mrsim.mrsim_profile_get(ctx.h).items()
                if v[0]}
        mrsim.mrsim_profile_enable(ctx.h, False)
        return e0.elapsed_time(e1) / reps / 1e3, sig.cpu().numpy().view(np.complex128).copy(), prof

    hs = ctx.sequence(seq)
    hg = ctx.group(hp, hs)
    groups = {n: mrsim.mrsim_group_info(hg, t)[0] for n, t in
              (("xy", mrsim.G_XY), ("x", mrsim.G_X), ("y", mrsim.G_Y), ("z", mrsim.G_Z))}
    t_g, s_g, k_g = timed(hs, hg, mrsim.GROUPED, steps)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 0)
    hs0 = ctx.sequence(seq)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_TWO_AXIS, 1)
    hg0 = ctx.group(hp, hs0)
    t_f, s_f, k_f = timed(hs0, hg0, mrsim.GROUPED, 1)
    t_p, s_p, k_p = timed(hs, None, mrsim.PLAIN, 1, warm=False)
    ctx.free("grp", hg0)
    ctx.free("seq", hs0)
    ctx.free("grp", hg)
    ctx.free("seq", hs)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"K": K, "spokes": 64, "samples": seq.n_samples, "groups": groups,
            "grouped_two_axis_s": round(t_g, 5), "general_fallback_s": round(t_f, 4),
            "plain_s": round(t_p, 3), "speedup_vs_plain": round(t_p / t_g, 1),
            "speedup_vs_general_fallback": round(t_f / t_g, 1),
            "kernels_ms_grouped": k_g, "kernels_ms_general_fallback": k_f,
            "kernels_ms_plain": k_p,
            "rel_l2_grouped_vs_plain": rel(s_g, s_p),
            "rel_l2_fallback_vs_plain": rel(s_f, s_p)}


def recon_workload(ctx, mrsim, torch, named_signals, steps):
    """Images of the simulated FSE and EPI k-space (mrsim_recon_cartesian on
    device buffers), timed with CUDA events, against the oracle's (numpy FFT)
    reconstruction of the stored FP64 oracle signals."""
    from mrsim_inputs.sequence import kspace_layout
    from oracle.recon import recon_cartesian
    out = {}
    stream = torch.cuda.current_stream()
    for name, seq, sig in named_signals:
        L = kspace_layout(seq)
        d_sig = torch.from_numpy(np.ascontiguousarray(sig).view(np.float64).copy()).cuda()
        d_img = torch.zeros(2 * L["n_pe"] * L["n_ro"], dtype=torch.float64, device="cuda")
        mrsim.mrsim_recon_cartesian(ctx.h, d_sig, L, d_img, mrsim.PTR_DEVICE)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            mrsim.mrsim_recon_cartesian(ctx.h, d_sig, L, d_img, mrsim.PTR_DEVICE)
        e1.record(stream)
        torch.cuda.synchronize()
        img = d_img.cpu().numpy().view(np.complex128).reshape(L["n_pe"], L["n_ro"])
        ent = {"matrix": [L["n_pe"], L["n_ro"]], "ms": round(e0.elapsed_time(e1) / steps, 4)}
        path = os.path.join(GOLDEN, f"{name}_27m_oracle.npz")
        if os.path.exists(path):
            ref = recon_cartesian(np.load(path)["signal"], L)
            ent["image_rel_l2_vs_oracle"] = float(np.linalg.norm(img - ref) / np.linalg.norm(ref))
        out[name] = ent
    return out


def cluster_workload(ctx, mrsim, torch, seqs, reps=2, sizes=(64, 128, 256)):
    """Group-reducing preprocessing (Sec. 3.3, Fig. 4) of the 27.5M-isochromat
    parameter-mapping phantom (T1 / T2 snapped to 100 log-spaced candidates,
    smooth dB0 field, so that nearly every isochromat is its own Gz group):
    clustering time, group counts and grouped time before and after for each
    (name, sequence) of ``seqs``, the signal error the clustering costs (rel-L2
    of the clustered phantom's grouped signal against the unclustered
    phantom's) and, as in Figs. 6-7, the error of the reconstructed images
    (mrsim_recon_cartesian) against the unclustered phantom's image."""
    from mrsim_inputs import configs
    from mrsim_inputs.sequence import kspace_layout
    ph = configs.mapped_27m()
    hp = ctx.phantom(ph)
    hss = [(name, seq, ctx.sequence(seq)) for name, seq in seqs]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def simulate(h, seq, hs):
        sig = torch.zeros(2 * seq.n_samples, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t = time.perf_counter()
        hg = ctx.group(h, hs)
        group_s = time.perf_counter() - t
        counts = {"gx": mrsim.mrsim_group_info(hg, mrsim.G_X)[0],
                  "gz": mrsim.mrsim_group_info(hg, mrsim.G_Z)[0]}
        run = lambda: mrsim.mrsim_run(ctx.h, h, hs, hg, mrsim.GROUPED, mrsim.FP32, sig, None,
                                      mrsim.OUT_DEVICE)
        run()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        s = sig.cpu().numpy().view(np.complex128).copy()
        ctx.free("grp", hg)
        return {"s": round(e0.elapsed_time(e1) / reps / 1e3, 5), "groups": counts,
                "grouping_s": round(group_s, 3)}, s

    def image_error(s, s0, seq):
        try:
            L = kspace_layout(seq)
            im, im0 = (mrsim.mrsim_recon_cartesian(ctx.h, np.ascontiguousarray(x), L)
                       for x in (s, s0))
            d = np.abs(im - im0)
            return {"image_rel_l2": float(np.linalg.norm(d) / np.linalg.norm(im0)),
                    "image_max_error_of_peak": float(d.max() / np.abs(im0).max())}
        except Exception as e:  # the signal figures stand without the image
            return {"image_error": f"{type(e).__name__}: {e}"}

    ref = {}
    out = {"K": ph.K, "phantom": "mapped_27m (seed 1006): 16 regions, T1/T2 on 100 log-spaced "
                                 "candidates, dB0 smooth field (20 Hz scale)",
           "unclustered": {}, "clustered": [],
           "precompute_lanes": "size heuristic (the headline's tuned lane count suits its "
                               "945 pulse groups, not one group per isochromat)"}
    lanes_tuned = mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES, 0)
    # a failure in one sequence is reported under its name; the others stand
    for name, seq, hs in hss:
        try:
            out["unclustered"][name], ref[name] = simulate(hp, seq, hs)
        except Exception as e:
            out["unclustered"][name] = {"error": f"{type(e).__name__}: {e}"}
    for n in sizes:
        torch.cuda.synchronize()
        t = time.perf_counter()
        h, m, _, _ = ctx.cluster(hp, ph.K, n, want_labels=False)
        ent = {"n_clusters": m, "cluster_s": round(time.perf_counter() - t, 4)}
        for name, seq, hs in hss:
            if name not in ref:
                continue
            try:
                r, s = simulate(h, seq, hs)
                r["speedup_vs_unclustered"] = round(out["unclustered"][name]["s"] / r["s"], 2)
                r["signal_rel_l2_vs_unclustered"] = float(np.linalg.norm(s - ref[name]) /
                                                          np.linalg.norm(ref[name]))
                r.update(image_error(s, ref[name], seq))
            except Exception as e:
                r = {"error": f"{type(e).__name__}: {e}"}
            ent[name] = r
        out["clustered"].append(ent)
        ctx.free("ph", h)
    # per-kernel split of one clustering into the largest size (CUDA events)
    mrsim.mrsim_profile_reset(ctx.h)
    mrsim.mrsim_profile_enable(ctx.h, True)
    h, _, _, _ = ctx.cluster(hp, ph.K, sizes[-1], want_labels=False)
    torch.cuda.synchronize()
    out["kernels"] = {k: [int(v[0]), round(v[1], 4)]
                      for k, v in mrsim.mrsim_profile_get(ctx.h).items() if v[0]}
    mrsim.mrsim_profile_enable(ctx.h, False)
    ctx.free("ph", h)
    for _, _, hs in hss:
        ctx.free("seq", hs)
    ctx.free("ph", hp)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_PRECOMP_LANES, lanes_tuned)
    return out


def golden_check(name, sig, ph_digest, seq_digest):
    path = os.path.join(GOLDEN, f"{name}_27m_oracle.npz")
    if not os.path.exists(path):
        return None
    import oracle
    d = np.load(path)
    if str(d["phantom_digest"]) != ph_digest or str(d["sequence_digest"]) != seq_digest:
        return {"error": "stored oracle signal was made from different inputs"}
    return float(oracle.rel_l2(sig, d["signal"]))


def cpu_baseline(ph, seq, stride, threads=0):
    """FP64 oracle on every `stride`-th isochromat; time extrapolated to K
    (run time is linear in K: isochromats are independent)."""
    import oracle
    sub = ph.subset(np.arange(0, ph.K, stride))
    t0 = time.perf_counter()
    oracle.simulate(sub, seq, memo=True, adc_recurrence=True, n_threads=threads, want_M=False)
    wall = time.perf_counter() - t0
    cores = threads if threads > 0 else os.cpu_count()
    return wall * ph.K / sub.K, wall, sub.K, cores


def reduce_max(v, dist=None, device="cuda"):
    """Largest v over the ranks of the default process group (the slowest
    replica's time); v itself without a process group."""
    if not dist:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rf_runs(seq):
    """With-RF subsequences of a sequence (maximal runs of segments with RF):
    total sub-steps and segments over all of them, and sub-steps summed over
    the distinct ones (exact equality of their segments)."""
    rf = (seq.b1re != 0) | (seq.b1im != 0)
    edges = np.flatnonzero(np.diff(np.concatenate([[0], rf.astype(np.int8), [0]])))
    steps = segs = distinct_steps = 0
    seen = set()
    for b, e in zip(edges[0::2], edges[1::2]):
        n = int(seq.repeat[b:e].astype(np.int64).sum())
        steps += n
        segs += int(e - b)
        key = b"".join(np.ascontiguousarray(getattr(seq, f)[b:e]).tobytes()
                       for f in ("dt", "repeat", "b1re", "b1im", "gx", "gy", "gz"))
        if key not in seen:
            seen.add(key)
            distinct_steps += n
    return steps, segs, distinct_steps


# algorithmic work of the other kernels (flops, FMA = 2, sin / cos / exp = 1 each):
#   plain step (App. A per sub-step): |phi|^2 5, series of sin(t)/t and
#     (1-cos t)/t^2 16, two cross products 18, M += s q + c2 w 12, relaxation 7
#     -> 58 per isochromat-step, plus the rotation vector 10 per isochromat-segment
#   plain ADC (Eq. 6): phasor recurrence 6 + sum 2 -> 8 per isochromat-sample
#   group signal (Eqs. 8, 10): phase 4, sin + cos + exp 3, complex rotate-scale-add 10
#     -> 17 per (sample, group)
#   preparation (Eq. 7, FP32 runs): U - I 40, FP32 block composition 72, FP64 fold
#     every 8 steps ~9 -> ~120 per (group, sub-step)
#   network inference, 128x128 layer on tensor cores (h1 as hi + lo BF16 halves):
#     2 x 2 x 128 x 128 = 65,536 per served group
FLOPS_PLAIN_STEP, FLOPS_PLAIN_SEG, FLOPS_PLAIN_SAMPLE = 58, 10, 8
FLOPS_GSIG, FLOPS_PREP, FLOPS_SUR_INFER = 17, 120, 65536


def roof_entry_hbm(name, nbytes, ms, peak_gbs, unit_note):
    ach = nbytes / (ms / 1e3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": round(peak_gbs, 1),
            "unit": "GB/s", "frac": round(ach / peak_gbs, 4), "algorithmic_bytes": nbytes,
            "ms": round(ms, 4), "work": unit_note}


def roof_entry(name, flops, ms, peak, bound, unit_note):
    ach = flops / (ms / 1e3) / 1e12
    return {"kernel": name, "bound": bound, "achieved": round(ach, 3), "peak": round(peak, 2),
            "unit": "TFLOP/s", "frac": round(ach / peak, 4), "algorithmic_flops": flops,
            "ms": round(ms, 4), "work": unit_note}


# algorithmic FP32 work of the fused kernel (cell form) per isochromat and
# event, and the fewest thread instructions that can do it:
#   with-RF / END event: M <- C (Q M) with the cell's combined row C = T Adv:
#     3 rows x 4 FMA = 24 flops (12 FFMA); with a free-axis moment, Q M adds one
#     phasor load, its address and a complex rotation (4 FFMA/FMUL): 30 flops,
#     18 instructions
#   with-ADC window: sum of Q M_xy (4 FFMA = 8 flops) plus the phasor load and
#     its address: 6 instructions; without a free-axis moment 2 adds (4 flops)
# The per-thread and per-group work (secondary-axis phasor, group factor,
# staging, the flush) is amortised over the thread's isochromats and left out.
FLOPS_CELL_RF, FLOPS_CELL_RF_Q, FLOPS_CELL_ADC, FLOPS_CELL_ADC_Q = 24, 30, 4, 8
INST_CELL_RF, INST_CELL_RF_Q, INST_CELL_ADC, INST_CELL_ADC_Q = 12, 18, 2, 6


def profile_prep(configs):
    """One preparation of the 27.5M FSE through the public API, each call timed
    on the host clock (synchronised), with the library's kernel times."""
    import torch
    from paper_2508_03960_gb300 import mrsim
    ph, fse = configs.fse_27m()
    ctx = mrsim.Context(0, torch.cuda.current_stream().cuda_stream)
    mrsim.mrsim_profile_enable(ctx.h, True)
    split = {}

    def lap(name, fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        split[name] = round((time.perf_counter() - t) * 1e3, 2)
        return r

    hp = lap("phantom_upload", lambda: ctx.phantom(ph))
    hs = lap("sequence", lambda: ctx.sequence(fse))
    hg = lap("group", lambda: ctx.group(hp, hs))
    prof = mrsim.mrsim_profile_get(ctx.h)
    mrsim.mrsim_profile_enable(ctx.h, False)
    print(json.dumps({"case": "prep_fse_27m", "K": ph.K, "split_ms": split,
                      "groups": {"gx": mrsim.mrsim_group_info(hg, mrsim.G_X)[0],
                                 "gz": mrsim.mrsim_group_info(hg, mrsim.G_Z)[0]},
                      "kernels": {k: [v[0], round(v[1], 3)] for k, v in prof.items() if v[0]}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrsim", choices=["mrsim", "reference"])
    ap.add_argument("--plain-fse", default="on", choices=["on", "off"],
                    help="time one plain (per-isochromat) FSE run (~tens of seconds)")
    ap.add_argument("--cpu-stride", type=int, default=128)
    ap.add_argument("--case", default="fse_27m", choices=["fse_27m", "fse_6m"],
                    help="fse_6m: the same sequences on a 256x256x105 phantom (profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="only the grouped FSE/EPI steps (for profiler launch lists)")
    ap.add_argument("--tune", default="on", choices=["on", "off"],
                    help="off: default launch parameters, no autotuner launches (profiling)")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="one small run of each kernel besides the fused one, in this order: "
                         "plain EPI, grouped FSE, surrogate FSE on a continuous phantom "
                         "(for ncu captures; prints their CUDA-event times)")
    ap.add_argument("--profile-cluster", action="store_true",
                    help="time the clustering preprocessing kernels (27.5M, 256 clusters)")
    ap.add_argument("--profile-prep", action="store_true",
                    help="one preparation of the 27.5M FSE through the API (phantom upload, "
                         "sequence, groups and layout), for profiler launch lists; prints "
                         "the host-clock split and the kernels' CUDA-event times")
    a = ap.parse_args()
    a.warmup = max(3, a.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from mrsim_inputs import configs, phantom_digest, sequence_digest

    if a.profile_cluster:
        profile_cluster(a, configs)
        return
    if a.profile_kernels:
        profile_kernels(a, configs)
        return
    if a.profile_prep:
        profile_prep(configs)
        return

    if a.impl == "reference":
        if rank != 0:
            return
        reference_arm(a, configs)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_03960_gb300 import mrsim

    ph = configs.full_phantom() if a.case == "fse_27m" else configs.small_phantom(256, 256, 105)
    fse = configs.fse_sequence()
    epi = configs.epi_sequence()
    stream = torch.cuda.current_stream()
    ctx = mrsim.Context(local, stream.cuda_stream)
    pk, pk_kind = peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def maxr(v):
        return reduce_max(v, dist, "cuda")

    # ---- resident phantom, prepared sequences and groups (once per phantom) ----
    t0 = time.perf_counter()
    hp = ctx.phantom(ph)
    torch.cuda.synchronize()
    t_upload = time.perf_counter() - t0
    t0 = time.perf_counter()
    hs_f = ctx.sequence(fse)
    hg_f = ctx.group(hp, hs_f)
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    hs_e = ctx.sequence(epi)
    hg_e = ctx.group(hp, hs_e)
    groups = {n: mrsim.mrsim_group_info(hg_f, t)[0] for n, t in (("gx", mrsim.G_X), ("gz", mrsim.G_Z))}

    # autotuner: launch parameters picked by timing the grouped FSE run itself
    t0 = time.perf_counter()
    if a.tune == "on":
        tuned = mrsim.mrsim_autotune(ctx.h, hp, hs_f, hg_f, mrsim.GROUPED, mrsim.FP32, 2)
    else:
        tuned = {p: mrsim.mrsim_get_tuning(ctx.h, p) for p in
                 (mrsim.TUNE_FUSED_NI, mrsim.TUNE_PLAIN_RF_NI, mrsim.TUNE_ADC_CTAS_PER_SM,
                  mrsim.TUNE_PRECOMP_LANES, mrsim.TUNE_PRECOMP_STEPS, mrsim.TUNE_CELL_NI,
                  mrsim.TUNE_CELL_ROWS)}
    autotune_s = time.perf_counter() - t0

    ns_f, ns_e = fse.n_samples, epi.n_samples
    sig_f = torch.zeros(2 * ns_f, dtype=torch.float64, device="cuda")
    sig_e = torch.zeros(2 * ns_e, dtype=torch.float64, device="cuda")

    def step(hs, hg, sig, mode=mrsim.GROUPED):
        mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)

    # ---- headline: grouped FSE ----
    for _ in range(a.warmup):
        step(hs_f, hg_f, sig_f)
    mrsim.mrsim_profile_reset(ctx.h)
    mrsim.mrsim_profile_enable(ctx.h, True)
    n_launch0 = mrsim.mrsim_launch_count(ctx.h)
    barrier()
    with Clocks(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            step(hs_f, hg_f, sig_f)
        e1.record(stream)
        barrier()
    ms_total = e0.elapsed_time(e1)
    launches = mrsim.mrsim_launch_count(ctx.h) - n_launch0
    prof = mrsim.mrsim_profile_get(ctx.h)
    mrsim.mrsim_profile_enable(ctx.h, False)
    clocks = clk.summary()
    fse_s = maxr(ms_total / a.steps / 1e3)
    fse_sig = sig_f.cpu().numpy().view(np.complex128)

    # ---- grouped EPI ----
    for _ in range(a.warmup):
        step(hs_e, hg_e, sig_e)
    barrier()
    e0.record(stream)
    for _ in range(a.steps):
        step(hs_e, hg_e, sig_e)
    e1.record(stream)
    barrier()
    epi_s = maxr(e0.elapsed_time(e1) / a.steps / 1e3)
    epi_sig = sig_e.cpu().numpy().view(np.complex128)
    if a.quick:
        if rank == 0:
            print(json.dumps({"case": a.case, "K": ph.K, "fse_grouped_s": fse_s,
                              "epi_grouped_s": epi_s, "autotune": tuned,
                              "kernels": {k: v for k, v in prof.items()}}))
        ctx.close()
        return

    # ---- end to end through the public API from pinned host buffers ----
    # (measured here, right after the device-timed steps: after the 36 s plain
    # FSE run below, single steps stalled by 10-14 ms now and then, with the
    # same kernels, host work and median step)
    pin = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).pin_memory()
           for k, v in dict(x=ph.x, y=ph.y, z=ph.z, T1=ph.T1, T2=ph.T2, dB0=ph.dB0,
                            M0=ph.M0).items()}
    out_pin = torch.zeros(2 * ns_f, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * 4 for t in pin.values()) + sum(v.nbytes for v in fse.arrays().values())
    d2h = out_pin.numel() * 8

    def e2e_step():
        # the upload is queued without waiting, so the sequence's host work
        # overlaps the transfer (the pinned arrays stay alive throughout)
        p = mrsim.mrsim_phantom(ctx.h, ph.K, *[pin[k] for k in ("x", "y", "z", "T1", "T2", "dB0",
                                                                  "M0")],
                                flags=mrsim.PHANTOM_ASYNC)
        s = ctx.sequence(fse)
        g = mrsim.mrsim_group(ctx.h, p, s)
        mrsim.mrsim_run(ctx.h, p, s, g, mrsim.GROUPED, mrsim.FP32, out_pin, None, 0)
        mrsim.mrsim_free_groups(g)
        ctx.free("seq", s)
        mrsim.mrsim_free_phantom(p)

    # at least 20 steps: one host-side stall (a page fault burst, a collection
    # of Python garbage) then moves the mean by a few percent, not by 20
    e2e_steps = max(a.steps, 20)
    for _ in range(3):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    e0.record(stream)
    t_steps = []
    for _ in range(e2e_steps):
        ts = time.perf_counter()
        e2e_step()  # ends with the run's read-back (synchronous) and the frees
        t_steps.append((time.perf_counter() - ts) * 1e3)
    e1.record(stream)
    barrier()
    e2e_s = maxr(max(e0.elapsed_time(e1) / 1e3, time.perf_counter() - t0) / e2e_steps)
    # where one end-to-end step goes (host clock, synchronised after each call,
    # so the overlap of the upload with the sequence's host work is not in it)
    split = {}

    def lap(name, fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        split[name] = round((time.perf_counter() - t) * 1e3, 2)
        return r

    p_ = lap("phantom_upload", lambda: mrsim.mrsim_phantom(
        ctx.h, ph.K, *[pin[k] for k in ("x", "y", "z", "T1", "T2", "dB0", "M0")],
        flags=mrsim.PHANTOM_ASYNC))
    s_ = lap("sequence", lambda: ctx.sequence(fse))
    g_ = lap("group", lambda: mrsim.mrsim_group(ctx.h, p_, s_))
    lap("run_and_readback", lambda: mrsim.mrsim_run(ctx.h, p_, s_, g_, mrsim.GROUPED, mrsim.FP32,
                                                    out_pin, None, 0))
    lap("free", lambda: (mrsim.mrsim_free_groups(g_), ctx.free("seq", s_),
                         mrsim.mrsim_free_phantom(p_)))

    # ---- plain forms on the same GPU ----
    def timed_once(fn, prof_out=None):
        if prof_out is not None:
            mrsim.mrsim_profile_reset(ctx.h)
            mrsim.mrsim_profile_enable(ctx.h, True)
        barrier()
        e0.record(stream)
        fn()
        e1.record(stream)
        barrier()
        if prof_out is not None:
            prof_out.update(mrsim.mrsim_profile_get(ctx.h))
            mrsim.mrsim_profile_enable(ctx.h, False)
        return maxr(e0.elapsed_time(e1) / 1e3)

    # plain kernels: tuned on the plain EPI run (the FSE run uses the same kernels)
    fused_ni = mrsim.mrsim_get_tuning(ctx.h, mrsim.TUNE_FUSED_NI)
    tuned_plain = mrsim.mrsim_autotune(ctx.h, hp, hs_e, None, mrsim.PLAIN, mrsim.FP32, 1)
    mrsim.mrsim_set_tuning(ctx.h, mrsim.TUNE_FUSED_NI, fused_ni)
    tuned.update({k: v for k, v in tuned_plain.items() if k != mrsim.TUNE_FUSED_NI})
    step(hs_e, None, sig_e, mrsim.PLAIN)  # warm the plain kernels
    prof_epi_plain, prof_fse_plain = {}, {}
    epi_plain_s = timed_once(lambda: step(hs_e, None, sig_e, mrsim.PLAIN), prof_epi_plain)
    epi_plain_sig = sig_e.cpu().numpy().view(np.complex128).copy()
    fse_plain_s = fse_plain_sig = None
    fse_cache_s = None
    if a.plain_fse == "on":
        fse_cache_s = timed_once(lambda: step(hs_f, None, sig_f, mrsim.PLAIN_CACHE))
        fse_plain_s = timed_once(lambda: step(hs_f, None, sig_f, mrsim.PLAIN), prof_fse_plain)
        fse_plain_sig = sig_f.cpu().numpy().view(np.complex128).copy()

    # ---- reproducible sums (fixed-point block and signal sums): cost and
    # bit-identical repeats, beside two repeats of the default path ----
    def two_runs():
        step(hs_f, hg_f, sig_f)
        first = sig_f.cpu().numpy().copy()
        step(hs_f, hg_f, sig_f)
        return first, sig_f.cpu().numpy().copy()

    d1, d2 = two_runs()
    mrsim.mrsim_set_reproducible(ctx.h, True)
    try:
        r1, r2 = two_runs()
        repro_s = timed_once(lambda: [step(hs_f, hg_f, sig_f) for _ in range(a.steps)]) / a.steps
    finally:
        mrsim.mrsim_set_reproducible(ctx.h, False)
    rv, dv = r1.view(np.complex128), d1.view(np.complex128)
    reproducible = {
        "fse_grouped_ms": round(repro_s * 1e3, 3),
        "default_fse_grouped_ms": round(fse_s * 1e3, 3),
        "cost_vs_default": round(repro_s / fse_s, 3),
        "repeat_bit_identical": bool(np.array_equal(r1, r2)),
        "default_repeat_bit_identical": bool(np.array_equal(d1, d2)),
        "default_repeat_max_abs_diff": float(np.max(np.abs(d1 - d2))),
        "rel_l2_vs_default": float(np.linalg.norm(rv - dv) / np.linalg.norm(dv)),
    }

    # ---- batched workload: 64 uneven jobs in one graph launch ----
    batch = batch_workload(ctx, mrsim, torch, a.steps, a.warmup)
    try:
        batch_mixed = batch_workload(ctx, mrsim, torch, a.steps, a.warmup, mixed=True)
    except Exception as e:  # reported in the line; the main metric stands on its own
        batch_mixed = {"error": f"{type(e).__name__}: {e}"}
    # ---- learned with-RF transitions ----
    surrogate = surrogate_workload(ctx, mrsim, torch)
    # ---- image reconstruction of the simulated k-space ----
    recon = recon_workload(ctx, mrsim, torch, (("fse", fse, fse_sig), ("epi", epi, epi_sig)),
                           a.steps)
    # ---- receive coils (Eq. 6 with P coils) ----
    multicoil = multicoil_workload(ctx, mrsim, torch, ph, fse, hp, hg_f, a.steps)
    # ---- two-axis gradient types: radial readouts ----
    try:
        radial = radial_workload(ctx, mrsim, torch, hp, ph.K, a.steps)
    except Exception as e:  # reported in the line; the main metric stands on its own
        radial = {"error": f"{type(e).__name__}: {e}"}
    # ---- group-reducing preprocessing (clustering) of a mapped phantom ----
    try:
        clustering = cluster_workload(ctx, mrsim, torch, (("fse", fse), ("epi", epi)))
    except Exception as e:  # reported in the line; the main metric stands on its own
        clustering = {"error": f"{type(e).__name__}: {e}"}

    # ---- roofline of the dominant kernel (fused isochromat pass) ----
    name = max(prof, key=lambda n: prof[n][1])
    n_l, ms_l = prof[name]
    avg_s = ms_l / n_l / 1e3
    roof = None
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = pk.get("sm_max_mhz", 2070.0)
    alu_peak = 2 * 128 * n_sm * mhz * 1e6 / 1e12
    if name.startswith("fused_cell"):
        ev_rf, ev_rf_q, ev_adc, ev_adc_q = cell_event_work(fse, mrsim, hs_f)
        per_iso = ((ev_rf - ev_rf_q) * FLOPS_CELL_RF + ev_rf_q * FLOPS_CELL_RF_Q +
                   (ev_adc - ev_adc_q) * FLOPS_CELL_ADC + ev_adc_q * FLOPS_CELL_ADC_Q)
        inst = ((ev_rf - ev_rf_q) * INST_CELL_RF + ev_rf_q * INST_CELL_RF_Q +
                (ev_adc - ev_adc_q) * INST_CELL_ADC + ev_adc_q * INST_CELL_ADC_Q)
        flops = ph.K * per_iso
        ach = flops / avg_s / 1e12
        # issue bound: every SM sub-partition issues one warp instruction per cycle
        t_issue = ph.K * inst / 32 / (n_sm * 4 * mhz * 1e6)
        roof = {"kernel": name, "bound": "alu", "achieved": round(ach, 3),
                "peak": round(alu_peak, 2), "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4),
                "traffic": fused_traffic(ph.K, "fused_cell"),
                "peak_source": f"{n_sm} SMs (device) x 128 FP32 lanes x 2 x sm_max_mhz "
                               f"{mhz:.0f} from MEASURED_PEAKS.json ({pk_kind})",
                "algorithmic_flops_per_launch": flops, "avg_launch_ms": round(avg_s * 1e3, 4),
                "launches": n_l,
                "issue": {"min_thread_inst_per_launch": ph.K * inst,
                          "events": {"rf_end": ev_rf, "rf_end_free_phase": ev_rf_q,
                                     "adc": ev_adc, "adc_free_phase": ev_adc_q},
                          "t_min_ms": round(t_issue * 1e3, 4),
                          "frac": round(t_issue / avg_s, 4),
                          "peak": f"{n_sm} SMs x 4 warp instructions per cycle at {mhz:.0f} MHz"},
                "algorithmic_bytes_per_isochromat": 21}

    # ---- achieved fraction of roofline of the other kernels ----
    bf16_peak = pk.get("bf16_tflops", 1900.0)
    kroof = {}
    f_steps, f_segs, f_distinct = rf_runs(fse)
    gz_f = mrsim.mrsim_group_info(hg_f, mrsim.G_Z)[0]
    if "precompute_f32" in prof:
        n_l, ms_l = prof["precompute_f32"]
        kroof["precompute_f32"] = roof_entry(
            "k_precompute (FSE)", FLOPS_PREP * gz_f * f_distinct, ms_l / a.steps, alu_peak, "alu",
            f"{FLOPS_PREP} flops x {gz_f} Gz groups x {f_distinct} sub-steps of the distinct pulses")
    if "group_signal_f32" in prof:
        n_l, ms_l = prof["group_signal_f32"]
        gx_f = mrsim.mrsim_group_info(hg_f, mrsim.G_X)[0]
        kroof["group_signal_f32"] = roof_entry(
            "k_group_signal (FSE)", FLOPS_GSIG * ns_f * gx_f, ms_l / a.steps, alu_peak, "alu",
            f"{FLOPS_GSIG} flops x {ns_f} samples x {gx_f} Gx groups")
    for nm, pr, seq_, ns_ in (("fse", prof_fse_plain, fse, ns_f), ("epi", prof_epi_plain, epi, ns_e)):
        steps_, segs_, _ = rf_runs(seq_)
        if "plain_rf_f32" in pr:
            kroof[f"plain_rf_{nm}"] = roof_entry(
                f"k_plain_rf ({nm.upper()})",
                ph.K * (FLOPS_PLAIN_STEP * steps_ + FLOPS_PLAIN_SEG * segs_), pr["plain_rf_f32"][1],
                alu_peak, "alu", f"K x ({FLOPS_PLAIN_STEP} x {steps_} sub-steps + "
                                 f"{FLOPS_PLAIN_SEG} x {segs_} segments)")
        if "plain_adc_f32" in pr:
            kroof[f"plain_adc_{nm}"] = roof_entry(
                f"k_plain_adc ({nm.upper()})", ph.K * FLOPS_PLAIN_SAMPLE * ns_,
                pr["plain_adc_f32"][1], alu_peak, "alu",
                f"K x {FLOPS_PLAIN_SAMPLE} x {ns_} samples")
    if surrogate.get("sur_infer_ms"):
        kroof["sur_infer"] = roof_entry(
            "k_sur_infer (27.5M surrogate FSE)", FLOPS_SUR_INFER * surrogate["groups_served_per_run"],
            surrogate["sur_infer_ms"], bf16_peak, "tensor",
            f"{FLOPS_SUR_INFER} tensor flops x {surrogate['groups_served_per_run']} served "
            "(group, pulse) pairs per run (peak: measured cuBLAS bf16 burst)")

    ck = clustering.get("kernels", {})
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    for kname, bpi, note in (("cluster_apply", 28, "key id 4 + M0 4 read, T1, T2, dB0, M0 16 "
                                                    "+ label 4 written"),
                             ("cluster_quantize", 24, "T1, T2, dB0 12 read, 3 features 12 "
                                                      "written")):
        if kname in ck:
            n_l, ms_l = ck[kname]
            kroof[kname] = roof_entry_hbm(f"k_cl_{kname.split('_')[1]} (27.5M mapped phantom)",
                                          bpi * clustering["K"], ms_l / n_l, hbm_peak,
                                          f"{bpi} B per isochromat ({note}) x K")

    # ---- parity against the stored oracle signals ----
    pd, sd_f, sd_e = phantom_digest(ph), sequence_digest(fse), sequence_digest(epi)
    parity = {"fse_grouped_rel_l2": golden_check("fse", fse_sig, pd, sd_f),
              "epi_grouped_rel_l2": golden_check("epi", epi_sig, pd, sd_e),
              "epi_plain_rel_l2": golden_check("epi", epi_plain_sig, pd, sd_e)}
    if fse_plain_sig is not None:
        parity["fse_plain_rel_l2"] = golden_check("fse", fse_plain_sig, pd, sd_f)

    cpu = cpu_epi = None
    if rank == 0 and world == 1:
        v, wall, n, cores = cpu_baseline(ph, fse, a.cpu_stride)
        cpu = {"value": round(v, 2), "unit": "s", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle on every {a.cpu_stride}th isochromat ({n} of {ph.K}) of "
                         f"the FSE workload, {wall:.2f} s wall, extrapolated x{ph.K / n:.1f} "
                         "(linear in K)"}
        stride_e = 8 * a.cpu_stride
        v, wall, n, cores = cpu_baseline(ph, epi, stride_e)
        cpu_epi = {"value": round(v, 2), "unit": "s", "cores": cores, "kind": "oracle",
                   "sample": f"FP64 oracle on every {stride_e}th isochromat ({n} of {ph.K}) of "
                             f"the EPI workload, {wall:.2f} s wall, extrapolated "
                             f"x{ph.K / n:.1f} (linear in K)",
                   "gpu_grouped_s": round(epi_s, 6)}

    steps_fse = ph.K * (sum(int(r) for r, b1, b2 in zip(fse.repeat, fse.b1re, fse.b1im)
                            if b1 != 0 or b2 != 0) + ns_f)
    out = {
        "metric": METRIC, "value": round(fse_s, 6), "unit": "s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(fse_s * 1e3, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "K": ph.K, "mode": "grouped", "precision": "fp32",
                   "l2": "inputs larger than L2 (27.5M isochromats x 40 B resident)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "fse_grouped_s": round(fse_s, 6), "epi_grouped_s": round(epi_s, 6),
        "fse_plain_s": None if fse_plain_s is None else round(fse_plain_s, 4),
        "fse_plain_cache_s": None if fse_cache_s is None else round(fse_cache_s, 4),
        "epi_plain_s": round(epi_plain_s, 5),
        "speedup_grouped_vs_plain": {
            "fse": None if fse_plain_s is None else round(fse_plain_s / fse_s, 1),
            "epi": round(epi_plain_s / epi_s, 1)},
        "isochromat_steps_per_s_equiv": round(steps_fse / fse_s, 1),
        "prep_s": round(prep_s, 4), "phantom_upload_s": round(t_upload, 4), "groups": groups,
        "autotune": {"cell_isochromats_per_thread": tuned[mrsim.TUNE_CELL_NI],
                     "cell_rows": {0: "auto", 1: "table", 2: "per thread"}[
                         tuned[mrsim.TUNE_CELL_ROWS]],
                     "fused_isochromats_per_thread": tuned[mrsim.TUNE_FUSED_NI],
                     "plain_rf_isochromats_per_thread": tuned[mrsim.TUNE_PLAIN_RF_NI],
                     "plain_adc_ctas_per_sm": tuned[mrsim.TUNE_ADC_CTAS_PER_SM],
                     "precompute_lanes": tuned[mrsim.TUNE_PRECOMP_LANES],
                     "precompute_fp32_block_steps": tuned[mrsim.TUNE_PRECOMP_STEPS],
                     "seconds": round(autotune_s, 2)},
        "parity": parity,
        "batch64": batch,
        "batch_mixed": batch_mixed,
        "surrogate": surrogate,
        "multicoil": multicoil,
        "reproducible": reproducible,
        "recon": recon,
        "radial": radial,
        "clustering": clustering,
        "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()},
        "roofline": roof, "kernel_roofline": kroof, "cpu_baseline": cpu,
        "cpu_baseline_epi": cpu_epi,
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "steps": e2e_steps,
                "step_ms": {"min": round(min(t_steps), 2),
                            "median": round(statistics.median(t_steps), 2),
                            "max": round(max(t_steps), 2)},
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "split_ms": split},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def profile_kernels(a, configs):
    """Small runs of the kernels other than the fused one, each launched a few
    times, for ncu captures: the plain step and ADC kernels (plain EPI on the
    256x256x105 phantom), the preparation and group-signal kernels (grouped FSE
    on it), and the surrogate gate and inference (a briefly trained network on
    the 2 ms-pulse FSE, run on a 256x256x105 phantom with per-isochromat dB0 and
    b1).  Prints the per-kernel CUDA-event times of one run of each."""
    import torch
    from paper_2508_03960_gb300 import mrsim
    from mrsim_inputs.phantom import continuous_phantom
    torch.cuda.set_device(0)
    ctx = mrsim.Context(0, torch.cuda.current_stream().cuda_stream)
    out = {}

    def runs(hp, hs, hg, mode, ns, name, n=3):
        sig = torch.zeros(2 * ns, dtype=torch.float64, device="cuda")
        for i in range(n):
            last = i == n - 1
            if last:
                mrsim.mrsim_profile_reset(ctx.h)
                mrsim.mrsim_profile_enable(ctx.h, True)
            mrsim.mrsim_run(ctx.h, hp, hs, hg, mode, mrsim.FP32, sig, None, mrsim.OUT_DEVICE)
            torch.cuda.synchronize()
        out[name] = {k: [v[0], round(v[1], 4)] for k, v in mrsim.mrsim_profile_get(ctx.h).items()
                     if v[0]}
        mrsim.mrsim_profile_enable(ctx.h, False)

    ph = configs.small_phantom(256, 256, 105)
    hp = ctx.phantom(ph)
    epi, fse = configs.epi_sequence(), configs.fse_sequence()
    hs_e, hs_f = ctx.sequence(epi), ctx.sequence(fse)
    runs(hp, hs_e, None, mrsim.PLAIN, epi.n_samples, "plain_epi")
    runs(hp, hs_f, ctx.group(hp, hs_f), mrsim.GROUPED, fse.n_samples, "grouped_fse")
    _, seq = configs.surrogate_fse()
    hs = ctx.sequence(seq)
    sur = mrsim.mrsim_surrogate_train(ctx.h, hs, SUR_LO, SUR_HI, n_train=1 << 18, epochs=10,
                                      batch=8192, lr=1e-2, seed=1005, bound=1e-3)
    cph = continuous_phantom(256, 256, 105, 8, seed=1005)
    hp2 = ctx.phantom(cph)
    hg2 = ctx.group(hp2, hs)
    mrsim.mrsim_surrogate_use(ctx.h, sur)
    runs(hp2, hs, hg2, mrsim.SURROGATE, seq.n_samples, "surrogate_fse")
    mrsim.mrsim_surrogate_use(ctx.h, None)
    mrsim.mrsim_free_surrogate(sur)
    ctx.close()
    print(json.dumps({"profile_kernels": out, "K": ph.K}))


def profile_cluster(a, configs):
    """The clustering preprocessing of the 27.5M-isochromat parameter-mapping
    phantom into 256 clusters, twice; prints the wall time and the per-kernel
    CUDA-event times of the second call."""
    import torch
    from paper_2508_03960_gb300 import mrsim
    torch.cuda.set_device(0)
    ph = configs.mapped_27m()
    ctx = mrsim.Context(0, torch.cuda.current_stream().cuda_stream)
    hp = ctx.phantom(ph)
    ctx.cluster(hp, ph.K, 256, want_labels=False)
    torch.cuda.synchronize()
    mrsim.mrsim_profile_reset(ctx.h)
    mrsim.mrsim_profile_enable(ctx.h, True)
    t = time.perf_counter()
    _, n, _, _ = ctx.cluster(hp, ph.K, 256, want_labels=False)
    wall_prof = time.perf_counter() - t
    prof = {k: [int(v[0]), round(v[1], 4)] for k, v in mrsim.mrsim_profile_get(ctx.h).items()
            if v[0]}
    mrsim.mrsim_profile_enable(ctx.h, False)
    # the wall time without the per-launch events of the profile
    torch.cuda.synchronize()
    t = time.perf_counter()
    ctx.cluster(hp, ph.K, 256, want_labels=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    ctx.close()
    print(json.dumps({"profile_cluster": prof, "wall_s": round(wall, 4),
                      "wall_profiled_s": round(wall_prof, 4), "n_clusters": n, "K": ph.K}))


def reference_arm(a, configs):
    """The FP64 CPU oracle as it stands, on this host's cores, on a bounded
    sample of the FSE workload each step; value extrapolated to K."""
    ph = configs.full_phantom()
    fse = configs.fse_sequence()
    stride = 1024
    vals = []
    walls = []
    for i in range(a.warmup + a.steps):
        v, wall, n, cores = cpu_baseline(ph, fse, stride)
        if i >= a.warmup:
            vals.append(v)
            walls.append(wall)
    value = statistics.mean(vals)
    sample = (f"FP64 oracle on every {stride}th isochromat ({n} of {ph.K}) per step, "
              f"extrapolated x{ph.K / n:.1f} (linear in K)")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "s",
           "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": round(statistics.mean(walls) * 1e3, 2), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "K": ph.K, "mode": "oracle (ungrouped, FP64)"},
           "cpu_baseline": {"value": round(value, 3), "unit": "s", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 3), "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
