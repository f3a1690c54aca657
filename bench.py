"""Throughput of the embedded H psi hot path on one GB300 (or N replicas under torchrun).

Workloads (seeded synthetic inputs, paper_1406_7803_gb300.workloads):
  molecule-on-slab (default): 16 x 16 x 40 bohr, 72 x 72 x 180 grid, 20 Ha; a 36-atom Z=3
    slab with 64 bands x 4 k-points (Fermi smearing) plus a 6-atom Z=4 molecule with 12 bands
    at Gamma, PBE + revAPBEK, 2 Gaussian KB projectors per atom: 268 band-applies per step.
  batched (--workload batched): 24^3 bohr, 96^3 grid, 20 Ha; a 54-atom slab with 96 bands x
    2 k-points plus 16 molecules of 8..64 bands at Gamma: 778 band-applies per step.
  large (--workload large): 30 x 30 x 60 bohr, 144 x 144 x 288 grid, 25 Ha; a 216-atom slab
    with 512 bands x 8 k-points plus 32 molecules of 16..48 bands: 5209 band-applies per step.
  plain (--workload plain): 10^3 bohr, 32^3 grid, 15 Ha; two 3-atom subsystems with 4 bands
    each, LDA + Thomas-Fermi: 8 band-applies per step.

One step = one pass of the hot path over the whole cell: the embedding-potential build
(rho = sum rho_I, FFT Poisson, FFT gradients, pointwise xc and GGA kinetic potentials,
divergence, assembly of V_eff^I) followed by H_I psi for every band of every (subsystem,
k-point).  value = band-applies per second over all ranks.

Also in the JSON line: a per-kernel table (CUDA events around every launch of a profiled
pass of the same step, algorithmic bytes or flops per launch and the roof each is held
to), the FP64 path's band-applies/s on the same cell, the step replayed from a CUDA
graph, and (N = 1, skipped with --no-ft) seconds per freeze-and-thaw cycle at 1e-6 Ha on
the molecule-on-slab cell: mixed precision with and without the learned preconditioner,
against the plain FP64 GPU path ("ft_cycle").

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
                       [--workload molecule-on-slab|batched|large|plain] [--impl ours|reference]
                       [--no-cpu] [--no-fp64] [--no-ft]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1406_7803_gb300 import workloads  # noqa: E402

METRIC = "Embedded H·ψ band-applies/s"
UNIT = "band-applies/s"
WORKLOADS = {"molecule-on-slab": workloads.molecule_on_slab, "batched": workloads.batched_uneven,
             "large": workloads.large_cell, "plain": workloads.plain_fde_32}
REFERENCE_BUDGET_S = 150.0  # wall time the reference arm's K + W steps should stay within


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"fde_bench_clocks_gpu{index}_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except OSError:
            return out
        rows = [[x.strip() for x in r] for r in rows if len(r) >= 9]
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        out["sm_mhz"] = float(np.median(sm)) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(n)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def kernel_source_digest(files, function=None):
    """SHA-256 (16 hex digits) of the sources a kernel is built from: whole files, plus, for
    (file, name), the text of the __global__ function `name` in that file."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    if function:
        f, name = function
        text = open(os.path.join(ROOT, f)).read()
        a = text.index(name + "(")
        a = text.rindex("template", 0, a)
        b = text.index("\n}\n", a) + 3
        h.update(name.encode() + b"\0" + text[a:b].encode())
    return h.hexdigest()[:16]


def _profile_traffic(name, files, function=None):
    """DRAM bytes per launch of a kernel from its committed ncu summary (profiles/<name>.md),
    or None when the kernel's sources have changed since the counters were taken."""
    try:
        text = open(os.path.join(ROOT, "profiles", name + ".md")).read()
    except OSError:
        return None
    fields = dict(l.split(":", 1) for l in text.splitlines()
                  if l.startswith(("traffic_bytes_per_launch:", "source_sha256:")))
    if fields.get("source_sha256", "").split()[0:1] != [kernel_source_digest(files, function)]:
        return None
    return float(fields["traffic_bytes_per_launch"])


# the plane pass: its own function text in hpsi_ct.cuh plus the staged-transform core
PLANE_SOURCES = ["paper_1406_7803_gb300/csrc/fftct.cuh", "paper_1406_7803_gb300/csrc/fft.cuh",
                 "paper_1406_7803_gb300/csrc/common.cuh"]
PLANE_FUNCTION = ("paper_1406_7803_gb300/csrc/hpsi_ct.cuh", "k_plane_ct")


def max_over_ranks(x, ws, device):
    """The largest value of x over the ranks of the process group (x itself for one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job(total_ms_local, steps, units, ws, device):
    """(ms per step, whole-job units/s): the slowest rank's time, every rank's units."""
    ms = max_over_ranks(total_ms_local, ws, device) / steps
    return ms, ws * units / (ms / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- the oracle's step (reference arm and cpu_baseline) --------------------------------------
class OracleStep:
    """One pass of the hot path by the FP64 oracle: one V_eff build for every subsystem, then
    H psi of a band block of each (subsystem, k), each block in one batched oracle call.
    The orbitals are drawn once, outside the timed region."""

    def __init__(self, wl, bands=None):
        from oracle import fde as ofde
        self.sy = ofde.System(wl)
        self.rhos = np.array([workloads.initial_density(wl, I) for I in range(wl.nsub)])
        self.blocks = []
        for I, s in enumerate(wl.subsystems):
            for k in range(s.nk):
                nb = s.nbands if bands is None else min(s.nbands, bands)
                npw = self.sy.basis[I][k][0].shape[0]
                self.blocks.append((I, k, workloads.raw_orbitals(5, I, k, nb, npw)))
        self.units = sum(c.shape[0] for _, _, c in self.blocks)

    def __call__(self):
        t0 = time.perf_counter()
        pot = self.sy.build_veff(self.rhos)
        self.veff_s = time.perf_counter() - t0
        for I, k, c in self.blocks:
            self.sy.apply_h(I, k, c, pot["veff"][I])
        return time.perf_counter() - t0


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(wl, bands=None):
    """The FP64 oracle timed on this host's cores on one step of the workload (the same batched
    oracle call the reference arm times): every band, or `bands` per (subsystem, k)."""
    t0 = time.perf_counter()
    st = OracleStep(wl, bands=bands)
    setup = time.perf_counter() - t0
    sec = st()
    cores = _cores()
    what = "one full step" if bands is None else f"one step with {bands} band(s) per (subsystem, k)"
    return {"value": st.units / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}: FP64 v_eff build of {wl.nsub} subsystems + {st.units} band-applies "
                      f"in one oracle call per (subsystem, k) ({sec:.2f} s; scipy.fft workers={cores}); "
                      f"oracle setup {setup:.1f} s excluded"}


def run_reference(args):
    """The reference arm: the FP64 oracle (the slow, obviously correct CPU statement of the
    method) timed step by step on the host cores, on the same workload and metric.  A step is
    the whole hot path over the cell when K + W such steps fit the time budget, else the
    potential build plus an equal band sample of every (subsystem, k)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]()
    # a one-band-per-block step sizes the sample (untimed, counts as no warm-up): the whole
    # hot path when K + W such steps fit the budget, else the largest equal band sample
    probe = OracleStep(wl, bands=1)
    t_probe = probe()
    per_band = max((t_probe - probe.veff_s) / max(probe.units, 1), 1e-5)
    n = max(1, args.steps + args.warmup)
    nblocks = len(probe.blocks)
    full_est = probe.veff_s + per_band * wl.band_k_pairs()
    if n * full_est <= REFERENCE_BUDGET_S:
        step = OracleStep(wl)
    else:
        spare = REFERENCE_BUDGET_S / n - probe.veff_s
        bands = max(1, int(spare / (per_band * nblocks))) if spare > 0 else 1
        step = OracleStep(wl, bands=bands) if bands > 1 else probe
    for _ in range(args.warmup):
        step()
    wall0 = time.perf_counter()
    times = [step() for _ in range(args.steps)]
    wall = time.perf_counter() - wall0
    ms = 1e3 * float(np.mean(times))
    val = step.units / (ms / 1e3)
    cores = _cores()
    sample = ("each step the whole hot path: v_eff build + every band" if step.units == wl.band_k_pairs() else
              f"each step: v_eff build + a {step.units}-band sample ({len(step.blocks)} (subsystem, k) blocks)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "band_applies_per_step": step.units, "seed": wl.seed},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))
    return 0


# ---- per-kernel roofline table ------------------------------------------------------------
def _sm_count():
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp_peaks(peaks):
    """Nominal CUDA-core rates from this device's SM count and the measured maximum SM clock:
    FP32 128 lanes and FP64 2 lanes per SM, a fused multiply-add counted as 2 flops."""
    sms = _sm_count()
    clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
    return {"sms": sms, "fp32_tflops": sms * 128 * 2 * clk / 1e12, "fp64_tflops": sms * 2 * 2 * clk / 1e12,
            "tf32_tflops": peaks.get("bf16_tflops", 1900.0) / 2.0}


def step_work(wl, ctx, prec):
    """Algorithmic work of one hot step per kernel family, summed over the step's launches:
    bytes that must cross HBM (compulsory: every operand read once, every result written once)
    and flops (5 N log2 N per transformed line of length N, 8 real flops per complex MAC)."""
    n1, n2, n3 = wl.grid
    nr = n1 * n2 * n3
    cw = 8 if prec == "mixed" else 16  # bytes per complex value of the working precision
    rw = cw // 2
    w = {k: {"bytes": 0.0, "flops": 0.0} for k in ("k_zinv", "k_plane", "k_zfwd", "k_gemm_hn", "k_gemm_rot",
                                                  "k_kb_couple", "k_fft_axis_f64", "k_fft_axis_dd", "k_fft_axis_f32",
                                                  "k_pw_total", "k_pw_pair", "k_unpack_density", "k_assemble_pair")}
    for I, s in enumerate(wl.subsystems):
        for k in range(s.nk):
            mil = ctx.basis(I, k)
            npw = mil.shape[0]
            ncol = len({(a, b) for a, b in mil[:, :2].tolist()})
            nrow = len(np.unique(mil[:, 0]))
            nb = s.nbands
            w["k_zinv"]["bytes"] += nb * (npw + n3 * ncol) * cw
            w["k_zinv"]["flops"] += nb * ncol * 5 * n3 * math.log2(n3)
            w["k_plane"]["bytes"] += nb * 2 * n3 * ncol * cw
            w["k_plane"]["flops"] += nb * n3 * (2 * (nrow * 5 * n2 * math.log2(n2) + n2 * 5 * n1 * math.log2(n1))
                                                + 2 * n1 * n2)
            w["k_zfwd"]["bytes"] += nb * (n3 * ncol + 2 * npw) * cw
            w["k_zfwd"]["flops"] += nb * ncol * 5 * n3 * math.log2(n3)
            npj = len(s.proj_sigma) * s.natoms
            if npj:
                w["k_gemm_hn"]["bytes"] += (npj + nb) * npw * cw
                w["k_gemm_hn"]["flops"] += 8.0 * npj * nb * npw
                w["k_gemm_rot"]["bytes"] += (npj + 2 * nb) * npw * cw
                w["k_gemm_rot"]["flops"] += 8.0 * npj * nb * npw
        w["k_plane"]["bytes"] += nr * rw  # each subsystem's potential planes once
    # the potential build: 8 complex 3D transforms per pair of subsystems (GGA), each 3 axis
    # passes reading and writing the grid once.  FP64 contexts: all in FP64.  Mixed: the density
    # and its 3 gradient transforms in double-float (16 bytes a value, one profiled scope per 3D
    # transform), the 3 divergence and the potential transforms in FP32.
    npairs = (wl.nsub + 1) // 2
    per_tr = 5 * nr * math.log2(nr)
    if prec == "mixed":
        w["k_fft_axis_dd"]["bytes"] = 4 * npairs * 3 * 2 * nr * 16
        w["k_fft_axis_dd"]["flops"] = 4 * npairs * per_tr
        w["k_fft_axis_f32"]["bytes"] = 4 * npairs * 3 * 2 * nr * 8
        w["k_fft_axis_f32"]["flops"] = 4 * npairs * per_tr
    else:
        w["k_fft_axis_f64"]["bytes"] = 8 * npairs * 3 * 2 * nr * 16
        w["k_fft_axis_f64"]["flops"] = 8 * npairs * per_tr
    # the G-space and pointwise passes of a GGA build, per grid point (FP64 grids 8 bytes a
    # value, packed complex grids 16; the divergence arguments in the working precision):
    #   k_unpack_density  C in, rho_tot(G) out, three packed gradient grids out (+ rho_tot in
    #                     for every pair after the first);
    #   k_pw_total        rho_tot and every pair's three packed gradients in, v and h_x,y,z out;
    #   k_pw_pair         both densities, three packed gradients, h_x,y,z and v in; both w and
    #                     three packed divergence arguments out;
    #   k_assemble_pair   rho_tot(G) and the three divergence grids in, F out.
    td = 8 if prec == "mixed" else 16
    w["k_unpack_density"]["bytes"] = nr * (npairs * (16 + 16 + 48) + (npairs - 1) * 16)
    w["k_pw_total"]["bytes"] = nr * (8 + npairs * 48 + 32)
    w["k_pw_pair"]["bytes"] = nr * npairs * (16 + 48 + 24 + 8 + 16 + 3 * td)
    w["k_assemble_pair"]["bytes"] = nr * npairs * (16 + 3 * td + td)
    return w


def kernel_table(wl, ctx, prec, peaks, src, nsteps=5):
    """Per-kernel device time of a profiled pass (CUDA events around every launch on the
    context stream) and each kernel's achieved fraction of the roof that bounds it."""
    import torch
    fp = fp_peaks(peaks)
    hbm = peaks.get("hbm_gbs", 6800.0)
    names = ["k_zinv", "k_plane", "k_zfwd", "k_fft_axis_f64", "k_fft_axis_dd", "k_fft_axis_f32", "k_pw_total",
             "k_pw_pair", "k_unpack_density",
             "k_assemble_pair", "k_finish_pair", "k_pack2", "k_combine", "k_nonfinite", "k_gemm_hn_tc",
             "k_gemm_hn_partial", "k_gemm_hn_reduce", "k_gemm_rot", "k_gemm_rot_tc", "k_kb_couple"]
    ctx.sync()
    ctx.profile_enable(2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ev0.record(stream)
    for _ in range(nsteps):
        ctx.hot_step(False)
    ev1.record(stream)
    torch.cuda.synchronize()
    step_ms = ev0.elapsed_time(ev1) / nsteps
    got = {n: ctx.profile_get(n) for n in names}
    ctx.profile_enable(0)
    work = step_work(wl, ctx, prec)
    rows = []
    for n in names:
        cnt, ms = got[n]
        if not cnt:
            continue
        per_step_ms = ms / nsteps
        row = {"kernel": n, "launches_per_step": cnt / nsteps, "avg_us": 1e3 * ms / cnt,
               "share": per_step_ms / step_ms}
        fam = "k_gemm_hn" if n in ("k_gemm_hn_tc", "k_gemm_hn_partial") else n
        fam = "k_gemm_rot" if n in ("k_gemm_rot", "k_gemm_rot_tc") else fam
        wk = work.get(fam)
        if wk and (wk["bytes"] or wk["flops"]):
            sec = per_step_ms / 1e3
            gbs = wk["bytes"] / sec / 1e9
            row["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                          "algorithmic_bytes_per_launch": wk["bytes"] / (cnt / nsteps)}
            if n == "k_fft_axis_f64":
                tf = wk["flops"] / sec / 1e12
                row["fp64"] = {"achieved_tflops": tf, "peak_tflops": fp["fp64_tflops"], "frac": tf / fp["fp64_tflops"]}
            elif n == "k_fft_axis_dd":
                # transform flops at ~48-bit precision, against the FP64 roof they replace
                tf = wk["flops"] / sec / 1e12
                row["fp64_equivalent"] = {"achieved_tflops": tf, "peak_tflops": fp["fp64_tflops"],
                                          "frac": tf / fp["fp64_tflops"],
                                          "note": "double-float on the FP32 pipes; > 1 means above the FP64 roof"}
            elif n in ("k_gemm_hn_tc",):
                tf = wk["flops"] / sec / 1e12
                row["tensor_tf32"] = {"achieved_tflops": tf, "peak_tflops": fp["tf32_tflops"],
                                      "frac": tf / fp["tf32_tflops"]}
            elif wk["flops"]:
                pk = fp["fp32_tflops"] if prec == "mixed" else fp["fp64_tflops"]
                tf = wk["flops"] / sec / 1e12
                row["fp32" if prec == "mixed" else "fp64"] = {"achieved_tflops": tf, "peak_tflops": pk,
                                                               "frac": tf / pk}
        rows.append(row)
    rows.sort(key=lambda r: -r["share"])
    return {"step_ms_profiled": step_ms, "rows": rows,
            "peaks": {"hbm_gbs": hbm, "hbm_source": src, "fp32_tflops": fp["fp32_tflops"],
                      "fp64_tflops": fp["fp64_tflops"], "tf32_tflops": fp["tf32_tflops"], "sms": fp["sms"],
                      "cuda_core_source": "nominal: device SM count x lanes x 2 x measured max SM clock",
                      "tf32_source": f"measured bf16 burst / 2 ({src})"}}


def ft_cycles(tol=1e-6):
    """Seconds per freeze-and-thaw cycle on the molecule-on-slab cell at tol Ha: the mixed path
    (FP32 cycle, FP64 refinement), the plain FP64 GPU path, and the mixed path with the
    learned preconditioner in its FP32 stage (network trained on the GPU on (residual, error)
    pairs recorded over the eigensolves of the 8x8x20 bohr slab + molecule cell).  Every run
    starts from the same seeded orbitals and densities; wall time of the synchronising call."""
    import torch
    from paper_1406_7803_gb300 import fde
    out = {"tol_ha": tol}
    # learned weights from the small cell
    small = workloads.molecule_on_slab_small()
    cs = fde.context_from_workload(small, prec="mixed")
    fde.seed_workload(cs, small)
    cs.build_vemb()
    cs.precond_record(60)
    t0 = time.perf_counter()
    for I, s in enumerate(small.subsystems):
        for k in range(s.nk):
            cs.subspace_solve(I, k, 3e-5, 300, fde.FDE_PRECOND_TPA)  # the FP32 solves' residual floor
    cs.precond_record(0)
    cs.precond_set_weights(fde.precond_initial_weights(0))
    l0, l1 = cs.precond_train(400, 3e-3)
    w, _ = cs.precond_get_weights()
    out["learned_training"] = {"cell": small.name, "steps": 400, "loss_first": l0, "loss_last": l1,
                               "seconds": time.perf_counter() - t0}
    del cs
    wl = workloads.molecule_on_slab()
    for name, prec, learned in (("mixed", "mixed", False), ("fp64", "fp64", False), ("mixed_learned", "mixed", True)):
        ctx = fde.context_from_workload(wl, prec=prec)
        fde.seed_workload(ctx, wl)
        if learned:
            ctx.precond_set_weights(w)
            ctx.set_precond(fde.FDE_PRECOND_LEARNED)
        ctx.sync()
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, e = ctx.freeze_thaw_cycle(tol, 100)
        ctx.sync()
        dt = time.perf_counter() - t
        dav, hb = ctx.stats()
        out[name] = {"seconds": dt, "status": int(st), "F_fde": e["F_fde"], "E_fde": e["E_fde"],
                     "scf_iterations": e.get("iters"), "eigensolver_iterations": dav, "band_applies": hb}
        del ctx
        torch.cuda.empty_cache()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    out["speedup_mixed_learned_vs_fp64"] = out["fp64"]["seconds"] / out["mixed_learned"]["seconds"]
    out["dF_mixed_vs_fp64_ha"] = out["mixed"]["F_fde"] - out["fp64"]["F_fde"]
    out["dF_mixed_learned_vs_fp64_ha"] = out["mixed_learned"]["F_fde"] - out["fp64"]["F_fde"]
    return out


def precond_kernels(ctx, wl, stream):
    """The learned preconditioner's kernels on the first slab k-point's band block (n_b x npw,
    working precision): inference with the bf16 weights (average of 10 calls) and one
    loss-and-gradient evaluation over the same block as training pairs (average of 3), wall
    time of the synchronising calls, on the tensor cores and on the CUDA cores."""
    import torch
    from paper_1406_7803_gb300 import fde
    s = wl.subsystems[0]
    npw = ctx.basis(0, 0).shape[0]
    rng = np.random.default_rng(7)
    rh = (rng.standard_normal((s.nbands, npw)) + 1j * rng.standard_normal((s.nbands, npw))) / np.sqrt(npw)
    dh = rh * 0.5 + 0.1 * (rng.standard_normal((s.nbands, npw)) + 1j * rng.standard_normal((s.nbands, npw))) / np.sqrt(npw)
    tb = np.linspace(0.5, 3.0, s.nbands)
    w0 = fde.precond_initial_weights(0)
    w0[-65:-1] = 0.05 * np.random.default_rng(8).standard_normal(64)  # a nonzero output layer
    ctx.precond_set_weights(w0)
    ctx.precond_add_pairs(0, 0, rh, dh, tb)
    r = torch.from_numpy(rh).to(device="cuda",
                                dtype=torch.complex64 if ctx.prec == fde.FDE_PREC_MIXED else torch.complex128)
    w = torch.zeros_like(r)
    torch.cuda.synchronize()
    out = {"block": f"{s.nbands} bands x {npw} plane waves", "pairs": s.nbands * npw}
    for path, name in ((1, "tensor_cores"), (0, "cuda_cores")):
        fde.set_precond_path(path)
        ctx.precond_apply(0, 0, r, w, s.nbands, tb)
        ctx.precond_loss_grad()
        t0 = time.perf_counter()
        for _ in range(10):
            ctx.precond_apply(0, 0, r, w, s.nbands, tb)
        t_apply = (time.perf_counter() - t0) / 10
        t0 = time.perf_counter()
        for _ in range(3):
            ctx.precond_loss_grad()
        t_grad = (time.perf_counter() - t0) / 3
        out[name] = {"apply_ms": 1e3 * t_apply, "loss_grad_ms": 1e3 * t_grad}
    fde.set_precond_path(1)
    ctx.precond_clear()
    return out


def time_steps(ctx, stream, flush, steps, use_graph=False):
    """Device time (ms) of each of `steps` hot steps, L2 flushed before each."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        ctx.hot_step(use_graph)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1406_7803_gb300 import fde
    wl = WORKLOADS[args.workload]()
    # one non-default stream for the library, the L2 flush and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = fde.context_from_workload(wl, prec=args.prec, stream=stream.cuda_stream)
    fde.seed_workload(ctx, wl)
    ctx.build_vemb()
    ctx.sync()
    units = wl.band_k_pairs()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    for _ in range(max(args.warmup, 3)):
        ctx.hot_step(False)
    ctx.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.profile_enable(1)  # the three H psi passes, timed inside the timed region
    launches0 = ctx.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ctx.hot_step(False)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launches = ctx.launch_count() - launches0
    total_ms = float(np.sum(step_ms))
    prof = {n: ctx.profile_get(n) for n in ("k_zinv", "k_plane", "k_zfwd")}
    ctx.profile_enable(0)
    ms, value = whole_job(total_ms, args.steps, units, ws, "cuda")

    # the same pass replayed from a captured CUDA graph (launch overhead removed)
    ctx.hot_step(True)
    torch.cuda.synchronize()
    graph_ms = float(np.mean(time_steps(ctx, stream, flush, args.steps, use_graph=True)))

    peaks, src = _peaks()
    table = kernel_table(wl, ctx, args.prec, peaks, src) if rank == 0 else None

    large = args.workload == "large"
    # end to end through the C ABI with host buffers in page-locked memory: densities in, H psi
    # out, every copy inside the timed region (not for the large cell: its orbitals and H psi
    # would take ~55 GB of page-locked host memory)
    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t, t.numpy()

    keep = []
    rhos_h = []
    for I in (range(wl.nsub) if not large else []):
        t, a = pinned(workloads.initial_density(wl, I))
        keep.append(t)
        rhos_h.append(a)
    psi_h, h_out, h2d, d2h = [], [], 0, 0
    for I, s in enumerate(wl.subsystems if not large else []):
        for k in range(s.nk):
            npw = ctx.basis(I, k).shape[0]
            t, a = pinned(workloads.raw_orbitals(9, I, k, s.nbands, npw))
            t2, o = pinned(np.zeros((s.nbands, npw), dtype=np.complex128))
            keep += [t, t2]
            psi_h.append((I, k, s.nbands, a))
            h_out.append(o)
    for r in rhos_h:
        h2d += r.nbytes
    for (_, _, _, c), o in zip(psi_h, h_out):
        h2d += c.nbytes
        d2h += o.nbytes

    def e2e_step():
        # densities and every orbital block in, every H psi block out, through the host form
        # of the hot step (orbital uploads overlap the potential build)
        ctx.hot_step_host(rhos_h, [c for (_, _, _, c) in psi_h], h_out)

    e2e_s = None
    if not large:
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ne = max(2, min(args.steps // 2, 20))
        for _ in range(ne):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / ne
        e2e_s = max_over_ranks(e2e_s, ws, "cuda")

    # roofline of the dominant kernel (the fused plane pass of the local H psi), from the
    # events taken inside the timed region
    n_plane, ms_plane = prof["k_plane"]
    roof = None
    if n_plane:
        fp = fp_peaks(peaks)
        work = step_work(wl, ctx, args.prec)["k_plane"]
        per_launch_flops = work["flops"] * args.steps / n_plane
        per_launch_bytes = work["bytes"] * args.steps / n_plane
        sec = ms_plane / n_plane / 1e3
        pk = fp["fp32_tflops"] if args.prec == "mixed" else fp["fp64_tflops"]
        achieved = per_launch_flops / sec / 1e12
        traffic = (_profile_traffic("k_plane_ct_molecule_on_slab", PLANE_SOURCES, PLANE_FUNCTION)
                   if (args.prec == "mixed" and args.workload == "molecule-on-slab") else None)
        hbm_gbs = per_launch_bytes / sec / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                "traffic": traffic, "kernel": "k_plane", "launches": n_plane, "avg_launch_us": 1e6 * sec,
                "algorithmic_flops_per_launch": per_launch_flops,
                "peak_source": f"nominal {'FP32' if args.prec == 'mixed' else 'FP64'} rate: {fp['sms']} SMs (device) "
                               f"x {'128' if args.prec == 'mixed' else '2'} lanes x 2 flops x "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({src} max SM clock)",
                "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": peaks.get("hbm_gbs"), "frac": hbm_gbs / peaks.get("hbm_gbs"),
                        "algorithmic_bytes_per_launch": per_launch_bytes, "peak_source": src},
                "share_of_step": (ms_plane / args.steps) / ms}

    # the FP64 path's hot step on the same cell (the FP64 half of the metric's comparison)
    fp64 = None
    if args.prec == "mixed" and not args.no_fp64 and not large:  # no FP64 context holds a 144^2 plane
        c64 = fde.context_from_workload(wl, prec="fp64", stream=stream.cuda_stream)
        fde.seed_workload(c64, wl)
        c64.build_vemb()
        for _ in range(3):
            c64.hot_step(False)
        c64.sync()
        k64 = max(3, min(args.steps, 20))
        t64 = time_steps(c64, stream, flush, k64)
        ms64 = float(np.mean(t64))
        fp64 = {"value": ws * units / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                "dtype": "f64", "note": "the same hot step in an FP64 context, L2 flushed between steps"}
        del c64
        torch.cuda.empty_cache()

    pre = precond_kernels(ctx, wl, stream) if not large else None
    cpu = cpu_baseline(wl, bands=2 if large else None) if (rank == 0 and not args.no_cpu) else None
    ft = ft_cycles() if (ws == 1 and not args.no_ft and args.workload == "molecule-on-slab") else None
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": wl.name, "band_applies_per_step": units, "precision": args.prec,
                           "plane_variant": fde.tuned_plane_variant(wl.grid[0], wl.grid[2]),
                           "l2": "flushed between steps (256 MB write)", "seed": wl.seed,
                           "parallelism": f"replicas x{ws}"},
                "e2e": ({"value": ws * units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h, "host_buffers": "page-locked (torch pin_memory)"}
                        if e2e_s else None),
                "gpu_launches": launches, "roofline": roof, "kernels": table, "fp64": fp64,
                "cpu_baseline": cpu, "clocks": clocks, "ft_cycle": ft, "precond": pre,
                "wall_s": wall, "step_ms": step_ms,
                "graph": {"ms_per_step": graph_ms, "value": ws * units / (graph_ms / 1e3),
                          "note": "the same step replayed from a captured CUDA graph"}}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="molecule-on-slab", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 context's hot-step timing")
    ap.add_argument("--no-ft", action="store_true", help="skip the freeze-and-thaw cycle timings (~4 min)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
