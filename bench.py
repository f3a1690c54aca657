"""Throughput of the embedded H psi hot path on one GB300 (or N replicas under torchrun).

Workload: the molecule-on-slab cell (16 x 16 x 40 bohr, 72 x 72 x 180 grid, 20 Ha): a 36-atom
Z=3 slab with 64 bands x 4 k-points (Fermi smearing) plus a 6-atom Z=4 molecule with
12 bands at Gamma, PBE + revAPBEK, 2 Gaussian KB projectors per atom; seeded synthetic
inputs (paper_1406_7803_gb300.workloads).

One step = one pass of the hot path over the whole cell: the embedding-potential build
(rho = sum rho_I, FFT Poisson, FFT gradients, pointwise xc and GGA kinetic potentials,
divergence, assembly of V_eff^I) followed by H_I psi for every band of every (subsystem,
k-point): 4 x 64 + 12 = 268 band-applies.  value = band-applies per second over all ranks.

Second part of the metric (N = 1, skipped with --no-ft): seconds per freeze-and-thaw cycle
at 1e-6 Ha on the same cell, mixed precision (with and without the learned preconditioner)
against the plain FP64 GPU path ("ft_cycle" in the JSON line).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
                       [--impl ours|reference] [--no-cpu] [--no-ft]
"""
from __future__ import annotations

import argparse
import json
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
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
    fields = dict(l.split(":", 1) for l in text.splitlines() if l.startswith(("traffic_bytes_per_launch:", "source_sha256:")))
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


def cpu_baseline(wl, max_seconds=15.0):
    """The FP64 oracle timed on this host's cores on a bounded sample of the workload:
    one embedding-potential build plus H psi for as many bands as fit in ~max_seconds;
    band-applies/s of a full step is extrapolated from the two measured parts."""
    from oracle import basis as obasis
    from oracle import fde as ofde
    t0 = time.perf_counter()
    sy = ofde.System(wl)
    rhos = np.array([workloads.initial_density(wl, I) for I in range(wl.nsub)])
    t1 = time.perf_counter()
    pot = sy.build_veff(rhos)
    t_veff = time.perf_counter() - t1
    done, t_h = 0, 0.0
    I, k = 0, 0
    s = wl.subsystems[0]
    npw = sy.basis[I][k][0].shape[0]
    while t_h < max_seconds and done < 64:
        c = workloads.raw_orbitals(5, I, k, 1, npw)
        t1 = time.perf_counter()
        sy.apply_h(I, k, c, pot["veff"][I])
        t_h += time.perf_counter() - t1
        done += 1
    t_band = t_h / max(done, 1)
    units = wl.band_k_pairs()
    step = t_veff + units * t_band
    cores = os.cpu_count()
    return {"value": units / step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one FP64 v_eff build ({t_veff:.2f} s) + {done} slab band-applies "
                      f"({t_band * 1e3:.1f} ms each, scipy.fft workers={cores}), extrapolated to "
                      f"{units} band-applies per step; setup {t1 - t0:.1f} s excluded"}


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


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = workloads.molecule_on_slab()
    from oracle import fde as ofde
    sy = ofde.System(wl)
    rhos = np.array([workloads.initial_density(wl, I) for I in range(wl.nsub)])
    units = wl.band_k_pairs()
    sample_bands = 4
    npw = sy.basis[0][0][0].shape[0]

    def step():
        t0 = time.perf_counter()
        pot = sy.build_veff(rhos)
        t1 = time.perf_counter()
        c = workloads.raw_orbitals(5, 0, 0, sample_bands, npw)
        sy.apply_h(0, 0, c, pot["veff"][0])
        t2 = time.perf_counter()
        return (t1 - t0) + units * (t2 - t1) / sample_bands

    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    ms = 1e3 * float(np.mean(times))
    val = units / (ms / 1e3)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "band_applies_per_step": units, "seed": wl.seed},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: one FP64 v_eff build + {sample_bands} slab band-applies, "
                                       f"extrapolated to {units}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1406_7803_gb300 import fde
    wl = workloads.molecule_on_slab()
    # one non-default stream for the library, the L2 flush and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = fde.context_from_workload(wl, prec=args.prec, stream=stream.cuda_stream)
    fde.seed_workload(ctx, wl)
    ctx.build_vemb()
    ctx.sync()
    units = wl.band_k_pairs()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        ctx.hot_step(False)

    for _ in range(max(args.warmup, 3)):
        step()
    ctx.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.profile_enable(True)
    launches0 = ctx.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launches = ctx.launch_count() - launches0
    total_ms = float(np.sum(step_ms))
    prof = {n: ctx.profile_get(n) for n in ("k_zinv", "k_plane", "k_zfwd")}
    ctx.profile_enable(False)
    ms, value = whole_job(total_ms, args.steps, units, ws, "cuda")

    # the same pass replayed from a captured CUDA graph (launch overhead removed)
    ctx.hot_step(True)
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        gev[i][0].record(stream)
        ctx.hot_step(True)
        gev[i][1].record(stream)
    torch.cuda.synchronize()
    graph_ms = float(np.mean([a.elapsed_time(b) for a, b in gev]))

    # end to end through the C ABI with host buffers: densities in, H psi out
    rhos_h = [workloads.initial_density(wl, I) for I in range(wl.nsub)]
    psi_h, h_out, h2d, d2h = [], [], 0, 0
    for I, s in enumerate(wl.subsystems):
        for k in range(s.nk):
            npw = ctx.basis(I, k).shape[0]
            psi_h.append((I, k, s.nbands, workloads.raw_orbitals(9, I, k, s.nbands, npw)))
            h_out.append(np.zeros((s.nbands, npw), dtype=np.complex128))
    for r in rhos_h:
        h2d += r.nbytes
    for (_, _, _, c), o in zip(psi_h, h_out):
        h2d += c.nbytes
        d2h += o.nbytes

    def e2e_step():
        for I, r in enumerate(rhos_h):
            ctx.set_density(I, r)
        ctx.build_vemb()
        for (I, k, nb, c), o in zip(psi_h, h_out):
            ctx.apply_h_host(I, k, c, o, nb)

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(2, args.steps // 2)
    for _ in range(ne):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ne
    e2e_s = max_over_ranks(e2e_s, ws, "cuda")

    # roofline of the dominant kernel (the fused plane pass of the local H psi)
    peaks, src = _peaks()
    n_plane, ms_plane = prof["k_plane"]
    roof = None
    if n_plane:
        # ALU bound: FFT flops of the (x, y) plane passes the kernel performs, counted with
        # the 5 N log2 N convention per line, plus the potential multiply.
        g = wl.grid
        flops = 0.0
        for I, s in enumerate(wl.subsystems):
            for k in range(s.nk):
                mil = ctx.basis(I, k)
                nrow = len(np.unique(mil[:, 0]))
                per_plane = 2 * (nrow * 5 * g[1] * np.log2(g[1]) + g[1] * 5 * g[0] * np.log2(g[0])) + 2 * g[0] * g[1]
                flops += s.nbands * g[2] * per_plane
        flops_per_launch = flops * args.steps / n_plane
        sec = ms_plane / n_plane / 1e3
        sm_mhz = peaks.get("clocks_under_load", {}).get("sm_mhz_median") or peaks.get("sm_max_mhz", 2070.0)
        lanes = 4 * 32  # FP32 lanes per SM
        fp_peak = 152 * lanes * 2 * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12  # FMA = 2 flops
        if args.prec == "fp64":
            fp_peak = 1.25  # nominal FP64 rate of the part (TFLOP/s)
        achieved = flops_per_launch / sec / 1e12
        traffic = (_profile_traffic("k_plane_ct_molecule_on_slab", PLANE_SOURCES, PLANE_FUNCTION)
                   if args.prec == "mixed" else None)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp_peak, "unit": "TFLOP/s", "frac": achieved / fp_peak,
                "traffic": traffic, "kernel": "k_plane", "launches": n_plane,
                "avg_launch_us": 1e6 * sec, "peak_source": f"{'FP32' if args.prec != 'fp64' else 'FP64'} lanes x "
                f"clock ({'152 SMs x 128 lanes x 2 x sm_max' if args.prec != 'fp64' else 'nominal'}); "
                f"HBM peak {peaks.get('hbm_gbs')} GB/s {src}",
                "share_of_step": (ms_plane / args.steps) / ms}
        del sm_mhz
    cpu = cpu_baseline(wl) if (rank == 0 and not args.no_cpu) else None
    ft = ft_cycles() if (ws == 1 and not args.no_ft) else None
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": wl.name, "band_applies_per_step": units, "precision": args.prec,
                           "plane_variant": fde.tuned_plane_variant(wl.grid[0], wl.grid[2]),
                           "l2": "flushed between steps (256 MB write)", "seed": wl.seed,
                           "parallelism": f"replicas x{ws}"},
                "e2e": {"value": ws * units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "ft_cycle": ft,
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
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ft", action="store_true", help="skip the freeze-and-thaw cycle timings (~4 min)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
