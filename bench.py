#!/usr/bin/env python3
"""Benchmark of the periodic cubic-spline particle-tracking hot path on GB300.

Workload (one "step"): the spline-coefficient solve of a 512^3 three-component
FP32 field (random-phase k^-5/3 spectrum, 1 <= |k| <= 170, unit rms), then 10
Heun RK2 steps (dt = 1e-3) of 16,777,216 FP64 particles (uniform in the box)
with re-binning into 8^3-cell bricks before every RK2 step.  Inputs are larger
than L2 (1.6 GB field, 0.4 GB positions), so no L2 flush is added.

Unit: one particle interpolation of (u, v, w) at one position; an RK2 step
interpolates every particle twice, so value = n_gpus * 2 * 10 * Np / t_step.

`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s interpolated (u,v,w tricubic) + spline GB/s, % HBM roofline, 1 GB300"
UNIT = "particles/s"
N = 512
KMAX = 170
NP = 1 << 24
RK_STEPS = 10
DT = 1e-3
BRICK = (8, 8, 8)
FIELD_SEED = 1001
POS_SEED = 2001
WORKLOAD = ("mid: 512^3 FP32 u,v,w (k^-5/3, 1<=|k|<=170, unit rms), 16,777,216 uniform FP64 "
            "particles; spline solve + 10 Heun RK2 steps (dt 1e-3) with re-binning into 8^3 "
            "bricks every step")
# kernels of libps launched per bench step: 3 solve passes + 10 x (3 scan passes, 1 scatter
# and the RK2 step, which also counts the next sort's bins)
LAUNCHES_PER_STEP = 3 + RK_STEPS * 5
DOMINANT = "interp_staged<float4,3,RK2> (fused binned Heun step, halo by tensor copy)"
SOURCE_FOR_TRAFFIC = os.path.join(ROOT, "paper_2005_13193_gb300", "csrc", "interp.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default="interp,forms,batch,solve,prec",
                    help="comma list of the extra measurements to run (rank 0): interp, "
                         "forms, batch, solve, prec")
    # smaller cases of the same workload (profiling captures); defaults = mid
    ap.add_argument("--grid", type=int, default=None)
    ap.add_argument("--particles", type=int, default=None)
    ap.add_argument("--rk-steps", type=int, default=None)
    args = ap.parse_args()
    global N, NP, RK_STEPS, KMAX, LAUNCHES_PER_STEP, WORKLOAD
    args.reduced = bool(args.grid or args.particles or args.rk_steps)
    if args.reduced:
        N = args.grid or N
        NP = args.particles or NP
        RK_STEPS = args.rk_steps or RK_STEPS
        KMAX = N // 3
        LAUNCHES_PER_STEP = 3 + RK_STEPS * 5
        WORKLOAD = (f"reduced case: {N}^3 FP32 u,v,w (k^-5/3, 1<=|k|<={KMAX}), {NP} particles, "
                    f"solve + {RK_STEPS} RK2 steps, 8^3 bricks")
    return args


# Shared-memory wavefronts (128 B) per particle of the binned Heun step: two
# 64-point float4 gathers (16) plus the particle records, as counted by ncu
# (l1tex__data_pipe_lsu_wavefronts_mem_shared_op_{ld,st}) for the node form.
SMEM_WAVEFRONTS = 24.5


def smem_bound_ms(np_: int, sms: int = 152, clock_ghz: float = 2.07) -> float:
    """Time the shared-memory pipe needs for the Heun step's wavefronts."""
    return SMEM_WAVEFRONTS * np_ / (sms * clock_ghz * 1e9) * 1e3


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, pg, device) -> float:
    """The slowest rank's time: every rank's units count only once all are done."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units processed by all ranks (replicas of the same problem) per second."""
    return world * units_per_rank / (ms * 1e-3)


# ------------------------------------------------------------------ clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.idx = gpu_index
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def traffic_for(kernel_key: str):
    """Per-launch DRAM bytes from a committed ncu summary, or None if absent or
    taken on a different version of the kernel source."""
    try:
        sha = hashlib.sha256(open(SOURCE_FOR_TRAFFIC, "rb").read()).hexdigest()[:12]
        for line in open(TRAFFIC_FILE):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == sha:
                return float(parts[2])
    except Exception:
        pass
    return None


# --------------------------------------------------------------- our arm ----

def run_ours(args):
    import numpy as np
    import torch

    import paper_2005_13193_gb300 as ps
    from paper_2005_13193_gb300 import synth

    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    field = synth.spectral_field(N, KMAX, seed=FIELD_SEED, device=dev, dtype=torch.float32)
    pos_host = synth.uniform_particles(NP, seed=POS_SEED)
    pos0 = torch.from_numpy(pos_host).to(dev)
    n3 = (N, N, N)
    # FP32 coefficients stored as interleaved (u, v, w, 0) nodes
    coef = torch.empty(ps.coef_shape((N, N, N), 3, ps.F32X4), dtype=torch.float32, device=dev)
    ws_solve = ps.workspace(ps.ps_spline_coeffs_workspace_size((N, N, N), 3, ps.F32X4), dev)
    nb = [-(-N // b) for b in BRICK]
    nbins = nb[0] * nb[1] * nb[2]
    offsets = torch.empty(nbins + 1, dtype=torch.int32, device=dev)
    ws_rk = ps.workspace(ps.ps_rk2_workspace_size(n3, BRICK, NP), dev)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    vel = torch.empty((3, NP), dtype=torch.float32, device=dev)
    bufs = [pos0.clone(), torch.empty_like(pos0)]
    stream = torch.cuda.current_stream(dev)

    counted = [False]  # ws holds the counts of bufs[0]'s positions

    def one_step(ev_solve=None, ev_rk=None):
        if ev_solve:
            ev_solve[0].record(stream)
        ps.ps_spline_coeffs(field, coef, ws=ws_solve)
        if ev_solve:
            ev_solve[1].record(stream)
        for r in range(RK_STEPS):
            src, dst = bufs[0], bufs[1]
            # sort (from the counts the previous step's kernel took), then the
            # fused Heun step, which counts the bins of the positions it writes
            ps.ps_rk2_sort(n3, BRICK, src, dst, offsets, ws_rk, counted=counted[0],
                           status=status)
            if ev_rk:
                ev_rk[r][0].record(stream)
            ps.ps_rk2_step(coef, n3, dst, DT, vel_out=vel, brick=BRICK, rebin=0,
                           bin_offsets=offsets, ws=ws_rk, status=status)
            if ev_rk:
                ev_rk[r][1].record(stream)
            counted[0] = True
            bufs[0], bufs[1] = dst, src

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    st = ps.ps_status_read(status)
    if st[0] != 0:
        raise RuntimeError(f"device status after warm-up: {st}")

    K = args.steps
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ev_solve = [(mk(), mk()) for _ in range(K)]
    ev_rk = [[(mk(), mk()) for _ in range(RK_STEPS)] for _ in range(K)]
    t0, t1 = mk(), mk()
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0.record(stream)
    for k in range(K):
        one_step(ev_solve[k], ev_rk[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if pg:
        pg.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1) / K, pg, dev)

    solve_ms = statistics.mean(a.elapsed_time(b) for a, b in ev_solve)
    rk_ms = [a.elapsed_time(b) for step in ev_rk for a, b in step]
    rk_avg = statistics.mean(rk_ms)
    peak, peak_kind = measured_peaks()
    coef_bytes = 3 * 4 * (N + 3) ** 3
    # positions in and out, u1 out, the next sort's bin and rank out; the
    # coefficients once
    rk_alg_bytes = NP * (24 + 24 + 12 + 8) + coef_bytes
    solve_min_bytes = 3 * 4 * N ** 3 + coef_bytes
    # the two streamed passes: field in, intermediate out and back in, 16-byte
    # nodes out (the periodic images' copies, under 1%, left out)
    solve_pass_bytes = 3 * 4 * N ** 3 * 3 + 16 * (N + 3) ** 3
    achieved = rk_alg_bytes / (rk_avg * 1e-3) / 1e9
    units = 2 * RK_STEPS * NP
    value = whole_job_rate(units, ws_, ms)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded spectral field, uniform particles)",
        "config": {"workload": WORKLOAD, "grid": N, "particles": NP, "rk2_steps": RK_STEPS,
                   "dt": DT, "brick": list(BRICK), "coef_dtype": "f32",
                   "coef_storage": "f32x4 nodes (u, v, w, 0)",
                   "positions": "f64", "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{ws_} (independent problems)"},
        # the unit is one interpolation; a Heun step interpolates each particle
        # twice, so particle steps per second are half the value
        "rates": {"interpolations_per_s": value, "particle_rk2_steps_per_s": value / 2,
                  "unit_note": "value counts interpolations of (u, v, w); each Heun RK2 "
                               "step interpolates every particle twice"},
        "gpu_launches": LAUNCHES_PER_STEP * K,
        "clocks": clk,
        "roofline": {"bound": "hbm", "kernel": DOMINANT, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     # ncu bytes of the mid launch; other sizes have no entry
                     "traffic": traffic_for("rk2_staged_f32x4") if not args.reduced else None,
                     "alg_bytes_per_launch": rk_alg_bytes, "avg_launch_ms": rk_avg,
                     # the shared-memory pipe: one 128-byte wavefront per clock per SM;
                     # SMEM_WAVEFRONTS per particle from the ncu summary in profiles/
                     "smem_bound_ms": smem_bound_ms(NP),
                     "frac_of_smem_bound": smem_bound_ms(NP) / rk_avg},
        "breakdown": {"solve_ms": solve_ms,
                      "solve_gbs_min_bytes": solve_min_bytes / (solve_ms * 1e-3) / 1e9,
                      "solve_gbs_pass_bytes": solve_pass_bytes / (solve_ms * 1e-3) / 1e9,
                      "solve_frac_of_peak_min_bytes": solve_min_bytes / (solve_ms * 1e-3) / 1e9
                      / peak,
                      "rk2_kernel_ms_avg": rk_avg,
                      "rk2_kernel_particles_per_s": 2 * NP / (rk_avg * 1e-3),
                      "bin_and_rest_ms_per_rk_step": (ms - solve_ms) / RK_STEPS - rk_avg},
    }

    if not args.no_extras and rank == 0:
        want = set(args.extras.split(","))
        if "interp" in want:
            result["interp_sorted_vs_unsorted"] = interp_extras(ps, torch, dev, coef, bufs[0], n3)
        if "forms" in want:
            result["coef_forms"] = precision_forms(ps, torch, dev, field, coef, bufs[0], n3)
        if "batch" in want:
            result["batched_48_fields"] = batch_extras(ps, torch, dev)
        if "solve" in want:
            result["solve_forms"] = solve_forms(ps, torch, dev, field)
        if "prec" in want:
            result["precision_1536"] = precision_extras(ps, torch, dev)
    if not args.no_e2e:
        result["e2e"] = e2e_measure(ps, torch, dev, field, pos_host, coef, ws_solve, n3, K, ws_,
                                    pg)
    if rank == 0 and ws_ == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(field.cpu().numpy(), pos_host)
    if rank == 0:
        print(json.dumps(result))
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def interp_extras(ps, torch, dev, coef, pos_sorted_by_bin, n3):
    """One interpolation of all particles, unsorted (random storage order, direct
    gathers) vs sorted (bin order, staged halos); then, on the sorted order, the
    velocity gradient, the second derivatives and the Lagrangian acceleration."""
    g = torch.Generator(device="cpu").manual_seed(5)
    perm = torch.randperm(NP, generator=g).to(dev)
    pos_rand = pos_sorted_by_bin[:, perm].contiguous()
    vel = torch.empty((3, NP), dtype=torch.float32, device=dev)
    grad = torch.empty((3, 3, NP), dtype=torch.float32, device=dev)
    hess = torch.empty((3, 6, NP), dtype=torch.float32, device=dev)
    acc = torch.empty((3, NP), dtype=torch.float32, device=dev)
    # physically sorted copy
    bins2, pos_sorted = ps.bin_particles(n3, BRICK, pos_sorted_by_bin, want_sorted=True)
    out = {}
    for name, fn in (
            ("unsorted_direct", lambda: ps.ps_interp(coef, n3, pos_rand, vel)),
            ("sorted_direct", lambda: ps.ps_interp(coef, n3, pos_sorted, vel)),
            ("sorted_staged", lambda: ps.ps_interp(coef, n3, pos_sorted, vel,
                                                   bin_offsets=bins2.offsets, brick=BRICK)),
            ("sorted_staged_grad", lambda: ps.ps_interp(coef, n3, pos_sorted, vel, grad=grad,
                                                        bin_offsets=bins2.offsets,
                                                        brick=BRICK)),
            # second derivatives: direct quad-per-particle gathers
            ("sorted_hessian_direct", lambda: ps.ps_interp_hessian(coef, n3, pos_sorted, hess)),
            # du/dt + (u . grad) u with a second field: 2 + 9 sums per particle
            ("sorted_accel_direct", lambda: ps.ps_lagrangian_accel(coef, n3, pos_sorted, acc,
                                                                   coef_np1=coef,
                                                                   dt_field=1.0)),
            # the same two from each brick's staged halo (the second field's
            # stencils from global memory)
            ("sorted_staged_hessian", lambda: ps.ps_interp_hessian(
                coef, n3, pos_sorted, hess, bin_offsets=bins2.offsets, brick=BRICK)),
            ("sorted_staged_accel", lambda: ps.ps_lagrangian_accel(
                coef, n3, pos_sorted, acc, coef_np1=coef, dt_field=1.0,
                bin_offsets=bins2.offsets, brick=BRICK))):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            fn()
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 5
        out[name] = {"ms": t, "particles_per_s": NP / (t * 1e-3)}
    del grad, hess, acc
    return out


def _event_ms(torch, fn, reps, warmup=2):
    for _ in range(warmup):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def precision_forms(ps, torch, dev, field, coef_nodes, pos_now, n3):
    """The same solve and binned RK2 step with FP32 planar, BF16 and FP16
    coefficients (power-of-two scale per component and x-line; as nodes and
    planar) beside the FP32 node form the benchmark runs: kernel times, and the
    velocity error of every particle against FP32, relative to the rms
    velocity."""
    # positions stored in bin order (the staged kernel's precondition)
    bins, pos_binned = ps.bin_particles(n3, BRICK, pos_now, want_sorted=True,
                                        want_perm=False)
    offs = bins.offsets
    del bins
    vel32 = torch.empty((3, NP), dtype=torch.float32, device=dev)
    vel = torch.empty_like(vel32)
    pos = torch.empty_like(pos_binned)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    out = {}
    for name, dt_ in (("f32x4", ps.F32X4), ("f32", torch.float32), ("bf16x4", ps.BF16X4),
                      ("f16x4", ps.F16X4), ("bf16", torch.bfloat16), ("f16", torch.float16)):
        if dt_ == ps.F32X4:
            c = coef_nodes
        else:
            c = torch.empty(ps.coef_shape(n3, 3, dt_), dtype=ps._storage_dtype(dt_), device=dev)
        shp = ps.scale_shape(n3, 3, dt_)
        s = torch.empty(shp, dtype=torch.float32, device=dev) if shp is not None else None
        need = ps.ps_spline_coeffs_workspace_size(n3, 3, dt_)
        wsq = ps.workspace(need, dev) if need else None
        t_solve = _event_ms(torch, lambda: ps.ps_spline_coeffs(field, c, scale=s, ws=wsq), 3)

        evs = []

        def rk():
            # every run starts from the binned positions (the bins stay valid)
            pos.copy_(pos_binned)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ps.ps_rk2_step(c, n3, pos, DT, scale_n=s, vel_out=vel, brick=BRICK, rebin=False,
                           bin_offsets=offs, status=status)
            b.record()
            evs.append((a, b))
        for _ in range(2):
            rk()
        evs.clear()
        for _ in range(5):
            rk()
        torch.cuda.synchronize()
        t_rk = statistics.mean(a.elapsed_time(b) for a, b in evs)
        e = {"solve_ms": t_solve, "rk2_kernel_ms": t_rk,
             "rk2_particles_per_s": 2 * NP / (t_rk * 1e-3),
             "coef_bytes": c.numel() * c.element_size()}
        if dt_ == ps.F32X4:
            vel32.copy_(vel)
        else:
            d = (vel - vel32).double()
            rms = float(torch.sqrt((vel32.double() ** 2).mean()))
            e["max_err_vs_f32_rel_rms"] = float(d.abs().max()) / rms
            e["rms_err_vs_f32_rel_rms"] = float(torch.sqrt((d ** 2).mean())) / rms
        out[name] = e
        del c, s, wsq
    if ps.ps_status_read(status)[0] != 0:
        raise RuntimeError("device status set in the coefficient-form runs")
    return out


def solve_forms(ps, torch, dev, field):
    """The same 512^3 three-component solve, planar FP32 output: the exact
    chunked recursions (ps_spline_coeffs) against the convolution with the
    periodic inverse cut to |d| <= 15 (ps_spline_coeffs_truncated)."""
    n3 = (N, N, N)
    exact = torch.empty(ps.coef_shape(n3, 3, torch.float32), dtype=torch.float32, device=dev)
    trunc = torch.empty_like(exact)
    ws_e = ps.workspace(ps.ps_spline_coeffs_workspace_size(n3, 3, torch.float32), dev)
    ws_t = ps.workspace(ps.ps_spline_truncated_workspace_size(n3, 3), dev)
    t_exact = _event_ms(torch, lambda: ps.ps_spline_coeffs(field, exact, ws=ws_e), 5)
    t_trunc = _event_ms(torch, lambda: ps.ps_spline_coeffs_truncated(field, trunc, K=15,
                                                                     ws=ws_t), 5)
    diff = (trunc - exact).abs().max().item() / exact.abs().max().item()
    out = {"exact_ms": t_exact, "truncated_k15_ms": t_trunc,
           "max_diff_rel_max_coef": diff}
    del exact, trunc, ws_e, ws_t
    return out


PREC_N = 1536
PREC_NP = 300_000_000
# single-interpolation floors at the measured HBM peak (positions 24 B in,
# velocities 12 B out per particle, the coefficients once at 12 B (FP32) or
# 6 B (16-bit) per node); the prec rows of the roofline table
PREC_FLOOR = {"f32x4": 3.7e10, "bf16x4": 6.2e10, "f16x4": 6.2e10}


def precision_extras(ps, torch, dev):
    """The 1536^3 workload: FP32 field (k^-5/3, 1 <= |k| <= 512), 300,000,000
    uniform particles; per coefficient storage (FP32, BF16 and FP16 nodes):
    the solve, one binned interpolation of every particle and one binned Heun
    step, device-timed with CUDA events.  Skipped below 200 GB of free
    device memory."""
    from paper_2005_13193_gb300 import synth
    free, _ = torch.cuda.mem_get_info(dev)
    if free < 200e9:
        return {"skipped": f"needs 200 GB of free device memory, {free / 1e9:.0f} GB free"}
    n3 = (PREC_N,) * 3
    peak, _ = measured_peaks()
    field = synth.spectral_field_planes(PREC_N, 512, seed=1002, device=dev)
    pos = torch.from_numpy(synth.uniform_particles(PREC_NP, seed=2002)).to(dev)
    bins, pos_b = ps.bin_particles(n3, BRICK, pos, want_sorted=True, want_perm=False)
    offs = bins.offsets
    del bins, pos
    vel = torch.empty((3, PREC_NP), dtype=torch.float32, device=dev)
    work = torch.empty_like(pos_b)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    out = {"grid": PREC_N, "particles": PREC_NP, "brick": list(BRICK)}
    for name, dt_, cb in (("f32x4", ps.F32X4, 12), ("bf16x4", ps.BF16X4, 6),
                          ("f16x4", ps.F16X4, 6)):
        c = torch.empty(ps.coef_shape(n3, 3, dt_), dtype=ps._storage_dtype(dt_), device=dev)
        shp = ps.scale_shape(n3, 3, dt_)
        sc = torch.empty(shp, dtype=torch.float32, device=dev) if shp is not None else None
        wsq = ps.workspace(ps.ps_spline_coeffs_workspace_size(n3, 3, dt_), dev)
        t_solve = _event_ms(torch, lambda: ps.ps_spline_coeffs(field, c, scale=sc, ws=wsq), 3,
                            warmup=1)
        del wsq
        t_int = _event_ms(torch, lambda: ps.ps_interp(c, n3, pos_b, vel, scale=sc,
                                                      bin_offsets=offs, brick=BRICK,
                                                      status=status), 3, warmup=1)
        evs = []

        def rk():
            work.copy_(pos_b)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ps.ps_rk2_step(c, n3, work, DT, scale_n=sc, vel_out=vel, brick=BRICK, rebin=False,
                           bin_offsets=offs, status=status)
            b.record()
            evs.append((a, b))
        rk()
        evs.clear()
        for _ in range(3):
            rk()
        torch.cuda.synchronize()
        t_rk = statistics.mean(a.elapsed_time(b) for a, b in evs)
        coef_alg = cb * (PREC_N + 3) ** 3  # cb: bytes of the three components of a node
        solve_min = 3 * 4 * PREC_N ** 3 + coef_alg
        interp_alg = PREC_NP * 36 + coef_alg
        rk_alg = PREC_NP * 60 + coef_alg
        out[name] = {
            "solve_ms": t_solve, "solve_gbs_min_bytes": solve_min / (t_solve * 1e-3) / 1e9,
            "solve_frac_of_peak": solve_min / (t_solve * 1e-3) / 1e9 / peak,
            "interp_ms": t_int, "interp_particles_per_s": PREC_NP / (t_int * 1e-3),
            "interp_frac_of_peak": interp_alg / (t_int * 1e-3) / 1e9 / peak,
            "interp_vs_floor": PREC_NP / (t_int * 1e-3) / PREC_FLOOR[name],
            "rk2_kernel_ms": t_rk, "rk2_interpolations_per_s": 2 * PREC_NP / (t_rk * 1e-3),
            "rk2_frac_of_peak": rk_alg / (t_rk * 1e-3) / 1e9 / peak,
            "coef_bytes": c.numel() * c.element_size()}
        del c, sc
        torch.cuda.empty_cache()
    out["status"] = [int(v) for v in ps.ps_status_read(status)]
    del field, pos_b, offs, vel, work
    torch.cuda.empty_cache()
    return out


def batch_extras(ps, torch, dev):
    """The many-fields workload: 48 fields with edges uniform over {64, 96,
    128, 192, 256}, 10k..2M particles per field (log-uniform), 20 Heun steps
    (dt 1e-3).  Batched plan (autotuned brick; the 48 solves and the 20 steps
    replayed from one CUDA graph, the steps as one persistent launch or as a
    launch per phase and step) against a loop of single-field Tracker steps
    on the same GPU."""
    from paper_2005_13193_gb300 import autotune, synth
    sizes, nps = synth.batch_sizes(48, seed=3000)
    nsteps, dt = 20, 1e-3
    flds = []
    for i, n in enumerate(sizes):
        f = synth.spectral_field(n, n // 3, seed=3100 + i, device=dev, dtype=torch.float32)
        flds.append((f, ps.SplineField.from_field(f, ps.F32X4)))
    pos0 = torch.cat([torch.from_numpy(synth.uniform_particles(v, seed=3200 + i))
                      for i, v in enumerate(nps)], dim=1).to(dev)
    grids = [(n,) * 3 for n in sizes]
    best, table = autotune.tune_batch(grids, nps, flds, pos0, coef_dtype=ps.F32X4)
    plan = ps.BatchPlan(grids, nps, coef_dtype=ps.F32X4, brick=best)
    pos = pos0.clone()
    ids = torch.arange(plan.np_total, dtype=torch.int64, device=dev)
    # the 48 solves and the 20 steps in one graph: the steps as one cooperative
    # persistent launch (default), and as a launch per phase and step
    timings = {}
    old = ps.ps_tune_get("batch_persistent")
    try:
        for name, pers in (("persistent", 1), ("launch_per_step", 0)):
            ps.ps_tune_set("batch_persistent", pers)
            plan.run(flds, pos, nsteps, dt, solve=True, ids=ids, use_graph=True)  # capture
            timings[name] = _event_ms(torch, lambda: plan.run(flds, pos, nsteps, dt, solve=True,
                                                              ids=ids, use_graph=True), 3,
                                      warmup=1)
        ps.ps_tune_set("batch_persistent", 1)
        plan.run(flds, pos, nsteps, dt, solve=False, ids=ids, use_graph=True)
        t_steps = _event_ms(torch, lambda: plan.run(flds, pos, nsteps, dt, solve=False, ids=ids,
                                                    use_graph=True), 3, warmup=1)
    finally:
        ps.ps_tune_set("batch_persistent", old)
    t_graph = timings["persistent"]
    trackers = []
    for f, (n, v) in enumerate(zip(sizes, nps)):
        b = plan.base[f]
        trackers.append(ps.Tracker(flds[f][1], pos0[:, b:b + v].clone(), brick=BRICK,
                                   keep_velocity=False))

    def loop():
        for _ in range(nsteps):
            for tr in trackers:
                tr.step(dt)
    t_loop = _event_ms(torch, loop, 2, warmup=1)
    units = 2 * nsteps * plan.np_total
    return {"fields": len(sizes), "particles": plan.np_total, "rk2_steps": nsteps,
            "coef_storage": "f32x4 nodes",
            "autotuned_brick": list(best),
            "autotune_ms_per_step": {"x".join(map(str, k)): v for k, v in table.items()},
            "graph": "48 solves + 20 Heun steps",
            "batched_graph_ms": t_graph, "batched_particles_per_s": units / (t_graph * 1e-3),
            "launch_per_step_graph_ms": timings["launch_per_step"],
            "steps_only_persistent_ms": t_steps,
            "steps_only_particles_per_s": units / (t_steps * 1e-3),
            "per_field_loop_ms": t_loop, "loop_particles_per_s": units / (t_loop * 1e-3),
            "loop_note": "per-field Tracker steps without the solves"}


def e2e_measure(ps, torch, dev, field, pos_host, coef, ws_solve, n3, K, ws_, pg):
    """The same step through the public API from pinned host buffers: every step
    copies the field and the positions in and reads the positions and
    velocities out.  Inputs are double-buffered; uploads and readbacks run on
    two copy streams (one per direction), and a field buffer is refilled as soon
    as the solve that read it has finished, so the copies overlap one another
    and the compute."""
    field_h = field.cpu().pin_memory()
    pos_h = torch.from_numpy(pos_host).pin_memory()
    pos_out_h = torch.empty_like(pos_h).pin_memory()
    vel_h = torch.empty((3, NP), dtype=torch.float32).pin_memory()
    field_d = [torch.empty_like(field) for _ in range(2)]
    pos_d = [torch.empty((3, NP), dtype=torch.float64, device=dev) for _ in range(2)]
    vel_d = [torch.empty((3, NP), dtype=torch.float32, device=dev) for _ in range(2)]
    ids0 = torch.arange(NP, dtype=torch.int64, device=dev)
    ids = [torch.empty_like(ids0) for _ in range(2)]
    ws = ps.workspace(ps.ps_rk2_workspace_size(n3, BRICK, NP), dev)
    nb = [-(-N // b) for b in BRICK]
    offsets = torch.empty(nb[0] * nb[1] * nb[2] + 1, dtype=torch.int32, device=dev)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()  # noqa: E731
    ev_field_in, ev_pos_in = [ev(), ev()], [ev(), ev()]
    ev_field_free, ev_done, ev_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for b in range(2):  # every buffer starts free
        ev_field_free[b].record(st)
        ev_out[b].record(st)

    def upload(b):
        with torch.cuda.stream(up):
            up.wait_event(ev_field_free[b])   # the solve that read this field is done
            field_d[b].copy_(field_h, non_blocking=True)
            ev_field_in[b].record(up)
            up.wait_event(ev_out[b])          # this buffer's positions were read back
            pos_d[b].copy_(pos_h, non_blocking=True)
            ev_pos_in[b].record(up)

    def compute(b):
        st.wait_event(ev_field_in[b])
        ps.ps_spline_coeffs(field_d[b], coef, ws=ws_solve, stream=st)
        ev_field_free[b].record(st)
        st.wait_event(ev_pos_in[b])
        ids[b].copy_(ids0)
        for r in range(RK_STEPS):
            # the first step sorts the uploaded positions; each step's kernel
            # counts the bins of the positions it writes for the next sort
            ps.ps_rk2_step(coef, n3, pos_d[b], DT, ids=ids[b], vel_out=vel_d[b], brick=BRICK,
                           rebin=2 if r == 0 else 3, bin_offsets=offsets, ws=ws,
                           status=status, stream=st)
        ev_done[b].record(st)

    def readback(b):
        with torch.cuda.stream(down):
            down.wait_event(ev_done[b])
            pos_out_h.copy_(pos_d[b], non_blocking=True)
            vel_h.copy_(vel_d[b], non_blocking=True)
            ev_out[b].record(down)

    def run(steps, t0=None, t1=None):
        if t0 is not None:
            t0.record(st)
            up.wait_stream(st)
            down.wait_stream(st)
        upload(0)
        for k in range(steps):
            b = k & 1
            if k + 1 < steps:
                upload(1 - b)
            compute(b)
            readback(b)
        if t1 is not None:
            st.wait_stream(up)
            st.wait_stream(down)
            t1.record(st)

    run(2)
    torch.cuda.synchronize()
    steps = max(3, min(K, 6))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    run(steps, a, b)
    torch.cuda.synchronize()
    ms = max_over_ranks(a.elapsed_time(b) / steps, pg, dev)
    # the host link on its own, one direction at a time, best of three (context
    # for the number above)
    def link_gbs(dst, src):
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            dst.copy_(src, non_blocking=True)
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return src.numel() * src.element_size() / (best * 1e-3) / 1e9

    h2d_gbs = link_gbs(field_d[0], field_h)
    d2h_gbs = link_gbs(pos_out_h, pos_d[0])
    units = 2 * RK_STEPS * NP
    return {"value": whole_job_rate(units, ws_, ms), "unit": UNIT, "ms_per_step": ms,
            "steps": steps,
            "h2d_bytes_per_step": field_h.numel() * 4 + pos_h.numel() * 8,
            "d2h_bytes_per_step": pos_out_h.numel() * 8 + vel_h.numel() * 4,
            "host_link_gbs": {"h2d": h2d_gbs, "d2h": d2h_gbs},
            "api": "ps_spline_coeffs + ps_rk2_step(rebin=2, then 3, ids); inputs double-buffered, "
                   "one copy stream per direction"}


# ------------------------------------------------------------- the oracle ----

CPU_SAMPLE = 65536      # particles of the all-core sample
CPU_SAMPLE_1T = 8192    # particles of the single-thread sample
SOLVE_1T_N = 256        # grid of the single-thread solve


def oracle_step(oracle, field64, pos_sample):
    """One bounded sample of the workload on the host: the full 512^3 FP64
    solve, then 10 RK2 steps of a particle subsample on those coefficients.
    Returns (t_solve, t_rk2) in seconds, both measured."""
    t = time.perf_counter()
    coef = oracle.spline_coeffs(field64)
    t_solve = time.perf_counter() - t
    p = pos_sample.copy()
    t = time.perf_counter()
    for _ in range(RK_STEPS):
        p, _ = oracle.rk2_step(coef, p, DT)
    t_rk = time.perf_counter() - t
    return t_solve, t_rk


def full_step_rate(t_solve, t_rk, n_sample):
    """Interpolations per second of the full step (solve + 10 RK2 steps of NP
    particles) from its measured parts: the solve timed in full, the particle
    steps timed on n_sample particles and scaled by NP / n_sample (each
    particle's work does not depend on how many there are)."""
    t_full = t_solve + t_rk * (NP / n_sample)
    return 2 * RK_STEPS * NP / t_full


def _timed(fn):
    t = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t


def _rk2_sample(oracle, coef, pos_host, n_sample):
    p = pos_host[:, :n_sample].copy()
    t = time.perf_counter()
    for _ in range(RK_STEPS):
        p, _ = oracle.rk2_step(coef, p, DT)
    return time.perf_counter() - t


def cpu_baseline(field_np, pos_host):
    """The oracle timed on the host: all cores and one thread, the solve
    (GB/s of algorithmic bytes: FP64 field in, FP64 padded coefficients out)
    and the RK2 particle steps (interpolations/s) measured separately; value
    = the full step's rate built from the all-core parts."""
    import numpy as np
    import torch

    import oracle
    from paper_2005_13193_gb300 import synth
    cores = os.cpu_count() or 1
    field64 = field_np.astype(np.float64)
    sbytes = lambda n: 3 * 8 * (n ** 3 + (n + 3) ** 3)  # noqa: E731
    oracle.set_num_threads(cores)
    coef, t_solve = _timed(lambda: oracle.spline_coeffs(field64))
    t_rk = _rk2_sample(oracle, coef, pos_host, CPU_SAMPLE)
    allc = {"threads": oracle.num_threads(), "solve_grid": N, "solve_s": t_solve,
            "solve_gbs": sbytes(N) / t_solve / 1e9, "rk2_sample_particles": CPU_SAMPLE,
            "rk2_sample_s": t_rk, "interp_per_s": 2 * RK_STEPS * CPU_SAMPLE / t_rk}
    # one thread: the solve of a 256^3 field of the same recipe (the 512^3 one
    # would take most of a minute), the particle steps on the 512^3 coefficients
    f1 = synth.spectral_field(SOLVE_1T_N, SOLVE_1T_N // 3, seed=FIELD_SEED, device="cpu",
                              dtype=torch.float64).numpy()
    oracle.set_num_threads(1)
    _, t1_solve = _timed(lambda: oracle.spline_coeffs(f1))
    t1_rk = _rk2_sample(oracle, coef, pos_host, CPU_SAMPLE_1T)
    one = {"threads": oracle.num_threads(), "solve_grid": SOLVE_1T_N, "solve_s": t1_solve,
           "solve_gbs": sbytes(SOLVE_1T_N) / t1_solve / 1e9,
           "rk2_sample_particles": CPU_SAMPLE_1T, "rk2_sample_s": t1_rk,
           "interp_per_s": 2 * RK_STEPS * CPU_SAMPLE_1T / t1_rk}
    oracle.set_num_threads(cores)
    return {"value": full_step_rate(t_solve, t_rk, CPU_SAMPLE), "unit": UNIT,
            "cores": allc["threads"], "kind": "oracle", "extrapolated": True,
            "sample": (f"all cores: full 512^3 FP64 solve ({t_solve:.2f} s) + 10 RK2 steps of "
                       f"{CPU_SAMPLE} particles ({t_rk:.2f} s), both measured; value = the full "
                       f"step's rate with the particle part scaled to {NP} particles"),
            "full_step_s_extrapolated": t_solve + t_rk * NP / CPU_SAMPLE,
            "all_cores": allc, "single_thread": one}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores.  Each step is one
    measured bounded sample (the full 512^3 solve + 10 RK2 steps of
    CPU_SAMPLE particles); ms_per_step is that sample's measured time, value
    the full step's rate built from its measured parts (extrapolated: the
    particle steps scaled to NP)."""
    import numpy as np
    import torch

    import oracle
    from paper_2005_13193_gb300 import synth

    ws_, rank, _ = dist_env()
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    field = synth.spectral_field(N, KMAX, seed=FIELD_SEED, device=dev, dtype=torch.float32)
    field64 = field.cpu().numpy().astype(np.float64)
    del field
    pos = synth.uniform_particles(NP, seed=POS_SEED)[:, :CPU_SAMPLE].copy()
    cores = os.cpu_count() or 1
    oracle.set_num_threads(cores)
    for _ in range(args.warmup):
        oracle_step(oracle, field64, pos)
    solves, rks, walls = [], [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        ts, tr = oracle_step(oracle, field64, pos)
        walls.append(time.perf_counter() - t)
        solves.append(ts)
        rks.append(tr)
    wall = time.perf_counter() - t0
    t_solve, t_rk = statistics.mean(solves), statistics.mean(rks)
    value = full_step_rate(t_solve, t_rk, CPU_SAMPLE)
    sample_ms = 1e3 * statistics.mean(walls)
    sample = (f"full 512^3 FP64 solve ({t_solve:.2f} s) + 10 RK2 steps of {CPU_SAMPLE} "
              f"particles ({t_rk:.3f} s) per step, both measured; value = the full step's "
              f"rate with the particle part scaled to {NP} particles")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded spectral field, uniform particles)",
        "config": {"workload": WORKLOAD, "grid": N, "particles": NP, "rk2_steps": RK_STEPS,
                   "dt": DT, "brick": list(BRICK)},
        "extrapolated": True,
        "measured": {"solve_s": t_solve, "rk2_sample_s": t_rk, "sample_particles": CPU_SAMPLE,
                     "sample_step_ms": sample_ms,
                     "sample_interp_per_s": 2 * RK_STEPS * CPU_SAMPLE / t_rk,
                     "solve_gbs": 3 * 8 * (N ** 3 + (N + 3) ** 3) / t_solve / 1e9,
                     "full_step_s_extrapolated": t_solve + t_rk * NP / CPU_SAMPLE},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample, "extrapolated": True},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
