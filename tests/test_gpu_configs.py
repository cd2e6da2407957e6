"""Parity at the workloads' own sizes, in the launch configuration bench.py
times (spline solve, then binned RK2 steps with 8^3 bricks re-binned every
step), on outputs the FP64 oracle computes one by one.

Bars as in test_gpu_parity: interpolation max |du| <= 1e-5 rms(u); cell and
bin results bit-exact; one RK2 step <= dt * 1e-5 * rms(u) + 1e-14 in position;
gradients <= 1e-5 * 3 * (n/L) * max|c|.
"""
import json
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2005_13193_gb300 as ps
from paper_2005_13193_gb300 import synth

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi
DEV = "cuda"


def rel_err(gpu, ref):
    ref = np.asarray(ref)
    return np.abs(np.asarray(gpu, dtype=np.float64) - ref).max() / np.sqrt((ref ** 2).mean())


def test_tiny_config():
    # 32^3 FP64 field (k^-5/3, 1 <= |k| <= 10), 4096 particles, coefficients,
    # interpolation and one RK2 step with dt = 1e-3
    n, dt = 32, 1e-3
    field = synth.spectral_field(n, 10, seed=1000, device="cpu", dtype=torch.float64).numpy()
    pos = synth.uniform_particles(4096, seed=2000)
    cref = oracle.spline_coeffs(field)
    ref = oracle.interp(cref, pos)
    f = torch.from_numpy(field).to(DEV)
    for dtype, bound in ((torch.float32, 1e-5), (torch.float64, 5e-7)):
        sf = ps.SplineField.from_field(f, dtype)
        assert rel_err(sf.interp(torch.from_numpy(pos).to(DEV)).cpu().numpy(), ref) <= bound
    sf = ps.SplineField.from_field(f, torch.float32)
    tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=(8, 8, 8))
    tr.step(dt)
    new_ref, u1 = oracle.rk2_step(cref, pos, dt)
    ids = tr.ids.cpu().numpy()
    rms = np.sqrt((u1 ** 2).mean())
    assert np.abs(tr.pos.cpu().numpy() - new_ref[:, ids]).max() <= dt * 1e-5 * rms + 1e-14


def test_mid_config_full_size():
    # 512^3 FP32 (k^-5/3, 1 <= |k| <= 170), 16,777,216 particles, 10 RK2 steps
    # (dt = 1e-3) re-binned into 8^3 bricks every step.  After 9 steps the
    # bins, the velocities and the 10th step are checked particle by particle
    # on a seeded sample against the oracle started from the GPU's positions.
    N, NP, dt, brick = 512, 1 << 24, 1e-3, (8, 8, 8)
    free, _ = torch.cuda.mem_get_info()
    if free < 16e9:
        pytest.skip("needs 16 GB of free device memory")
    field = synth.spectral_field(N, 170, seed=1001, device=DEV, dtype=torch.float32)
    pos = torch.from_numpy(synth.uniform_particles(NP, seed=2001)).to(DEV)
    # the benchmark's storage: FP32 coefficients as interleaved nodes
    sf = ps.SplineField.from_field(field, ps.F32X4)
    tr = ps.Tracker(sf, pos, brick=brick)
    for _ in range(9):
        tr.step(dt)
    assert ps.ps_status_read(tr.status)[0] == 0
    x9 = tr.pos.cpu().numpy()
    ids9 = tr.ids.cpu().numpy()
    tr.step(dt)
    torch.cuda.synchronize()
    x10 = tr.pos.cpu().numpy()
    ids10 = tr.ids.cpu().numpy()
    u1 = tr.vel.cpu().numpy()
    offs = tr.offsets.cpu().numpy()
    # bins of x9 (the 10th step re-binned them): bit-exact
    _, off_ref, _ = oracle.bin_particles((N, N, N), brick, x9)
    np.testing.assert_array_equal(offs, off_ref)
    # oracle coefficients of the same FP32 field
    oracle.set_num_threads(0)
    cref = oracle.spline_coeffs(field.cpu().numpy().astype(np.float64))
    del field
    rng = np.random.default_rng(5)
    sample = rng.choice(NP, size=20000, replace=False)   # slots after step 10
    pid = ids10[sample]
    where9 = np.empty(NP, dtype=np.int64)
    where9[ids9] = np.arange(NP)
    xs9 = x9[:, where9[pid]]
    new_ref, u_ref = oracle.rk2_step(cref, xs9, dt)
    rms = np.sqrt((u_ref ** 2).mean())
    assert np.abs(u1[:, sample] - u_ref).max() <= 1e-5 * rms
    assert np.abs(x10[:, sample] - new_ref).max() <= dt * 1e-5 * rms + 1e-14


def test_diff_config_full_size():
    # 256^3 FP32 (k^-5/3, 1 <= |k| <= 85), 4,194,304 particles: forward
    # interpolation, the 9-component velocity-gradient tensor, and the
    # backward with respect to positions and to the field, against the oracle;
    # the gradient also against FP64 central differences (h = 1e-6) of the
    # oracle on 1024 particles.
    N, NP = 256, 1 << 22
    field = synth.spectral_field(N, 85, seed=1003, device=DEV, dtype=torch.float32)
    pos_h = synth.uniform_particles(NP, seed=2003)
    pos = torch.from_numpy(pos_h).to(DEV)
    sf = ps.SplineField.from_field(field, torch.float32)
    bins, pos_s = ps.bin_particles((N,) * 3, (8, 8, 8), pos, want_sorted=True)
    vel, grad = sf.interp(pos, grad=True, bins=bins)
    w = np.random.default_rng(6).standard_normal((3, NP)).astype(np.float32)
    g_pos = torch.empty_like(pos)
    g_field = torch.empty((3, N, N, N), dtype=torch.float32, device=DEV)
    ps.ps_interp_backward(sf.coef, sf.n, pos, torch.from_numpy(w).to(DEV), g_pos, g_field)
    torch.cuda.synchronize()
    oracle.set_num_threads(0)
    f64 = field.cpu().numpy().astype(np.float64)
    cref = oracle.spline_coeffs(f64)
    sample = np.random.default_rng(7).choice(NP, size=1024, replace=False)
    ps_ = pos_h[:, sample]
    v_ref, g_ref = oracle.interp(cref, ps_, grad=True)
    rms = np.sqrt((v_ref ** 2).mean())
    assert np.abs(vel.cpu().numpy()[:, sample] - v_ref).max() <= 1e-5 * rms
    gg = grad.cpu().numpy()[:, :, sample]
    cmax = np.abs(cref).max()
    tol = 1e-5 * 3 * (N / TWO_PI) * cmax
    assert np.abs(gg - g_ref).max() <= tol
    # FP64 central differences of the oracle, h = 1e-6
    for d in range(3):
        p1, p0 = ps_.copy(), ps_.copy()
        p1[d] += 1e-6
        p0[d] -= 1e-6
        fd = (oracle.interp(cref, p1) - oracle.interp(cref, p0)) / 2e-6
        assert np.abs(gg[:, d] - fd).max() <= tol + 1e-6 * np.abs(fd).max()
    # backward: positions on the sample, field everywhere
    gp_ref, _ = oracle.interp_backward(cref, ps_, w[:, sample].astype(np.float64),
                                       want_field=False)
    assert np.abs(g_pos.cpu().numpy()[:, sample] - gp_ref).max() <= 3 * tol * np.abs(w).max()
    _, gf_ref = oracle.interp_backward(cref, pos_h, w.astype(np.float64), want_pos=False)
    gf = g_field.cpu().numpy()
    assert np.abs(gf - gf_ref).max() <= 1e-5 * np.abs(gf_ref).max()


def test_precision_config_full_size():
    # 1536^3 FP32 field (k^-5/3, 1 <= |k| <= 512), 300,000,000 particles: one
    # coefficient solve, interpolation and one RK2 step (dt = 1e-3) with FP32,
    # BF16 and FP16 coefficients (BF16/FP16 with a power-of-two scale per
    # x-line), planar and as interleaved nodes (identical values, so identical
    # results).  FP32 is checked against the windowed FP64 oracle on 4096
    # particles with the bars above; BF16/FP16 against the FP32 result on a
    # seeded 1,000,000-particle subsample and against the oracle on the 4096,
    # at most 1e-2 (BF16) and 1e-3 (FP16) of the rms velocity, and within the
    # a-priori rounding bound 2^-8 max|c| (BF16), 2^-10 max|c| (FP16): the
    # basis weights are non-negative and sum to one.
    N, NP, dt, brick = 1536, 300_000_000, 1e-3, (8, 8, 8)
    free, _ = torch.cuda.mem_get_info()
    if free < 170e9:
        pytest.skip("needs 170 GB of free device memory")
    field = synth.spectral_field_planes(N, 512, seed=1002, device=DEV)
    pos_h = synth.uniform_particles(NP, seed=2002)
    pos = torch.from_numpy(pos_h).to(DEV)
    rng = np.random.default_rng(8)
    sub_h = np.sort(rng.choice(NP, size=1_000_000, replace=False))
    kpick = rng.choice(sub_h.size, size=4096, replace=False)
    sub = torch.from_numpy(sub_h).to(DEV)
    bins = ps.bin_particles((N,) * 3, brick, pos)
    got, cmax = {}, None
    for dtype in (torch.float32, torch.bfloat16, torch.float16, ps.F32X4, ps.BF16X4, ps.F16X4):
        sf = ps.SplineField.from_field(field, dtype)
        if dtype == torch.float32:
            cmax = max(float(sf.coef[c].abs().max()) for c in range(3))
        st = torch.zeros(4, dtype=torch.int32, device=DEV)
        vel = sf.interp(pos, bins=bins, status=st)
        u_sub = vel[:, sub].cpu().numpy()
        del vel
        tr = ps.Tracker(sf, pos.clone(), brick=brick, keep_velocity=False)
        tr.step(dt)
        where = torch.empty_like(tr.ids)
        where[tr.ids] = torch.arange(NP, dtype=torch.int64, device=DEV)
        x_sub = tr.pos[:, where[sub]].cpu().numpy()
        assert ps.ps_status_read(st)[0] == 0 and ps.ps_status_read(tr.status)[0] == 0
        got[dtype] = (u_sub, x_sub)
        del tr, where, sf
        torch.cuda.empty_cache()
    f_h = field.cpu().numpy()
    del field
    oracle.set_num_threads(0)
    xk = pos_h[:, sub_h[kpick]]
    u1 = oracle.interp_windowed(f_h, xk)
    # Heun step from the oracle's own predictor
    u2 = oracle.interp_windowed(f_h, xk + dt * u1)
    x1 = xk + 0.5 * dt * (u1 + u2)
    rms = np.sqrt((u1 ** 2).mean())
    # node storage holds the planar values: identical results
    for planar, node in ((torch.float32, ps.F32X4), (torch.bfloat16, ps.BF16X4),
                         (torch.float16, ps.F16X4)):
        assert np.array_equal(got[planar][0], got[node][0])
        assert np.array_equal(got[planar][1], got[node][1])
    u32, x32 = got[torch.float32]
    rms32 = np.sqrt((u32.astype(np.float64) ** 2).mean())
    report = {"rms_u": rms, "max_abs_c": cmax}
    for dtype, name, bar, ulp in ((torch.float32, "f32", 1e-5, 0.0),
                                  (torch.bfloat16, "bf16", 1e-2, 2.0 ** -8),
                                  (torch.float16, "f16", 1e-3, 2.0 ** -10)):
        u, x = got[dtype]
        e_ora = np.abs(u[:, kpick] - u1).max() / rms
        e_ora_rms = np.sqrt(((u[:, kpick] - u1) ** 2).mean()) / rms
        ex_ora = np.abs(x[:, kpick] - x1).max()
        report[name] = {"max_err_vs_oracle": e_ora, "rms_err_vs_oracle": e_ora_rms,
                        "pos_err_vs_oracle": ex_ora}
        assert e_ora <= bar
        assert ex_ora <= dt * bar * rms + 1e-14
        if dtype != torch.float32:
            d = np.abs(u.astype(np.float64) - u32)
            report[name]["max_err_vs_f32_1M"] = d.max() / rms32
            report[name]["rms_err_vs_f32_1M"] = np.sqrt((d ** 2).mean()) / rms32
            assert d.max() <= ulp * cmax + 1e-5 * rms32
            assert d.max() / rms32 + report["f32"]["max_err_vs_oracle"] <= bar
    print("PRECISION " + json.dumps(report))
