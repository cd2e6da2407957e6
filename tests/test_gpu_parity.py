"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic):
  * coefficients (FP32): each pencil pass is a pair of first-order recursions
    with |z| = 0.268 and gain 1.61; rounding grows by a few ulp per pass, so
    |c_gpu - c_ora| <= 2e-6 * max|field| (about 30 ulp of the largest value).
  * interpolation (FP32): max |u_gpu - u_ora| <= 1e-5 * rms(u_ora) -- the bar
    the method is held to.  64 non-negative weights summing to 1 bound the
    accumulation error by ~64 ulp of max|c|.
  * gradients: the derivative weights sum in absolute value to < 3 per axis,
    times n/L: |g_gpu - g_ora| <= 1e-5 * 3 * (n/L) * max|c|.
  * cell indices, bins, offsets, permutations: bit-exact / set-exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2005_13193_gb300 as ps
from paper_2005_13193_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
TWO_PI = 2 * math.pi


def rel_err(gpu, ref):
    ref = np.asarray(ref)
    rms = np.sqrt((ref ** 2).mean())
    return np.abs(np.asarray(gpu, dtype=np.float64) - ref).max() / rms


def coef_tol(field):
    return 2e-6 * float(np.abs(field).max())


# ------------------------------------------------------------------ solve ----

@pytest.mark.parametrize("n", [(3, 3, 3), (4, 5, 6), (12, 10, 9), (32, 32, 32), (37, 33, 40),
                               (100, 7, 65)])
def test_spline_coeffs_f32(n):
    field = synth.random_field(n, ncomp=3, seed=sum(n))
    ref = oracle.spline_coeffs(field)
    f = torch.from_numpy(field.astype(np.float32)).to(DEV)
    sf = ps.SplineField.from_field(f, torch.float32)
    ref32 = oracle.spline_coeffs(field.astype(np.float32).astype(np.float64))
    got = sf.padded().cpu().numpy()
    assert got.shape == ref.shape
    assert np.abs(got - ref32).max() <= coef_tol(field)


def test_spline_coeffs_f64_field_and_coef():
    n = (24, 20, 18)
    field = synth.random_field(n, ncomp=3, seed=5)
    ref = oracle.spline_coeffs(field)
    f = torch.from_numpy(field).to(DEV)
    c64 = ps.SplineField.from_field(f, torch.float64).padded().cpu().numpy()
    assert np.abs(c64 - ref).max() <= 1e-13 * np.abs(field).max()
    c32 = ps.SplineField.from_field(f, torch.float32).padded().cpu().numpy()
    assert np.abs(c32 - ref).max() <= coef_tol(field)


@pytest.mark.parametrize("n", [64, 200, 512, 700, 1100, 1536])
def test_spline_coeffs_long_pencils(n):
    # pencil lengths that select every chunking configuration of the passes
    dims = (n, 5, 4) if n > 600 else (n, 9, 7)
    for perm in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        shape = tuple(dims[p] for p in perm)
        field = synth.random_field(shape, ncomp=1, seed=n + perm[0])
        f = torch.from_numpy(field.astype(np.float32)).to(DEV)
        got = ps.SplineField.from_field(f, torch.float32).padded().cpu().numpy()
        ref = oracle.spline_coeffs(field.astype(np.float32).astype(np.float64))
        assert np.abs(got - ref).max() <= coef_tol(field), shape


@pytest.mark.parametrize("n", [(128, 40, 50), (256, 33, 47), (128, 32, 700), (512, 48, 32),
                               (128, 700, 34), (36, 40, 50), (100, 36, 33), (1028, 32, 33)])
def test_streamed_solve_matches_oracle(n):
    # The two-pass solve (x-y pass, then the z pass into the padded layout's
    # interior, then its periodic images) streams y and z in 16-line chunks:
    # ragged last chunks, every row width it takes (128, 256, 512), long
    # pencils; other row widths (a multiple of 4) stream y and z and keep
    # the x pass.  It meets the bar against the oracle, planar and node
    # storage hold the same bits, and the line streams' columns per block and
    # the x-y pass's stages change no bit.
    field = synth.random_field(n, ncomp=3, seed=sum(n) + 7)
    ref32 = oracle.spline_coeffs(field.astype(np.float32).astype(np.float64))
    f = torch.from_numpy(field.astype(np.float32)).to(DEV)
    keys = ("solve_stream", "solve_zt", "solve_stages")
    old = {k: ps.ps_tune_get(k) for k in keys}
    try:
        ps.ps_tune_set("solve_stream", 1)
        s32 = ps.SplineField.from_field(f, torch.float32)
        p32 = s32.padded()
        assert np.abs(p32.cpu().numpy() - ref32).max() <= coef_tol(field)
        assert torch.count_nonzero(s32.coef[..., n[0] + 3:]) == 0  # the row tail
        p4 = ps.SplineField.from_field(f, ps.F32X4)
        assert torch.equal(p4.padded(), p32)
        assert torch.count_nonzero(p4.coef[..., 3]) == 0
        for zt, stages in ((16, 2), (64, 4), (256, 3)):
            ps.ps_tune_set("solve_zt", zt)
            ps.ps_tune_set("solve_stages", stages)
            assert torch.equal(ps.SplineField.from_field(f, torch.float32).padded(), p32)
            assert torch.equal(ps.SplineField.from_field(f, ps.F32X4).padded(), p32)
        # the strided three-pass solve agrees: each is within the bar of the
        # oracle, so the two are within twice it
        ps.ps_tune_set("solve_stream", 0)
        p3 = ps.SplineField.from_field(f, torch.float32).padded()
        assert (p3 - p32).abs().max().item() <= 2 * coef_tol(field)
    finally:
        for k, v in old.items():
            ps.ps_tune_set(k, v)


# ---------------------------------------------------------------- binning ----

@pytest.mark.parametrize("n,brick", [((32, 32, 32), (8, 8, 8)), ((37, 20, 9), (8, 4, 5)),
                                     ((16, 16, 16), (1, 1, 1)), ((64, 48, 40), (16, 16, 16)),
                                     ((10, 10, 10), (3, 7, 10))])
def test_binning_bit_exact(n, brick):
    L = (TWO_PI, 3.5, 1.25)
    pos = synth.uniform_particles(5000, seed=7)
    pos = pos / TWO_PI * np.array(L)[:, None] * 2.2 - np.array(L)[:, None] * 0.6
    b_ora, off_ora, perm_ora = oracle.bin_particles(n, brick, pos, L=L)
    pg = torch.from_numpy(pos).to(DEV)
    bins, sorted_pos = ps.bin_particles(n, brick, pg, L=L, want_sorted=True)
    np.testing.assert_array_equal(bins.bin_of.cpu().numpy(), b_ora)
    off = bins.offsets.cpu().numpy()
    np.testing.assert_array_equal(off, off_ora)
    perm = bins.perm.cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(5000))
    for b in range(len(off) - 1):
        assert set(perm[off[b]:off[b + 1]]) == set(perm_ora[off[b]:off[b + 1]])
    np.testing.assert_array_equal(sorted_pos.cpu().numpy(), pos[:, perm])


def test_binning_adversarial_positions():
    # exact nodes, signed zeros, fractions that round to 1, far shadow images,
    # values just below/above faces: the integer floor must match FP64 floor.
    n, brick = (64, 48, 40), (8, 8, 8)
    L = (TWO_PI, 3.0, 1.0)
    rng = np.random.default_rng(3)
    cols = []
    for d in range(3):
        h = L[d] / n[d]
        nodes = np.arange(-3 * n[d], 4 * n[d]) * h
        v = np.concatenate([nodes, nodes + 1e-17, nodes - 1e-17, np.nextafter(nodes, np.inf),
                            np.nextafter(nodes, -np.inf), [0.0, -0.0, -1e-300, 1e-300, -5e-324],
                            rng.uniform(-1e6, 1e6, 2000), rng.uniform(-1e-9, 1e-9, 500)])
        cols.append(v)
    m = max(len(c) for c in cols)
    pos = np.stack([np.resize(c, m) for c in cols])
    for d in range(3):
        rng.shuffle(pos[d])
    b_ora, off_ora, _ = oracle.bin_particles(n, brick, pos, L=L)
    bins = ps.bin_particles(n, brick, torch.from_numpy(pos).to(DEV), L=L)
    np.testing.assert_array_equal(bins.bin_of.cpu().numpy(), b_ora)
    np.testing.assert_array_equal(bins.offsets.cpu().numpy(), off_ora)


def test_binning_empty_and_single():
    n, brick = (16, 16, 16), (8, 8, 8)
    pg = torch.empty((3, 0), dtype=torch.float64, device=DEV)
    bins = ps.bin_particles(n, brick, pg)
    assert bins.offsets.cpu().tolist() == [0] * 9
    pos = np.array([[1.0], [2.0], [6.0]])
    bins = ps.bin_particles(n, brick, torch.from_numpy(pos).to(DEV))
    _, off_ora, _ = oracle.bin_particles(n, brick, pos)
    np.testing.assert_array_equal(bins.offsets.cpu().numpy(), off_ora)


# ----------------------------------------------------------------- interp ----

@pytest.fixture
def brick_kernel():
    old = ps.ps_tune_get("brick_kernel")
    yield
    ps.ps_tune_set("brick_kernel", old)



def _case(n, np_, seed, L=(TWO_PI,) * 3, ncomp=3, spread=1.0):
    field = synth.random_field(n, ncomp=ncomp, seed=seed).astype(np.float32)
    pos = synth.uniform_particles(np_, seed=seed + 1)
    pos = pos / TWO_PI * np.array(L)[:, None] * spread
    coef_ref = oracle.spline_coeffs(field.astype(np.float64))
    return field, pos, coef_ref


@pytest.mark.parametrize("n,np_", [((32, 32, 32), 4096), ((37, 21, 10), 3001), ((3, 4, 5), 257),
                                   ((64, 64, 64), 1)])
def test_interp_direct(n, np_):
    L = (TWO_PI, 4.0, 2.5)
    field, pos, cref = _case(n, np_, seed=11, L=L, spread=1.7)
    ref = oracle.interp(cref, pos, L=L)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32, L=L)
    vel = sf.interp(torch.from_numpy(pos).to(DEV)).cpu().numpy()
    assert rel_err(vel, ref) <= 1e-5


@pytest.mark.parametrize("kernel", [0, 2, 5])
@pytest.mark.parametrize("brick", [(8, 8, 8), (4, 4, 4), (16, 8, 4), (5, 7, 3), (1, 1, 1)])
def test_interp_staged_sorted_and_perm(brick, kernel, brick_kernel):
    ps.ps_tune_set("brick_kernel", kernel)
    n = (40, 36, 33)
    field, pos, cref = _case(n, 20000, seed=21, spread=2.0)
    ref = oracle.interp(cref, pos)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    pg = torch.from_numpy(pos).to(DEV)
    bins, sorted_pos = ps.bin_particles(n, brick, pg, want_sorted=True)
    # via the permutation, outputs in the original order
    vel = sf.interp(pg, bins=bins).cpu().numpy()
    assert rel_err(vel, ref) <= 1e-5
    # physically sorted storage
    bins_sorted = ps.Bins(bins.brick, bins.offsets, bins.bin_of, None)
    vel_s = sf.interp(sorted_pos, bins=bins_sorted).cpu().numpy()
    perm = bins.perm.cpu().numpy()
    assert rel_err(vel_s, ref[:, perm]) <= 1e-5


def abs_err(gpu, ref):
    return np.abs(np.asarray(gpu, dtype=np.float64) - np.asarray(ref)).max()


@pytest.mark.parametrize("kernel", [-1, 0, 2, 5])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_brick_kernels_on_tiling_grids(kernel, dtype, brick_kernel):
    # Grids divisible by the brick: 16-byte halo rows, both brick kernels.
    # Bounds: FP32 1e-5 of rms.  BF16 stores c/s with s a power of two, so each
    # coefficient has relative error <= 2^-9; the basis weights are
    # non-negative and sum to one, so |du| <= 2^-9 max|c| (2^-8 with margin).
    # On this white-noise field max|c| is ~30x rms, hence an absolute bound.
    ps.ps_tune_set("brick_kernel", kernel)
    n = (48, 40, 32)
    field, pos, cref = _case(n, 30000, seed=27, spread=1.4)
    ref_v, ref_g = oracle.interp(cref, pos, grad=True)
    rms = np.sqrt((ref_v ** 2).mean())
    tol_u = 1e-5 * rms if dtype == torch.float32 else 2.0 ** -8 * np.abs(cref).max()
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), dtype)
    pg = torch.from_numpy(pos).to(DEV)
    bins, sorted_pos = ps.bin_particles(n, (8, 8, 8), pg, want_sorted=True)
    perm = bins.perm.cpu().numpy()
    # positions in bin order, and through the permutation
    v_s = sf.interp(sorted_pos, bins=ps.Bins(bins.brick, bins.offsets, bins.bin_of, None))
    assert abs_err(v_s.cpu().numpy(), ref_v[:, perm]) <= tol_u
    vel, grad = sf.interp(pg, grad=True, bins=bins)
    assert abs_err(vel.cpu().numpy(), ref_v) <= tol_u
    if dtype == torch.float32:
        cmax = np.abs(cref).max()
        for d in range(3):
            tol = 1e-5 * 3 * (n[d] / TWO_PI) * cmax
            assert np.abs(grad[:, d].cpu().numpy() - ref_g[:, d]).max() <= tol
    # fused RK2 step on the sorted positions
    dt = 1e-2
    new_ref, u1_ref = oracle.rk2_step(cref, pos[:, perm], dt)
    tr = ps.Tracker(sf, sorted_pos.clone(), brick=(8, 8, 8))
    tr.step(dt)
    ids = tr.ids.cpu().numpy()
    assert np.abs(tr.pos.cpu().numpy() - new_ref[:, ids]).max() <= dt * tol_u + 1e-14


def test_interp_stale_bins_fall_back_correctly():
    # bins computed for other positions: every particle takes the global path
    n = (32, 32, 32)
    field, pos, cref = _case(n, 3000, seed=31)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    pg = torch.from_numpy(pos).to(DEV)
    bins = ps.bin_particles(n, (8, 8, 8), pg)
    moved = (pos + 1.3) % TWO_PI
    vel = sf.interp(torch.from_numpy(moved).to(DEV), bins=bins).cpu().numpy()
    assert rel_err(vel, oracle.interp(cref, moved)) <= 1e-5


def test_interp_scalar_component():
    n = (20, 24, 28)
    field, pos, cref = _case(n, 2000, seed=41, ncomp=1)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    pg = torch.from_numpy(pos).to(DEV)
    ref = oracle.interp(cref, pos)
    assert rel_err(sf.interp(pg).cpu().numpy(), ref) <= 1e-5
    bins = ps.bin_particles(n, 8, pg)
    assert rel_err(sf.interp(pg, bins=bins).cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("staged", [False, True])
def test_gradient_tensor(staged):
    n = (32, 28, 24)
    L = (TWO_PI, 5.0, 3.0)
    field, pos, cref = _case(n, 4096, seed=51, L=L)
    ref_v, ref_g = oracle.interp(cref, pos, L=L, grad=True)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32, L=L)
    pg = torch.from_numpy(pos).to(DEV)
    bins = ps.bin_particles(n, 8, pg, L=L) if staged else None
    vel, grad = sf.interp(pg, grad=True, bins=bins)
    assert rel_err(vel.cpu().numpy(), ref_v) <= 1e-5
    cmax = np.abs(cref).max()
    for d in range(3):
        tol = 1e-5 * 3 * (n[d] / L[d]) * cmax
        assert np.abs(grad[:, d].cpu().numpy() - ref_g[:, d]).max() <= tol


def test_f64_coefficients_tight():
    n = (16, 18, 20)
    field = synth.random_field(n, ncomp=3, seed=61)
    pos = synth.uniform_particles(1000, seed=62) * 1.3
    ref = oracle.interp(oracle.spline_coeffs(field), pos)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float64)
    vel = sf.interp(torch.from_numpy(pos).to(DEV)).cpu().numpy()
    # FP64 coefficients, FP64 accumulation, FP32 output rounding only
    assert rel_err(vel, ref) <= 5e-7


@pytest.mark.parametrize("dtype,bound", [(torch.bfloat16, 1e-2), (torch.float16, 1e-3)])
def test_low_precision_coefficients(dtype, bound):
    n = (48, 48, 48)
    field = synth.spectral_field(48, kmax=16, seed=71, device="cpu", dtype=torch.float64).numpy()
    field32 = field.astype(np.float32)
    pos = synth.uniform_particles(8192, seed=72)
    ref = oracle.interp(oracle.spline_coeffs(field32.astype(np.float64)), pos)
    sf = ps.SplineField.from_field(torch.from_numpy(field32).to(DEV), dtype)
    assert sf.scale is not None
    sc = sf.scale.cpu().numpy()
    assert np.all(np.log2(sc) == np.round(np.log2(sc)))  # powers of two
    pg = torch.from_numpy(pos).to(DEV)
    err = rel_err(sf.interp(pg).cpu().numpy(), ref)
    assert err <= bound, err
    bins = ps.bin_particles(n, 8, pg)
    assert rel_err(sf.interp(pg, bins=bins).cpu().numpy(), ref) <= bound


@pytest.mark.parametrize("dtype,ulp", [(torch.bfloat16, 2.0 ** -8), (torch.float16, 2.0 ** -11)])
@pytest.mark.parametrize("n", [(1100, 6, 5), (1028, 32, 33)])
def test_low_precision_wide_rows(dtype, ulp, n):
    # rows over 512 values take W warps per x-line (carries and the line's
    # maximum through shared memory); (1028, 32, 33) also streams y and z.
    # Each stored value is its FP32 coefficient rounded to 16 bits after
    # division by the line's power-of-two scale: within half an ulp of the
    # scaled value, plus the FP32 solve's bar.
    field = synth.random_field(n, ncomp=3, seed=sum(n) + 9)
    ref = oracle.spline_coeffs(field.astype(np.float32).astype(np.float64))
    f = torch.from_numpy(field.astype(np.float32)).to(DEV)
    sf = ps.SplineField.from_field(f, dtype)
    sc = sf.scale.cpu().numpy()  # [ncomp][nz+3][ny+3]
    assert np.all(np.log2(sc) == np.round(np.log2(sc)))
    got = sf.padded().float().cpu().numpy() * sc[..., None]
    # a line's scale is at least its largest value: the rounding is at most
    # half an ulp of the scale
    tol = 0.5 * ulp * sc[..., None] + coef_tol(field)
    assert np.all(np.abs(got - ref) <= tol)
    # the per-line scale is the least power of two at or above the line's
    # largest coefficient
    mx = np.abs(ref[..., : n[0] + 3]).max(axis=-1)
    assert np.all(sc >= mx * (1 - 1e-6)) and np.all(sc < 2 * mx * (1 + 1e-6))


def test_planar_solve_without_workspace_matches():
    # planar FP32 without a workspace runs the three passes in place; with one
    # it streams; each is within the bar of the oracle, so within twice it of
    # the other
    n = (96, 40, 36)
    field = synth.random_field(n, ncomp=3, seed=191)
    f = torch.from_numpy(field.astype(np.float32)).to(DEV)
    with_ws = ps.SplineField.from_field(f, torch.float32).padded()
    coef = torch.empty_like(ps.SplineField.from_field(f, torch.float32).coef)
    ps.ps_spline_coeffs(f, coef, None, None)
    no_ws = coef[..., : n[0] + 3]
    ref = oracle.spline_coeffs(field.astype(np.float32).astype(np.float64))
    assert np.abs(no_ws.cpu().numpy() - ref).max() <= coef_tol(field)
    assert np.abs(with_ws.cpu().numpy() - ref).max() <= coef_tol(field)
    assert (no_ws - with_ws).abs().max().item() <= 2 * coef_tol(field)


def test_nonfinite_position_flagged():
    n = (16, 16, 16)
    field, pos, cref = _case(n, 100, seed=81)
    pos[0, 7] = np.nan
    pos[2, 40] = np.inf
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    st = torch.zeros(4, dtype=torch.int32, device=DEV)
    pg = torch.from_numpy(pos).to(DEV)
    vel = sf.interp(pg, status=st).cpu().numpy()
    code, lo, hi, count = ps.ps_status_read(st)
    assert code == ps._abi.PS_DEV_NONFINITE_POS and count == 2 and lo in (7, 40)
    assert np.isnan(vel[:, [7, 40]]).all()
    good = np.ones(100, bool)
    good[[7, 40]] = False
    ref = oracle.interp(cref, pos[:, good])
    assert rel_err(vel[:, good], ref) <= 1e-5
    # binning puts them in bin 0 and flags them too
    st.zero_()
    bins = ps.bin_particles(n, 8, pg, status=st)
    assert ps.ps_status_read(st)[0] == ps._abi.PS_DEV_NONFINITE_POS
    assert set(bins.bin_of.cpu().numpy()[[7, 40]]) == {0}


# --------------------------------------------------------------- backward ----

def test_backward_positions_and_field():
    n = (20, 18, 16)
    field, pos, cref = _case(n, 3000, seed=91)
    w = np.random.default_rng(92).standard_normal((3, 3000)).astype(np.float32)
    gp_ref, gf_ref = oracle.interp_backward(cref, pos, w.astype(np.float64))
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    pg = torch.from_numpy(pos).to(DEV)
    g_pos = torch.empty_like(pg)
    g_field = torch.empty((3,) + tuple(reversed(n)), dtype=torch.float32, device=DEV)
    ps.ps_interp_backward(sf.coef, sf.n, pg, torch.from_numpy(w).to(DEV), g_pos, g_field)
    gp = g_pos.cpu().numpy()
    scale_p = 3 * (n[0] / TWO_PI) * np.abs(cref).max() * np.abs(w).max() * 3
    assert np.abs(gp - gp_ref).max() <= 1e-5 * scale_p
    gf = g_field.cpu().numpy()
    # scatter of 3000 * 64 weights with FP32 atomics, then three FP32 passes
    assert np.abs(gf - gf_ref).max() <= 1e-5 * np.abs(gf_ref).max() + 1e-6


def test_autograd_matches_oracle_and_fd():
    n = (16, 16, 16)
    field, pos, cref = _case(n, 512, seed=93)
    w = np.random.default_rng(94).standard_normal((3, 512))
    f = torch.from_numpy(field).to(DEV).requires_grad_(True)
    p = torch.from_numpy(pos).to(DEV).requires_grad_(True)
    vel = ps.interp_autograd(p, f)
    loss = (vel.double() * torch.from_numpy(w).to(DEV)).sum()
    loss.backward()
    gp_ref, gf_ref = oracle.interp_backward(cref, pos, w)
    assert np.abs(p.grad.cpu().numpy() - gp_ref).max() <= 1e-4 * np.abs(gp_ref).max()
    assert np.abs(f.grad.cpu().numpy() - gf_ref).max() <= 1e-5 * np.abs(gf_ref).max() + 1e-6


# -------------------------------------------------------------------- RK2 ----

@pytest.mark.parametrize("brick", [None, (8, 8, 8), (4, 4, 4)])
def test_rk2_step(brick):
    n = (32, 32, 32)
    field, pos, cref = _case(n, 8000, seed=101)
    dt = 1e-2  # large enough that x* leaves the brick halo for some particles
    new_ref, u1_ref = oracle.rk2_step(cref, pos, dt)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick)
    tr.step(dt)
    ids = tr.ids.cpu().numpy()
    assert np.array_equal(np.sort(ids), np.arange(8000))
    rms = np.sqrt((u1_ref ** 2).mean())
    got = tr.pos.cpu().numpy()
    assert np.abs(got - new_ref[:, ids]).max() <= dt * 1e-5 * rms + 1e-14
    assert rel_err(tr.vel.cpu().numpy(), u1_ref[:, ids]) <= 1e-5
    if brick is not None:
        # the new storage order is the bin order of x^n
        b_ora, off_ora, _ = oracle.bin_particles(n, brick, pos)
        np.testing.assert_array_equal(tr.offsets.cpu().numpy(), off_ora)
        assert np.all(np.diff(b_ora[ids]) >= 0)


def test_rk2_multi_step_and_time_dependent():
    n = (24, 24, 24)
    field, pos, cref = _case(n, 4000, seed=111)
    field2 = synth.random_field(n, ncomp=3, seed=112).astype(np.float32)
    cref2 = oracle.spline_coeffs(field2.astype(np.float64))
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    sf2 = ps.SplineField.from_field(torch.from_numpy(field2).to(DEV), torch.float32)
    tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=(8, 8, 8))
    ref = pos.copy()
    dt = 5e-3
    for step in range(4):
        two = step % 2 == 1
        tr.step(dt, field_np1=sf2 if two else None)
        ref, _ = oracle.rk2_step(cref, ref, dt, coef_np1=cref2 if two else None)
    ids = tr.ids.cpu().numpy()
    assert np.abs(tr.pos.cpu().numpy() - ref[:, ids]).max() <= 4 * dt * 3e-5 * 3 + 1e-13


@pytest.mark.parametrize("kernel", [0, 2, 5])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_rk2_every_autotune_candidate(kernel, dtype, brick_kernel):
    # every brick shape the autotuner may pick, with every brick kernel, on a
    # grid all of them tile (so the 16-byte staging path is taken where the
    # shape allows it) and on a ragged one
    from paper_2005_13193_gb300 import autotune
    ps.ps_tune_set("brick_kernel", kernel)
    for n in ((64, 32, 48), (37, 21, 26)):
        field, pos, cref = _case(n, 20000, seed=121, spread=1.3)
        dt = 1e-2
        new_ref, u1_ref = oracle.rk2_step(cref, pos, dt)
        rms = np.sqrt((u1_ref ** 2).mean())
        tol_u = 1e-5 * rms if dtype == torch.float32 else 2.0 ** -8 * np.abs(cref).max()
        sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), dtype)
        for brick in autotune.CANDIDATES:
            tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick)
            tr.step(dt)
            assert ps.ps_status_read(tr.status)[0] == 0
            ids = tr.ids.cpu().numpy()
            assert np.abs(tr.vel.cpu().numpy() - u1_ref[:, ids]).max() <= tol_u, brick
            assert np.abs(tr.pos.cpu().numpy() - new_ref[:, ids]).max() <= dt * tol_u + 1e-14


@pytest.mark.parametrize("min_stage", [0, 8, 1 << 20])
def test_sparse_brick_knob(min_stage):
    # bricks below the threshold gather from global memory instead of the
    # staged halo; results stay within the same bars either way
    old = ps.ps_tune_get("brick_min_stage")
    try:
        ps.ps_tune_set("brick_min_stage", min_stage)
        n = (64, 32, 40)
        field, pos, cref = _case(n, 6000, seed=131, spread=1.2)  # ~3 per 8^3 brick
        ref = oracle.interp(cref, pos)
        sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
        pg = torch.from_numpy(pos).to(DEV)
        bins = ps.bin_particles(n, (8, 8, 8), pg)
        assert rel_err(sf.interp(pg, bins=bins).cpu().numpy(), ref) <= 1e-5
        dt = 1e-2
        new_ref, u1_ref = oracle.rk2_step(cref, pos, dt)
        rms = np.sqrt((u1_ref ** 2).mean())
        tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=(8, 8, 8))
        tr.step(dt)
        ids = tr.ids.cpu().numpy()
        assert np.abs(tr.pos.cpu().numpy() - new_ref[:, ids]).max() <= dt * 1e-5 * rms + 1e-14
    finally:
        ps.ps_tune_set("brick_min_stage", old)


@pytest.mark.parametrize("n,brick", [((32, 32, 32), (8, 8, 8)), ((40, 24, 16), (8, 8, 8)),
                                     ((37, 21, 10), (8, 4, 5)), ((64, 48, 40), (16, 8, 4))])
def test_node4_storage_matches_planar(n, brick):
    # Interleaved (u, v, w, 0) nodes hold the very values of the planar FP32
    # coefficients (same passes, same arithmetic), and every kernel reads the
    # same values from them: all results must agree bit for bit.
    field, pos, cref = _case(n, 20000, seed=141, spread=1.3)
    f = torch.from_numpy(field).to(DEV)
    p32 = ps.SplineField.from_field(f, torch.float32)
    p4 = ps.SplineField.from_field(f, ps.F32X4)
    assert p4.coef.shape == (n[2] + 3, n[1] + 3, n[0] + 3, 4)
    assert torch.equal(p4.padded(), p32.padded())
    assert torch.count_nonzero(p4.coef[..., 3]) == 0
    pg = torch.from_numpy(pos).to(DEV)
    # direct gathers, values and gradients
    for grad in (False, True):
        a = p32.interp(pg, grad=grad)
        b = p4.interp(pg, grad=grad)
        for x, y in zip(a if grad else (a,), b if grad else (b,)):
            assert torch.equal(x, y)
    # staged gathers, every brick kernel
    bins, sorted_pos = ps.bin_particles(n, brick, pg, want_sorted=True)
    old = ps.ps_tune_get("brick_kernel")
    try:
        for k in (0, 2, 5):
            ps.ps_tune_set("brick_kernel", k)
            assert torch.equal(p32.interp(pg, bins=bins), p4.interp(pg, bins=bins))
            va, ga = p32.interp(pg, grad=True, bins=bins)
            vb, gb = p4.interp(pg, grad=True, bins=bins)
            assert torch.equal(va, vb) and torch.equal(ga, gb)
            outs = []
            for sf in (p32, p4):
                tr = ps.Tracker(sf, sorted_pos.clone(), brick=brick)
                tr.step(1e-2)
                # by particle label: the order inside a bin is unspecified
                lab = torch.empty_like(tr.ids)
                lab[tr.ids] = torch.arange(tr.ids.numel(), device=DEV)
                outs.append((tr.pos[:, lab], tr.vel[:, lab]))
            assert all(torch.equal(x, y) for x, y in zip(*outs))
    finally:
        ps.ps_tune_set("brick_kernel", old)
    # unbinned Heun step and the adjoint with respect to positions
    t32 = ps.Tracker(p32, pg.clone(), brick=None)
    t4 = ps.Tracker(p4, pg.clone(), brick=None)
    t32.step(1e-2)
    t4.step(1e-2)
    assert torch.equal(t32.pos, t4.pos)
    w = torch.randn((3, pg.shape[1]), device=DEV, generator=torch.Generator(DEV).manual_seed(3))
    g32, g4 = torch.empty_like(pg), torch.empty_like(pg)
    ps.ps_interp_backward(p32.coef, n, pg, w, g_pos=g32)
    ps.ps_interp_backward(p4.coef, n, pg, w, g_pos=g4)
    assert torch.equal(g32, g4)
    # and against the oracle, as for the planar form
    assert rel_err(p4.interp(pg).cpu().numpy(), oracle.interp(cref, pos)) <= 1e-5


def test_node4_tensor_copy_matches_loads():
    # the halo by tensor copy and by plain loads holds the same values
    n = (64, 32, 48)
    field, pos, cref = _case(n, 30000, seed=151, spread=1.1)
    p4 = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), ps.F32X4)
    pg = torch.from_numpy(pos).to(DEV)
    bins = ps.bin_particles(n, (8, 8, 8), pg)
    old = ps.ps_tune_get("node_tma")
    try:
        outs = []
        for on in (1, 0):
            ps.ps_tune_set("node_tma", on)
            st = torch.zeros(4, dtype=torch.int32, device=DEV)
            outs.append(p4.interp(pg, grad=True, bins=bins, status=st))
            assert ps.ps_status_read(st)[0] == 0
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    finally:
        ps.ps_tune_set("node_tma", old)
    assert rel_err(outs[0][0].cpu().numpy(), oracle.interp(cref, pos)) <= 1e-5


@pytest.mark.parametrize("kernel", [0, 5])
def test_halo_wait_timeout_reads_global_memory(kernel, brick_kernel):
    # The bounded wait for a brick's halo copy must end without trapping and
    # leave correct results.  The test knob "wait_probe" makes every staged
    # brick wait, after its copy has landed, on a barrier that nothing
    # completes, bounded by that many clocks: every wait gives up, the status
    # word reads PS_DEV_TIMEOUT and the brick's particles take the global
    # memory gathers, so velocities, gradients and the Heun step still match
    # the oracle at the usual bars.
    ps.ps_tune_set("brick_kernel", kernel)
    n = (32, 24, 40)
    field, pos, cref = _case(n, 12000, seed=191, spread=1.2)
    p4 = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), ps.F32X4)
    pg = torch.from_numpy(pos).to(DEV)
    bins = ps.bin_particles(n, (8, 8, 8), pg)
    ref_v, ref_g = oracle.interp(cref, pos, grad=True)
    rms = np.sqrt((ref_v ** 2).mean())
    old = ps.ps_tune_get("wait_probe")
    try:
        ps.ps_tune_set("wait_probe", 20000)
        for grad in (False, True):
            st = torch.zeros(4, dtype=torch.int32, device=DEV)
            out = p4.interp(pg, grad=grad, bins=bins, status=st)
            code, _, _, count = ps.ps_status_read(st)
            assert code == ps._abi.PS_DEV_TIMEOUT and count > 0
            vel = (out[0] if grad else out).cpu().numpy()
            assert abs_err(vel, ref_v) <= 1e-5 * rms
            if grad:
                cmax = np.abs(cref).max()
                for d in range(3):
                    tol = 1e-5 * 3 * (n[d] / TWO_PI) * cmax
                    assert np.abs(out[1][:, d].cpu().numpy() - ref_g[:, d]).max() <= tol
        dt = 1e-2
        new_ref, u1_ref = oracle.rk2_step(cref, pos, dt)
        tr = ps.Tracker(p4, pg.clone(), brick=(8, 8, 8))
        tr.step(dt)
        code = ps.ps_status_read(tr.status)[0]
        assert code == ps._abi.PS_DEV_TIMEOUT
        ids = tr.ids.cpu().numpy()
        assert np.abs(tr.pos.cpu().numpy() - new_ref[:, ids]).max() <= dt * 1e-5 * rms + 1e-14
    finally:
        ps.ps_tune_set("wait_probe", old)
    # the knob off: no timeout, same results
    st = torch.zeros(4, dtype=torch.int32, device=DEV)
    vel = p4.interp(pg, bins=bins, status=st)
    assert ps.ps_status_read(st)[0] == 0
    assert abs_err(vel.cpu().numpy(), ref_v) <= 1e-5 * rms


@pytest.mark.parametrize("planar,node", [(torch.bfloat16, "bf16x4"), (torch.float16, "f16x4")])
@pytest.mark.parametrize("n", [(64, 32, 48), (37, 21, 10)])
@pytest.mark.parametrize("kernel", [0, 5])
def test_node16_storage_matches_planar(planar, node, n, kernel, brick_kernel):
    # 16-bit nodes hold the planar 16-bit values and per-line scales: every
    # path (direct, staged by tensor copy or by loads, Heun steps) agrees with
    # the planar form bit for bit, and both stay within the rounding bound.
    # Brick kernel 5 keeps the nodes 16-bit in shared memory and applies each
    # row's power-of-two scale as it widens them (exact), so it too agrees
    # with the planar form, whose halo holds the widened, scaled values.
    ps.ps_tune_set("brick_kernel", kernel)
    field, pos, cref = _case(n, 20000, seed=161, spread=1.2)
    f = torch.from_numpy(field).to(DEV)
    pp = ps.SplineField.from_field(f, planar)
    pn = ps.SplineField.from_field(f, node)
    assert pn.coef.dtype == planar and pn.coef.shape[-1] == 4
    assert torch.equal(pn.padded(), pp.padded())
    assert torch.equal(pn.scale[..., :3].permute(2, 0, 1), pp.scale)
    assert torch.count_nonzero(pn.coef[..., 3].float()) == 0
    pg = torch.from_numpy(pos).to(DEV)
    va, ga = pp.interp(pg, grad=True)
    vb, gb = pn.interp(pg, grad=True)
    assert torch.equal(va, vb) and torch.equal(ga, gb)
    bins, sorted_pos = ps.bin_particles(n, (8, 8, 8), pg, want_sorted=True)
    old = ps.ps_tune_get("node_tma")
    try:
        for on in (1, 0):
            ps.ps_tune_set("node_tma", on)
            st = torch.zeros(4, dtype=torch.int32, device=DEV)
            assert torch.equal(pp.interp(pg, bins=bins), pn.interp(pg, bins=bins, status=st))
            assert ps.ps_status_read(st)[0] == 0
            outs = []
            for sf in (pp, pn):
                tr = ps.Tracker(sf, sorted_pos.clone(), brick=(8, 8, 8))
                tr.step(1e-2)
                lab = torch.empty_like(tr.ids)
                lab[tr.ids] = torch.arange(tr.ids.numel(), device=DEV)
                outs.append((tr.pos[:, lab], tr.vel[:, lab]))
            assert all(torch.equal(x, y) for x, y in zip(*outs))
    finally:
        ps.ps_tune_set("node_tma", old)
    ulp = 2.0 ** -8 if planar == torch.bfloat16 else 2.0 ** -10
    assert abs_err(vb.cpu().numpy(), oracle.interp(cref, pos)) <= ulp * np.abs(cref).max()


# ---------------------------------------------------- second derivatives ----

@pytest.mark.parametrize("n,L", [((32, 32, 32), (TWO_PI,) * 3), ((37, 21, 10), (TWO_PI, 4.0, 2.5))])
def test_hessian_matches_oracle(n, L):
    # bar: 1e-5 relative rounding on weights summing (in absolute value) to at
    # most 4 per second-derivative axis and 1 per first-derivative axis
    field, pos, cref = _case(n, 5000, seed=171, L=L, spread=1.3)
    ref = oracle.interp_hessian(cref, pos, L=L)
    ih = np.array(n) / np.array(L)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    scale = np.array([ih[a] * ih[b] for a, b in pairs])[None, :, None]
    cmax = np.abs(cref).max()
    f = torch.from_numpy(field).to(DEV)
    pg = torch.from_numpy(pos).to(DEV)
    # binned: through the permutation, and physically sorted
    bins, sorted_pos = ps.bin_particles(n, (8, 8, 8), pg, want_sorted=True, L=L)
    sbins = ps.Bins(bins.brick, bins.offsets, bins.bin_of, None)
    perm = bins.perm.cpu().numpy()
    out, outb = {}, {}
    for dt, bar in ((torch.float32, 4e-5), (torch.float64, 1e-9), (ps.F32X4, 4e-5),
                    (torch.bfloat16, 4 * 2.0 ** -8), (ps.BF16X4, 4 * 2.0 ** -8)):
        sf = ps.SplineField.from_field(f, dt, L=L)
        st = torch.zeros(4, dtype=torch.int32, device=DEV)
        h = sf.hessian(pg, status=st).cpu().numpy()
        assert ps.ps_status_read(st)[0] == 0
        # plus the rounding of the FP32 output itself
        tol = bar * scale * cmax + 2.0 ** -23 * np.abs(ref)
        assert np.all(np.abs(h - ref) <= tol), dt
        out[dt] = h
        # from each brick's staged halo
        hb = sf.hessian(pg, status=st, bins=bins).cpu().numpy()
        hs = sf.hessian(sorted_pos, status=st, bins=sbins).cpu().numpy()
        assert ps.ps_status_read(st)[0] == 0
        assert np.all(np.abs(hb - ref) <= tol), dt
        assert np.all(np.abs(hs - ref[:, :, perm]) <= tol[:, :, perm]), dt
        outb[dt] = hb
    np.testing.assert_array_equal(out[ps.F32X4], out[torch.float32])
    np.testing.assert_array_equal(out[ps.BF16X4], out[torch.bfloat16])
    np.testing.assert_array_equal(outb[ps.F32X4], outb[torch.float32])
    np.testing.assert_array_equal(outb[ps.BF16X4], outb[torch.bfloat16])


def test_hessian_nonfinite_flagged():
    n = (16, 16, 16)
    field, pos, _ = _case(n, 64, seed=173)
    pos[1, 5] = np.nan
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    st = torch.zeros(4, dtype=torch.int32, device=DEV)
    pg = torch.from_numpy(pos).to(DEV)
    h = sf.hessian(pg, status=st).cpu().numpy()
    assert np.isnan(h[:, :, 5]).all() and np.isfinite(np.delete(h, 5, axis=2)).all()
    assert ps.ps_status_read(st)[0] == 1
    st.zero_()
    bins = ps.bin_particles(n, (8, 8, 8), pg)
    h = sf.hessian(pg, status=st, bins=bins).cpu().numpy()
    assert np.isnan(h[:, :, 5]).all() and np.isfinite(np.delete(h, 5, axis=2)).all()
    assert ps.ps_status_read(st)[0] == 1


@pytest.mark.parametrize("binned", [False, True])
@pytest.mark.parametrize("two_fields", [False, True])
def test_lagrangian_accel_matches_oracle(two_fields, binned):
    n = (24, 20, 28)
    field, pos, cref = _case(n, 6000, seed=175, spread=1.2)
    f2 = synth.random_field(n, ncomp=3, seed=176).astype(np.float32)
    cref2 = oracle.spline_coeffs(f2.astype(np.float64))
    dt = 0.05
    ref = oracle.lagrangian_accel(cref, pos, cref2 if two_fields else None, dt)
    u, G = oracle.interp(cref, pos, grad=True)
    pg = torch.from_numpy(pos).to(DEV)
    bins = ps.bin_particles(n, (8, 8, 8), pg) if binned else None
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    sf2 = ps.SplineField.from_field(torch.from_numpy(f2).to(DEV), torch.float32)
    a = sf.acceleration(pg, later=sf2 if two_fields else None, dt_field=dt,
                        bins=bins).cpu().numpy()
    if binned:
        # node storage holds the same values: the same bits
        n4 = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), ps.F32X4)
        n42 = ps.SplineField.from_field(torch.from_numpy(f2).to(DEV), ps.F32X4)
        a4 = n4.acceleration(pg, later=n42 if two_fields else None, dt_field=dt,
                             bins=bins).cpu().numpy()
        np.testing.assert_array_equal(a4, a)
    # sum over three axes of (gradient bar 1e-5 * 3 * n/L * max|c|) * |u|
    # + |grad u| * (velocity bar 1e-5 rms), plus both fields' velocity bars
    # over dt
    ih = max(n) / TWO_PI
    cmax = max(np.abs(cref).max(), np.abs(cref2).max())
    rms = np.sqrt((u ** 2).mean())
    tol = 3 * (1e-5 * 3 * ih * cmax * np.abs(u).max() + np.abs(G).max() * 1e-5 * rms)
    if two_fields:
        tol += 2 * 1e-5 * 3 * rms / dt
    assert np.abs(a - ref).max() <= tol


def _slot_bins(offs):
    return np.repeat(np.arange(len(offs) - 1), np.diff(offs))


@pytest.mark.parametrize("kernel", [0, 2, 5])
@pytest.mark.parametrize("kind", [torch.float32, ps.F32X4, torch.bfloat16, ps.BF16X4])
def test_rk2_counted_sort_matches_full_sort(kernel, kind, brick_kernel):
    # Steps whose sort starts from the counts the previous step's kernel took
    # while it stored the positions (rebin 2, then 3: the departing particles
    # found during the update, Sec. 4.3) give every particle the bits of steps
    # that sort from scratch (rebin 1) and the same bin bounds, which are
    # those of the oracle's counting sort of each step's starting positions.
    ps.ps_tune_set("brick_kernel", kernel)
    n, brick, np_ = (48, 40, 32), (8, 8, 8), 30000
    field, pos, _ = _case(n, np_, seed=151, spread=1.3)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), kind)
    dt = 4e-2  # a quarter of a cell per step at unit speed: many particles change brick
    full = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick, incremental=False)
    inc = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick)
    prev_bin = None
    moved = 0
    for _ in range(4):
        start = np.empty_like(pos)
        start[:, full.ids.cpu().numpy()] = full.pos.cpu().numpy()  # by particle id
        bin_id, off_ora, _ = oracle.bin_particles(n, brick, start)
        if prev_bin is not None:
            moved += int((bin_id != prev_bin).sum())
        prev_bin = bin_id
        full.step(dt)
        inc.step(dt)
        for tr in (full, inc):
            np.testing.assert_array_equal(tr.offsets.cpu().numpy(), off_ora)
            ids = tr.ids.cpu().numpy()
            # storage order: the bin order of the starting positions
            np.testing.assert_array_equal(bin_id[ids], _slot_bins(off_ora))
        fi, ii = np.argsort(full.ids.cpu().numpy()), np.argsort(inc.ids.cpu().numpy())
        assert np.array_equal(full.pos.cpu().numpy()[:, fi], inc.pos.cpu().numpy()[:, ii])
        assert np.array_equal(full.vel.cpu().numpy()[:, fi], inc.vel.cpu().numpy()[:, ii])
    assert ps.ps_status_read(full.status)[0] == 0
    assert ps.ps_status_read(inc.status)[0] == 0
    assert moved > 1000


def test_rk2_counted_sort_with_changed_positions():
    # positions changed between steps leave the counts in the workspace stale:
    # the sort then follows the old bins, and particles outside their brick's
    # halo read their stencils from global memory, so results stay exact
    n = (32, 32, 32)
    field, pos, cref = _case(n, 8000, seed=171)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=(8, 8, 8))
    dt = 1e-2
    tr.step(dt)
    tr.pos += 0.37  # 1.9 cells: most particles leave their brick
    ids0 = tr.ids.cpu().numpy()
    start = tr.pos.cpu().numpy()
    tr.step(dt)  # rebin 3 with the counts of the unshifted positions
    new_ref, u1_ref = oracle.rk2_step(cref, start, dt)
    by_id = np.empty_like(new_ref)
    by_id[:, ids0] = new_ref
    rms = np.sqrt((u1_ref ** 2).mean())
    ids = tr.ids.cpu().numpy()
    assert np.abs(tr.pos.cpu().numpy() - by_id[:, ids]).max() <= dt * 1e-5 * rms + 1e-13
    assert ps.ps_status_read(tr.status)[0] == 0
    # reset_bins: the next step sorts from the positions again
    tr.reset_bins()
    start = tr.pos.cpu().numpy()
    tr.step(dt)
    _, off_ora, _ = oracle.bin_particles(n, (8, 8, 8), start)
    np.testing.assert_array_equal(tr.offsets.cpu().numpy(), off_ora)


@pytest.mark.parametrize("fill", [0, 255])
def test_rk2_counted_sort_rejects_foreign_counts(fill):
    # rebin 3 on a workspace that holds no counts of these positions: slots
    # are checked against their bin's range and bin bounds are clamped to the
    # particle count, so every access stays inside the arrays; the status word
    # reports PS_DEV_BAD_BINS and the particles keep their positions.  A
    # rebin 2 step on the same workspace then restores the counts.
    n, brick, np_ = (32, 32, 32), (8, 8, 8), 5000
    field, pos, cref = _case(n, np_, seed=181)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    p = torch.from_numpy(pos.copy()).to(DEV)
    ws = ps.workspace(ps.ps_rk2_workspace_size(n, brick, np_), DEV)
    ws.fill_(fill)
    offs = torch.empty(4 ** 3 + 1, dtype=torch.int32, device=DEV)
    status = torch.zeros(4, dtype=torch.int32, device=DEV)
    ps.ps_rk2_step(sf.coef, n, p, 1e-2, brick=brick, rebin=3, bin_offsets=offs, ws=ws,
                   status=status)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert st[0] == ps._abi.PS_DEV_BAD_BINS
    assert torch.equal(p.cpu(), torch.from_numpy(pos))
    status.zero_()
    dt = 1e-2
    ps.ps_rk2_step(sf.coef, n, p, dt, brick=brick, rebin=2, bin_offsets=offs, ws=ws,
                   status=status)
    mid = p.cpu().numpy()
    ps.ps_rk2_step(sf.coef, n, p, dt, brick=brick, rebin=3, bin_offsets=offs, ws=ws,
                   status=status)
    torch.cuda.synchronize()
    assert status.cpu().numpy()[0] == 0
    _, off_ora, _ = oracle.bin_particles(n, brick, mid)
    np.testing.assert_array_equal(offs.cpu().numpy(), off_ora)


def test_rk2_sort_then_step_equals_rebinned_step():
    # ps_rk2_step(rebin 2, then 3) is ps_rk2_sort followed by the rebin 0 step
    # with the workspace: driven with the caller's own buffers in ping-pong the
    # two give the same bits, the same bin bounds and the same velocities
    n, brick, np_ = (40, 32, 24), (8, 8, 8), 12000
    field, pos, _ = _case(n, np_, seed=191, spread=1.2)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), ps.F32X4)
    dt = 3e-2
    tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick)
    ws = ps.workspace(ps.ps_rk2_workspace_size(n, brick, np_), DEV)
    offs = torch.empty_like(tr.offsets)
    status = torch.zeros(4, dtype=torch.int32, device=DEV)
    bufs = [torch.from_numpy(pos.copy()).to(DEV), torch.empty((3, np_), dtype=torch.float64,
                                                              device=DEV)]
    idb = [torch.arange(np_, dtype=torch.int64, device=DEV), torch.empty(np_, dtype=torch.int64,
                                                                         device=DEV)]
    vel = torch.empty((3, np_), dtype=torch.float32, device=DEV)
    for k in range(3):
        tr.step(dt)
        ps.ps_rk2_sort(n, brick, bufs[0], bufs[1], offs, ws, ids=idb[0], ids_sorted=idb[1],
                       counted=k > 0, status=status)
        ps.ps_rk2_step(sf.coef, n, bufs[1], dt, vel_out=vel, brick=brick, rebin=0,
                       bin_offsets=offs, ws=ws, status=status)
        bufs.reverse()
        idb.reverse()
        assert torch.equal(offs, tr.offsets)
        a, b = torch.argsort(tr.ids), torch.argsort(idb[0])
        assert torch.equal(tr.pos[:, a], bufs[0][:, b])
        assert torch.equal(tr.vel[:, a], vel[:, b])
    assert ps.ps_status_read(status)[0] == 0
    assert ps.ps_status_read(tr.status)[0] == 0


@pytest.mark.parametrize("kernel", [0, 2, 5])
def test_rk2_counted_sort_at_cell_faces(kernel, brick_kernel):
    # A constant field moves every particle by exactly dt u; targets are put on
    # cell faces, just either side of them (down to 1e-13 of a cell) and at the
    # 2^-10 margin of the step kernel's FP32 shortcut, some far from the
    # origin.  The counts the step takes must be the oracle's counts of the
    # positions it wrote, face for face.
    ps.ps_tune_set("brick_kernel", kernel)
    n, brick = (16, 16, 16), (8, 8, 8)
    h = TWO_PI / 16
    u = np.array([0.75, -0.5, 0.3125])
    field = np.broadcast_to(u[:, None, None, None], (3, 16, 16, 16)).astype(np.float32).copy()
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), ps.F32X4)
    dt = 0.37 * h
    eps = [0.0, 1e-13, -1e-13, 1e-9, -1e-9, 1e-6, -1e-6, 2.0 ** -10, -(2.0 ** -10),
           2.0 ** -10 + 1e-6, 2.0 ** -10 - 1e-6, 0.5]
    rng = np.random.default_rng(7)
    tgt = []
    for e in eps:
        for far in (0, 1 << 20, -(1 << 31), 3 << 40):
            face = rng.integers(0, 16, size=3) + far
            tgt.append((face + e) * h)
    tgt = np.array(tgt).T  # [3][m]
    m = tgt.shape[1]
    pos0 = tgt - dt * u[:, None]
    p = torch.from_numpy(pos0.copy()).to(DEV)
    tr = ps.Tracker(sf, p, brick=brick)
    tr.step(dt)  # rebin 2: counts the written positions
    after = tr.pos.cpu().numpy()
    tr.step(dt)  # rebin 3: sorts from those counts
    _, off_ora, _ = oracle.bin_particles(n, brick, after)
    np.testing.assert_array_equal(tr.offsets.cpu().numpy(), off_ora)
    assert ps.ps_status_read(tr.status)[0] == 0
    assert m == len(eps) * 4


@pytest.mark.parametrize("brick", [(5, 7, 3), (16, 8, 4), (1, 1, 1)])
def test_rk2_counted_sort_other_bricks(brick):
    # bricks whose extents are not all powers of two (the new brick is a
    # division, not a shift) and single-cell bricks: counted sorts match full
    # sorts bit for bit, and their bounds the oracle's
    n = (40, 28, 24)
    field, pos, _ = _case(n, 12000, seed=201, spread=1.2)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), ps.F32X4)
    dt = 3e-2
    full = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick, incremental=False)
    inc = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick)
    for _ in range(3):
        start = inc.pos.cpu().numpy()
        full.step(dt)
        inc.step(dt)
        _, off_ora, _ = oracle.bin_particles(n, brick, start)
        np.testing.assert_array_equal(inc.offsets.cpu().numpy(), off_ora)
        np.testing.assert_array_equal(full.offsets.cpu().numpy(), off_ora)
        a, b = torch.argsort(full.ids), torch.argsort(inc.ids)
        assert torch.equal(full.pos[:, a], inc.pos[:, b])
    assert ps.ps_status_read(inc.status)[0] == 0


def test_rk2_counted_sort_degenerate_sets():
    # no particles at all, and every particle in one cell (one bin holds them
    # all, every other bin is empty)
    n, brick = (16, 16, 16), (8, 8, 8)
    field, _, cref = _case(n, 10, seed=211)
    sf = ps.SplineField.from_field(torch.from_numpy(field).to(DEV), torch.float32)
    ws = ps.workspace(ps.ps_rk2_workspace_size(n, brick, 0), DEV)
    offs = torch.empty(2 ** 3 + 1, dtype=torch.int32, device=DEV)
    empty = torch.empty((3, 0), dtype=torch.float64, device=DEV)
    for mode in (2, 3):
        ps.ps_rk2_step(sf.coef, n, empty, 1e-3, brick=brick, rebin=mode, bin_offsets=offs, ws=ws)
        torch.cuda.synchronize()
        assert torch.count_nonzero(offs).item() == 0
    ps.ps_rk2_sort(n, brick, empty, torch.empty_like(empty), offs, ws, counted=True)
    torch.cuda.synchronize()
    h = TWO_PI / 16
    pos = np.full((3, 3000), 2.5 * h) + np.linspace(0, 0.4 * h, 3000)[None, :]
    tr = ps.Tracker(sf, torch.from_numpy(pos.copy()).to(DEV), brick=brick)
    ref = pos.copy()
    for _ in range(3):
        tr.step(1e-3)
        ref, _ = oracle.rk2_step(cref, ref, 1e-3)
    ids = tr.ids.cpu().numpy()
    assert np.abs(tr.pos.cpu().numpy() - ref[:, ids]).max() <= 3 * 1e-3 * 1e-5 * 4 + 1e-13
    _, off_ora, _ = oracle.bin_particles(n, brick, tr.pos.cpu().numpy())
    tr.step(1e-3)
    np.testing.assert_array_equal(tr.offsets.cpu().numpy(), off_ora)
    assert ps.ps_status_read(tr.status)[0] == 0


def _trunc_bar(K, field):
    # three passes, each a sum of 2K + 1 FP32 products of values bounded by
    # 9 max|field| (sum |G| = 3 per axis already filtered)
    return 3 * (2 * K + 1) * 2.0 ** -24 * 9 * np.abs(field).max()


@pytest.mark.parametrize("n,K", [((32, 32, 32), 15), ((37, 33, 40), 12), ((12, 10, 9), 4),
                                 ((9, 9, 9), 4), ((64, 48, 40), 8), ((300, 31, 33), 15)])
def test_truncated_solve_matches_oracle(n, K):
    # the convolution with the periodic inverse's entries cut at |d| <= K,
    # against the oracle's FP64 convolution; the row padding stays zero
    field = synth.random_field(n, ncomp=3, seed=221).astype(np.float32)
    ref = oracle.spline_coeffs_truncated(field.astype(np.float64), K)
    f = torch.from_numpy(field).to(DEV)
    coef = torch.full(ps.coef_shape(n, 3, torch.float32), 7.0, dtype=torch.float32, device=DEV)
    ps.ps_spline_coeffs_truncated(f, coef, K=K)
    got = coef.cpu().numpy()
    assert np.abs(got[..., :n[0] + 3] - ref).max() <= _trunc_bar(K, field)
    assert not np.any(got[..., n[0] + 3:])


def test_truncated_solve_against_exact_solve():
    # with K = 15 the neglected entries are below FP32 rounding: the result
    # meets the exact solve (GPU and oracle) within the two rounding bars
    n = (64, 48, 40)
    field = synth.random_field(n, ncomp=3, seed=231).astype(np.float32)
    exact = oracle.spline_coeffs(field.astype(np.float64))
    f = torch.from_numpy(field).to(DEV)
    coef = torch.empty(ps.coef_shape(n, 3, torch.float32), dtype=torch.float32, device=DEV)
    ps.ps_spline_coeffs_truncated(f, coef, K=15)
    r = abs(math.sqrt(3.0) - 2.0)
    tail = 27 * 2 * math.sqrt(3.0) * r ** 16 / (1 - r) * np.abs(field).max()
    got = coef.cpu().numpy()[..., :n[0] + 3]
    assert np.abs(got - exact).max() <= _trunc_bar(15, field) + tail
    sf = ps.SplineField.from_field(f, torch.float32)
    gpu_exact = sf.padded().cpu().numpy()
    assert np.abs(got - gpu_exact).max() <= _trunc_bar(15, field) + tail + coef_tol(field)


def test_truncated_solve_rejects_bad_K():
    f = torch.zeros((3, 16, 16, 16), dtype=torch.float32, device=DEV)
    coef = torch.empty(ps.coef_shape((16, 16, 16), 3, torch.float32), dtype=torch.float32,
                       device=DEV)
    for K in (0, 8, 16):  # 2K+1 = 17 > 16 for K = 8
        with pytest.raises(ps.PSError):
            ps.ps_spline_coeffs_truncated(f, coef, K=K)
