"""Many-field form (ps_batch_plan / ps_batch_run).

Every particle's arithmetic in a batch is the per-field arithmetic, so batched
positions and velocities must equal per-field ps_rk2_step runs bit for bit
(compared by particle label, since the order inside a bin is unspecified), and
a replayed CUDA graph must equal eager execution.  The 48-field workload is
also spot-checked against the FP64 oracle.
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


def _fields(sizes, seed, dtype=torch.float32):
    out = []
    for i, n in enumerate(sizes):
        f = synth.spectral_field(n, n // 3, seed=seed + i, device=DEV, dtype=torch.float32)
        out.append((f, ps.SplineField.from_field(f, dtype)))
    return out


def _positions(nps, seed):
    cols = [synth.uniform_particles(n, seed=seed + i) for i, n in enumerate(nps)]
    return np.concatenate(cols, axis=1) if cols else np.zeros((3, 0))


def _by_label(x, ids):
    out = np.empty_like(x)
    out[..., ids] = x
    return out


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, ps.F32X4, ps.BF16X4])
def test_batch_equals_per_field_runs(dtype):
    # the last field is sparse (about 4 particles per 8^3 brick): the plan
    # bins it in runs of particles and gathers from global memory
    sizes = [16, 24, 32, 48, 32, 64]
    nps = [1000, 50000, 3000, 20000, 0, 2000]
    dt, nsteps = 4e-3, 3
    flds = _fields(sizes, 300, dtype)
    pos0 = _positions(nps, 400)
    plan = ps.BatchPlan([(n,) * 3 for n in sizes], nps, coef_dtype=dtype)
    assert plan.np_total == sum(nps) and plan.base == list(np.cumsum([0] + nps))
    pos = torch.from_numpy(pos0.copy()).to(DEV)
    ids = torch.arange(plan.np_total, dtype=torch.int64, device=DEV)
    vel = torch.empty((3, plan.np_total), dtype=torch.float32, device=DEV)
    st = torch.zeros(4, dtype=torch.int32, device=DEV)
    plan.run([(f, sf) for f, sf in flds], pos, nsteps, dt, solve=True, ids=ids, vel=vel,
             use_graph=False, status=st)
    assert ps.ps_status_read(st)[0] == 0
    got_x = _by_label(pos.cpu().numpy(), ids.cpu().numpy())
    got_v = _by_label(vel.cpu().numpy(), ids.cpu().numpy())
    # the batched form runs the phased brick kernel (0); per-field runs take
    # the same kernel so that the arithmetic, and the bits, are the same
    old = ps.ps_tune_get("brick_kernel")
    ps.ps_tune_set("brick_kernel", 0)
    try:
        for f, (n, npf) in enumerate(zip(sizes, nps)):
            if npf == 0:
                continue
            b = plan.base[f]
            sf = ps.SplineField.from_field(flds[f][0], dtype)
            tr = ps.Tracker(sf, torch.from_numpy(pos0[:, b:b + npf].copy()).to(DEV),
                            brick=(8, 8, 8))
            for _ in range(nsteps):
                tr.step(dt)
            ref_x = _by_label(tr.pos.cpu().numpy(), tr.ids.cpu().numpy())
            ref_v = _by_label(tr.vel.cpu().numpy(), tr.ids.cpu().numpy())
            np.testing.assert_array_equal(got_x[:, b:b + npf], ref_x)
            np.testing.assert_array_equal(got_v[:, b:b + npf], ref_v)
    finally:
        ps.ps_tune_set("brick_kernel", old)


def _run_batch(sizes, nps, dtype, seed, nsteps, dt, use_graph, status=None):
    flds = _fields(sizes, seed, dtype)
    pos0 = _positions(nps, seed + 100)
    plan = ps.BatchPlan([(n,) * 3 for n in sizes], nps, coef_dtype=dtype)
    pos = torch.from_numpy(pos0.copy()).to(DEV)
    ids = torch.arange(plan.np_total, dtype=torch.int64, device=DEV)
    vel = torch.empty((3, plan.np_total), dtype=torch.float32, device=DEV)
    plan.run([(f, sf) for f, sf in flds], pos, nsteps, dt, solve=True, ids=ids, vel=vel,
             use_graph=use_graph, status=status)
    return (_by_label(pos.cpu().numpy(), ids.cpu().numpy()),
            _by_label(vel.cpu().numpy(), ids.cpu().numpy()))


@pytest.mark.parametrize("dtype", [torch.float32, ps.F32X4, ps.BF16X4])
def test_persistent_launch_equals_launch_per_step(dtype):
    # All steps in one cooperative launch (the default: the sort's phases and
    # the brick pass separated by grid-wide barriers) give every particle the
    # bits of a launch per phase and step, eager or replayed from a graph that
    # also holds the solves.
    sizes, nps = [16, 24, 32, 48, 32, 64], [1000, 50000, 3000, 20000, 0, 2000]
    old = ps.ps_tune_get("batch_persistent")
    try:
        out = {}
        for persistent in (1, 0):
            ps.ps_tune_set("batch_persistent", persistent)
            for use_graph in (False, True):
                st = torch.zeros(4, dtype=torch.int32, device=DEV)
                out[(persistent, use_graph)] = _run_batch(sizes, nps, dtype, 800, 4, 4e-3,
                                                          use_graph, st)
                assert ps.ps_status_read(st)[0] == 0
    finally:
        ps.ps_tune_set("batch_persistent", old)
    ref = out[(0, False)]
    for k, (x, v) in out.items():
        np.testing.assert_array_equal(x, ref[0])
        np.testing.assert_array_equal(v, ref[1])


def test_persistent_barrier_wait_gives_up():
    # The test knob "wait_probe" makes every block, after the first grid
    # barrier, wait on a word that nothing sets, bounded by that many clocks:
    # the wait gives up, the status word reads PS_DEV_TIMEOUT, every block
    # leaves at its next barrier and the launch returns.  The device stays
    # usable: the next run, without the knob, matches a launch per step.
    sizes, nps = [16, 32, 24], [3000, 20000, 5000]
    old = ps.ps_tune_get("wait_probe")
    try:
        ps.ps_tune_set("wait_probe", 20000)
        st = torch.zeros(4, dtype=torch.int32, device=DEV)
        _run_batch(sizes, nps, torch.float32, 900, 3, 4e-3, False, st)
        code, _, _, count = ps.ps_status_read(st)
        assert code == ps._abi.PS_DEV_TIMEOUT and count > 0
    finally:
        ps.ps_tune_set("wait_probe", old)
    st = torch.zeros(4, dtype=torch.int32, device=DEV)
    got = _run_batch(sizes, nps, torch.float32, 900, 3, 4e-3, False, st)
    assert ps.ps_status_read(st)[0] == 0
    old_p = ps.ps_tune_get("batch_persistent")
    try:
        ps.ps_tune_set("batch_persistent", 0)
        ref = _run_batch(sizes, nps, torch.float32, 900, 3, 4e-3, False)
    finally:
        ps.ps_tune_set("batch_persistent", old_p)
    np.testing.assert_array_equal(got[0], ref[0])


def test_graph_replay_equals_eager_and_is_reused():
    sizes = [32, 64, 48]
    nps = [20000, 100000, 7000]
    dt, nsteps = 2e-3, 4
    flds = _fields(sizes, 500)
    pos0 = _positions(nps, 600)
    plan = ps.BatchPlan([(n,) * 3 for n in sizes], nps)
    runs = {}
    for use_graph in (False, True):
        pos = torch.from_numpy(pos0.copy()).to(DEV)
        ids = torch.arange(plan.np_total, dtype=torch.int64, device=DEV)
        # two calls in a row: the second replays the captured graph
        plan.run([(f, sf) for f, sf in flds], pos, nsteps, dt, solve=True, ids=ids,
                 use_graph=use_graph)
        plan.run([(f, sf) for f, sf in flds], pos, nsteps, dt, solve=False, ids=ids,
                 use_graph=use_graph)
        runs[use_graph] = _by_label(pos.cpu().numpy(), ids.cpu().numpy())
    np.testing.assert_array_equal(runs[True], runs[False])


def test_batch_config_48_fields():
    # 48 fields, edges uniform over {64, 96, 128, 192, 256}, 10k..2M particles
    # per field (log-uniform), 20 Heun steps captured in a CUDA graph.
    sizes, nps = synth.batch_sizes(48, seed=3000)
    dt, nsteps = 1e-3, 20
    flds = _fields(sizes, 3100)
    pos0 = _positions(nps, 3200)
    plan = ps.BatchPlan([(n,) * 3 for n in sizes], nps)
    pos = torch.from_numpy(pos0.copy()).to(DEV)
    ids = torch.arange(plan.np_total, dtype=torch.int64, device=DEV)
    st = torch.zeros(4, dtype=torch.int32, device=DEV)
    plan.run([(f, sf) for f, sf in flds], pos, nsteps, dt, solve=True, ids=ids, use_graph=True,
             status=st)
    assert ps.ps_status_read(st)[0] == 0
    got = _by_label(pos.cpu().numpy(), ids.cpu().numpy())
    assert np.isfinite(got).all()
    # oracle trajectories for a few particles of the three smallest fields
    rng = np.random.default_rng(11)
    for f in np.argsort(sizes)[:3]:
        n, b, npf = sizes[f], plan.base[f], nps[f]
        cref = oracle.spline_coeffs(flds[f][0].cpu().numpy().astype(np.float64))
        pick = b + rng.choice(npf, size=min(200, npf), replace=False)
        x = pos0[:, pick].copy()
        u_max = 0.0
        for _ in range(nsteps):
            x, u = oracle.rk2_step(cref, x, dt)
            u_max = max(u_max, float(np.abs(u).max()))
        # 20 steps of per-step error <= dt 1e-5 |u|, grown at most by the
        # trajectories' divergence over t = 0.02 (|grad u| <= n/3 |u|)
        growth = math.exp(nsteps * dt * (n / 3) * u_max)
        assert np.abs(got[:, pick] - x).max() <= nsteps * dt * 1e-5 * u_max * growth + 1e-13


def test_autotune_tracker_and_batch(tmp_path):
    from paper_2005_13193_gb300 import autotune
    old = ps.ps_tune_get("brick_kernel")
    try:
        f = synth.spectral_field(64, 21, seed=700, device=DEV, dtype=torch.float32)
        sf = ps.SplineField.from_field(f)
        pos = torch.from_numpy(synth.uniform_particles(200000, seed=701)).to(DEV)
        before = pos.clone()
        cache = str(tmp_path / "tracker.tune")
        best, table = autotune.tune_tracker(sf, pos, candidates=((8, 8, 8), (8, 8, 4)),
                                            kernels=(0, 2), cache=cache)
        assert best in table and len(table) == 4
        assert all(v > 0 for v in table.values())
        assert torch.equal(pos, before)
        assert ps.ps_tune_get("brick_kernel") == best[0]
        assert autotune.load_cache(cache) == {"kernel": (best[0],), "brick": best[1]}
    finally:
        ps.ps_tune_set("brick_kernel", old)

    sizes, nps = [32, 64, 48], [30000, 80000, 5000]
    flds = _fields(sizes, 710)
    pos0 = _positions(nps, 720)
    pos = torch.from_numpy(pos0.copy()).to(DEV)
    fields = [(fl, s) for fl, s in flds]
    cache = str(tmp_path / "batch.tune")
    bbest, btable = autotune.tune_batch([(n,) * 3 for n in sizes], nps, fields, pos,
                                        candidates=((8, 8, 8), (8, 4, 4), (16, 8, 8)),
                                        cache=cache)
    assert bbest in btable and np.array_equal(pos.cpu().numpy(), pos0)
    # a plan built from the cache runs the tuned shape: bit-identical (per
    # particle label; the order inside a bin is unspecified) to an explicit
    # plan with that brick
    outs = []
    for kw in ({"tune_cache": cache}, {"brick": bbest}):
        plan = ps.BatchPlan([(n,) * 3 for n in sizes], nps, **kw)
        p = torch.from_numpy(pos0.copy()).to(DEV)
        ids = torch.arange(plan.np_total, dtype=torch.int64, device=DEV)
        plan.run(fields, p, 3, 2e-3, solve=False, ids=ids, use_graph=False)
        outs.append(_by_label(p.cpu().numpy(), ids.cpu().numpy()))
    np.testing.assert_array_equal(outs[0], outs[1])
