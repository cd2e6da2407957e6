"""Host-side logic that needs no GPU: the autotuner's cache file and the
plane-by-plane spectral generator."""
import numpy as np
import torch

from paper_2005_13193_gb300 import autotune, synth


def test_tune_cache_round_trip(tmp_path):
    p = str(tmp_path / "x.tune")
    autotune.write_cache(p, {"kernel": 2, "brick": (16, 8, 4)}, comment="two\nlines")
    text = open(p).read()
    assert text.splitlines()[:2] == ["# two", "# lines"]
    assert "brick 16 8 4" in text  # the line ps_batch_plan parses
    assert autotune.load_cache(p) == {"kernel": (2,), "brick": (16, 8, 4)}
    assert autotune.load_cache(str(tmp_path / "missing")) == {}


def test_spectral_field_planes_recipe():
    n, kmax = 24, 8
    f = synth.spectral_field_planes(n, kmax, seed=9, dtype=torch.float64).numpy()
    g = synth.spectral_field_planes(n, kmax, seed=9, dtype=torch.float64).numpy()
    np.testing.assert_array_equal(f, g)  # seeded
    assert np.allclose(np.sqrt((f ** 2).mean(axis=(1, 2, 3))), 1.0, atol=1e-12)
    F = np.fft.fftn(f, axes=(1, 2, 3))
    k = np.fft.fftfreq(n, 1.0 / n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    shell = (k2 >= 1) & (k2 <= kmax * kmax)
    # energy only on the shell 1 <= |k| <= kmax
    assert np.abs(F[:, ~shell]).max() <= 1e-9 * np.abs(F[:, shell]).max()
    # amplitude per shell falls off (k^-5/3 shell energy): compare shells 2 and 6
    e = lambda s: (np.abs(F[:, (np.sqrt(k2) >= s - 0.5) & (np.sqrt(k2) < s + 0.5)]) ** 2).sum()
    assert e(2) > e(6)


def test_tracker_rebin_modes(monkeypatch):
    # Tracker picks ps_rk2_step's rebin mode on the host: sort from the
    # positions and count (2) on the first step, then sort from the counts its
    # previous step took (3); a step with given bins (0), reset_bins() or
    # incremental=False go back to sorting from the positions
    import types

    import paper_2005_13193_gb300 as ps
    seen = []
    monkeypatch.setattr(ps, "ps_rk2_step", lambda *a, **k: seen.append(k["rebin"]))
    monkeypatch.setattr(ps, "workspace", lambda nbytes, device="cpu": torch.empty(0))
    field = types.SimpleNamespace(n=(16, 16, 16), L=(2 * np.pi,) * 3, coef=None, scale=None)
    pos = torch.zeros((3, 100), dtype=torch.float64)
    tr = ps.Tracker(field, pos, brick=(8, 8, 8), keep_velocity=False)
    for _ in range(3):
        tr.step(1e-3)
    tr.step(1e-3, rebin=False)
    tr.step(1e-3)
    tr.reset_bins()
    tr.step(1e-3)
    tr.step(1e-3)
    assert seen == [2, 3, 3, 0, 2, 2, 3]
    seen.clear()
    full = ps.Tracker(field, pos, brick=(8, 8, 8), keep_velocity=False, incremental=False)
    full.step(1e-3)
    full.step(1e-3)
    assert seen == [1, 1]
