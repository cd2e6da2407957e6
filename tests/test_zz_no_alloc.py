"""Allocation-free binning (ps_bin_particles_noalloc) against the workspace
form, through the C ABI.  Collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test.

The entry point exists for callers that cannot allocate device memory or pass
a workspace when they bin particles; its scratch is a fixed device array
shared by all calls."""
import ctypes
import math

import numpy as np
import pytest
import torch

import paper_2005_13193_gb300 as ps
from paper_2005_13193_gb300 import _abi, synth

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_binning_matches_workspace_form_twice():
    lib = _abi.load()
    n, brick, L = (64, 48, 40), (8, 8, 8), (TWO_PI, 3.0, 2.5)
    np_ = 200_003
    pos = synth.uniform_particles(np_, seed=77) / TWO_PI * np.array(L)[:, None] * 1.5 - 0.4
    pg = torch.from_numpy(pos).cuda()
    ref, ref_sorted = ps.bin_particles(n, brick, pg, L=L, want_sorted=True)
    ref_of = ref.bin_of.cpu().numpy()
    ref_off = ref.offsets.cpu().numpy()
    ref_perm = ref.perm.cpu().numpy()
    nbins = len(ref_off) - 1
    grid = ps.make_grid(n, L)
    br = (ctypes.c_int32 * 3)(*brick)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        bin_of = torch.full((np_,), -7, dtype=torch.int32, device="cuda")
        offs = torch.full((nbins + 1,), -7, dtype=torch.int32, device="cuda")
        perm = torch.full((np_,), -7, dtype=torch.int64, device="cuda")
        srt = torch.empty_like(pg)
        status = torch.zeros(4, dtype=torch.int32, device="cuda")
        rc = lib.ps_bin_particles_noalloc(ctypes.byref(grid), br, np_, _p(pg), _p(bin_of),
                                          _p(offs), _p(perm), _p(srt), _p(status), stream)
        assert rc == 0, lib.ps_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(bin_of.cpu().numpy(), ref_of)
        off = offs.cpu().numpy()
        np.testing.assert_array_equal(off, ref_off)
        got = perm.cpu().numpy()
        assert np.array_equal(np.sort(got), np.arange(np_))
        for b in np.nonzero(np.diff(off))[0][:2000]:
            assert set(got[off[b]:off[b + 1]]) == set(ref_perm[off[b]:off[b + 1]])
        np.testing.assert_array_equal(srt.cpu().numpy(), pos[:, got])
        assert ps.ps_status_read(status)[0] == 0


def test_noalloc_binning_rejects_requests_beyond_its_scratch():
    lib = _abi.load()
    grid = ps.make_grid((256, 256, 256))
    br = (ctypes.c_int32 * 3)(1, 1, 1)  # 2^24 bins alone exceed 32 MiB of scratch
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.ps_bin_particles_noalloc(ctypes.byref(grid), br, 1, _p(dummy), _p(dummy), _p(dummy),
                                      None, None, None, None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    assert b"scratch" in lib.ps_last_error()
