"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the interpolation method's arithmetic: it only draws
the inputs that both the CUDA path and the FP64 oracle consume.

The paper tracks fluid particles in DNS fields of stationary isotropic
turbulence in a periodic box [0, 2 pi)^3 (Sec. 2.1), with particle positions
drawn uniformly at random over the whole domain (Sec. 2.2).  Those fields are
not available, so a random-phase solenoidal field with a k^-5/3 shell
spectrum stands in for them:

  for every integer wavevector with 1 <= |k|^2 <= kmax^2 draw a complex
  Gaussian 3-vector, project it perpendicular to k, normalise it and scale it
  to amplitude |k|^(-11/6) (shell energy ~ k^2 |k|^(-11/3) = k^(-5/3)); take
  the real part of the complex inverse FFT; rescale each component to unit rms.

Particles are i.i.d. uniform on [0, L)^3 in FP64 (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np
import torch

TWO_PI = 2.0 * math.pi


def spectral_field(n: int, kmax: int | None = None, seed: int = 1000,
                   device: str | torch.device = "cpu", dtype=torch.float32,
                   ncomp: int = 3) -> torch.Tensor:
    """Return a [ncomp][n][n][n] (z, y, x; x fastest) random-phase k^-5/3 field.

    The Gaussian draws come from a torch generator on `device` seeded with
    `seed`; the field is built one component at a time to bound memory.
    """
    if kmax is None:
        kmax = n // 3
    dev = torch.device(device)
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    rdt = torch.float64 if dtype == torch.float64 else torch.float32
    k1 = torch.fft.fftfreq(n, d=1.0 / n, device=dev, dtype=rdt)  # integer wavenumbers
    kz = k1.view(n, 1, 1)
    ky = k1.view(1, n, 1)
    kx = k1.view(1, 1, n)
    k2 = kz * kz + ky * ky + kx * kx
    mask = (k2 >= 1) & (k2 <= kmax * kmax)
    kmag = torch.sqrt(k2.clamp(min=1))
    amp = torch.where(mask, kmag.pow(-11.0 / 6.0), torch.zeros_like(kmag))
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    # complex Gaussian 3-vector per wavevector
    shape = (3, n, n, n)
    a = torch.complex(torch.randn(shape, generator=gen, device=dev, dtype=rdt),
                      torch.randn(shape, generator=gen, device=dev, dtype=rdt))
    # project perpendicular to k: a - k (k . a) / |k|^2
    kvec = (kx.expand(n, n, n), ky.expand(n, n, n), kz.expand(n, n, n))
    kd = (kvec[0] * a[0] + kvec[1] * a[1] + kvec[2] * a[2]) / k2.clamp(min=1)
    for d in range(3):
        a[d] -= kvec[d] * kd
    norm = torch.sqrt((a.real ** 2 + a.imag ** 2).sum(0)).clamp(min=1e-30)
    scale = (amp / norm).to(cdt)
    out = torch.empty((ncomp, n, n, n), device=dev, dtype=dtype)
    for c in range(ncomp):
        spec = a[c % 3] * scale
        comp = torch.fft.ifftn(spec, dim=(0, 1, 2)).real
        rms = torch.sqrt((comp.double() ** 2).mean())
        out[c] = (comp / rms).to(dtype)
        del spec, comp
    return out


def spectral_field_planes(n: int, kmax: int | None = None, seed: int = 1000,
                          device: str | torch.device = "cpu", dtype=torch.float32,
                          ncomp: int = 3, chunk: int = 64) -> torch.Tensor:
    """The same k^-5/3 random-phase recipe as `spectral_field`, built one kz
    plane at a time so that a 1536^3 field fits next to its coefficients.

    The Gaussian draws of plane kz come from a generator seeded with
    (seed << 12) + (plane index), so they differ from `spectral_field`'s;
    planes with |kz| > kmax are zero and draw nothing.  The inverse FFT is done
    separably (x-y per block of planes, then z per block of rows) in place on
    one complex component, and the rms rescale is accumulated in FP64 per
    block.  Peak extra memory: one complex component (8 n^3 bytes).
    """
    if kmax is None:
        kmax = n // 3
    if n > 4096:
        raise ValueError("n <= 4096")
    dev = torch.device(device)
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    rdt = torch.float64 if dtype == torch.float64 else torch.float32
    k1 = torch.fft.fftfreq(n, d=1.0 / n, device=dev, dtype=rdt)
    kz_host = np.fft.fftfreq(n, d=1.0 / n)
    ky = k1.view(n, 1)
    kx = k1.view(1, n)
    kin = ky * ky + kx * kx
    out = torch.empty((ncomp, n, n, n), device=dev, dtype=dtype)
    spec = torch.empty((n, n, n), device=dev, dtype=cdt)
    gen = torch.Generator(device=dev)
    for c in range(ncomp):
        for iz in range(n):
            kz = float(kz_host[iz])
            if abs(kz) > kmax:
                spec[iz].zero_()
                continue
            k2 = kin + kz * kz
            mask = (k2 >= 1) & (k2 <= kmax * kmax)
            amp = torch.where(mask, torch.sqrt(k2.clamp(min=1)).pow(-11.0 / 6.0),
                              torch.zeros_like(k2))
            gen.manual_seed((int(seed) << 12) + iz)
            a = torch.complex(torch.randn((3, n, n), generator=gen, device=dev, dtype=rdt),
                              torch.randn((3, n, n), generator=gen, device=dev, dtype=rdt))
            kd = (kx * a[0] + ky * a[1] + kz * a[2]) / k2.clamp(min=1)
            kv = (kx, ky, kz)
            ac = a[c % 3] - kv[c % 3] * kd
            others = [a[d] - kv[d] * kd for d in range(3)]
            norm = torch.sqrt(sum((o.real ** 2 + o.imag ** 2) for o in others)).clamp(min=1e-30)
            spec[iz] = ac * (amp / norm)
        for z0 in range(0, n, chunk):
            spec[z0:z0 + chunk] = torch.fft.ifft2(spec[z0:z0 + chunk], dim=(1, 2))
        for y0 in range(0, n, chunk):
            spec[:, y0:y0 + chunk] = torch.fft.ifft(spec[:, y0:y0 + chunk], dim=0)
        ss = 0.0
        for z0 in range(0, n, chunk):
            ss += float((spec[z0:z0 + chunk].real.double() ** 2).sum())
        rms = math.sqrt(ss / float(n) ** 3)
        for z0 in range(0, n, chunk):
            out[c, z0:z0 + chunk] = (spec[z0:z0 + chunk].real / rms).to(dtype)
    del spec
    return out


def uniform_particles(np_: int, seed: int = 2000, L: float = TWO_PI) -> np.ndarray:
    """[3][np] FP64 positions, i.i.d. uniform on [0, L)^3 (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return rng.random((3, int(np_)), dtype=np.float64) * L


def random_field(n, ncomp=3, seed=0, dtype=np.float64) -> np.ndarray:
    """Unstructured Gaussian field [ncomp][nz][ny][nx] for small parity cases.
    `n` is an int or (nx, ny, nz)."""
    if isinstance(n, int):
        n = (n, n, n)
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return rng.standard_normal((ncomp, nz, ny, nx)).astype(dtype)


def batch_sizes(nfields=48, seed=3000, sizes=(64, 96, 128, 192, 256),
                np_lo=10_000, np_hi=2_000_000):
    """Grid edge and particle count per field for the many-fields workload:
    edges uniform over `sizes`, particle counts log-uniform in [np_lo, np_hi]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    edges = rng.choice(np.array(sizes), size=nfields)
    nps = np.exp(rng.uniform(math.log(np_lo), math.log(np_hi), size=nfields))
    return [int(e) for e in edges], [int(round(v)) for v in nps]
