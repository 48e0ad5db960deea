"""Seeded synthetic scalar fields on regular 3-D grids.

This module only draws inputs; it holds none of the merge-tree arithmetic.
Both the CUDA path and the CPU oracle consume the bytes it produces, so a
field is generated once and handed to both sides.

Array layout everywhere: C order ``[nz][ny][nx]``, x fastest, so the linear
index of vertex (x, y, z) is ``x + nx * (y + ny * z)``.

The paper evaluates on simulation and CT volumes (Section 4, "Datasets") that
are not available here; these generators stand in for them with the shapes
and value statistics of scientific fields:

* ``white_noise``  i.i.d. uniform[0, 1) float32 (many minima, short basins)
* ``grf``          Gaussian random field with power spectrum P(k) ~ k^slope
* ``quantize``     snap a field to a fixed number of levels (forces ties)
* ``lognormal``    exp(sigma * g) of a GRF g (density-like, heavy tail)
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "white_noise",
    "grf",
    "quantize",
    "lognormal",
    "named_field",
    "batch_shapes",
    "batch_field",
    "ServeRequest",
    "serve_stream",
]


def _shape3(shape) -> tuple[int, int, int]:
    if len(shape) != 3:
        raise ValueError("shape must be (nz, ny, nx)")
    nz, ny, nx = (int(s) for s in shape)
    if min(nz, ny, nx) < 1:
        raise ValueError("grid sides must be >= 1")
    return nz, ny, nx


def white_noise(shape, seed: int) -> np.ndarray:
    """i.i.d. uniform[0, 1) float32 values, shape (nz, ny, nx)."""
    return np.random.default_rng(seed).random(_shape3(shape), dtype=np.float32)


def grf(shape, slope: float, seed: int, device: str = "cpu"):
    """Gaussian random field with P(k) proportional to |k|**slope.

    Seeded N(0,1) white noise is filtered in Fourier space by the amplitude
    |k|**(slope/2) (k from ``fftfreq`` per axis, DC mode zeroed), transformed
    back and standardised to zero mean and unit variance.

    On the CPU the arithmetic is float64 and a float64 numpy array is
    returned; on a CUDA device it is float32 (the 1024^3 case needs ~13 GB)
    and a float32 torch tensor on that device is returned.
    """
    nz, ny, nx = _shape3(shape)
    import torch

    on_cpu = str(device) == "cpu"
    dt = torch.float64 if on_cpu else torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    noise = torch.randn((nz, ny, nx), generator=gen, dtype=dt, device=device)
    spec = torch.fft.rfftn(noise)
    del noise
    kz = torch.fft.fftfreq(nz, dtype=dt, device=device).view(nz, 1, 1)
    ky = torch.fft.fftfreq(ny, dtype=dt, device=device).view(1, ny, 1)
    kx = torch.fft.rfftfreq(nx, dtype=dt, device=device).view(1, 1, nx // 2 + 1)
    # amplitude |k|^(slope/2), built one z-slab at a time to bound memory
    for z0 in range(0, nz, 64):
        z1 = min(nz, z0 + 64)
        k2 = kz[z0:z1] ** 2 + ky**2 + kx**2
        amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** (slope / 4.0), torch.zeros_like(k2))
        spec[z0:z1] *= amp
    g = torch.fft.irfftn(spec, s=(nz, ny, nx))
    del spec
    g -= g.mean()
    std = g.std()
    if float(std) > 0:
        g /= std
    if on_cpu:
        return g.numpy()
    return g


def quantize(g, levels: int = 4096) -> np.ndarray:
    """Snap ``g`` to ``levels`` equally spaced values in [0, 1] (float32).

    q = round((levels-1) * (g - min) / (max - min)); value = q / (levels-1).
    """
    g = np.asarray(g, dtype=np.float64)
    lo, hi = float(g.min()), float(g.max())
    span = hi - lo if hi > lo else 1.0
    q = np.rint((levels - 1) * (g - lo) / span)
    return (q / (levels - 1)).astype(np.float32)


def lognormal(shape, seed: int, sigma: float = 0.8, slope: float = -2.0, device: str = "cpu"):
    """exp(sigma * g), g a unit-variance GRF with P(k) ~ k^slope (float32)."""
    g = grf(shape, slope, seed, device=device)
    if isinstance(g, np.ndarray):
        return np.exp(sigma * g).astype(np.float32)
    g.mul_(sigma).exp_()
    return g.to(dtype=__import__("torch").float32)


def named_field(name: str, seed: int = 1, side: int | None = None, device: str = "cpu"):
    """The benchmark workloads by name.

    ``white64``     64^3 white noise
    ``grf256q12``   256^3 GRF P(k)~k^-3 quantised to 4096 levels
    ``lognorm1024`` 1024^3 exp(0.8 g), g a GRF with P(k)~k^-2
    ``side`` overrides the cube side (used for scaled-down test copies).
    """
    if name == "white64":
        n = side or 64
        return white_noise((n, n, n), seed)
    if name == "grf256q12":
        n = side or 256
        g = grf((n, n, n), -3.0, seed, device="cpu")
        return quantize(g, 4096)
    if name == "lognorm1024":
        n = side or 1024
        return lognormal((n, n, n), seed, 0.8, -2.0, device=device)
    raise KeyError(name)


def batch_shapes(count: int = 512, lo: int = 16, hi: int = 128, seed: int = 7) -> list[tuple[int, int, int]]:
    """Uneven grid shapes: each side round(exp(U(ln lo, ln hi))), drawn per axis.

    Returns (nz, ny, nx) tuples; non-cubic shapes and odd nx occur.
    """
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=(count, 3))
    sides = np.rint(np.exp(u)).astype(np.int64)
    return [tuple(int(v) for v in row) for row in sides]


def batch_field(i: int, shape) -> np.ndarray:
    """Field ``i`` of the uneven batch: first half white noise, second half
    GRF P(k)~k^-3 (float32), each seeded with 1000 + i."""
    _shape3(shape)
    if (i % 512) < 256:
        return white_noise(shape, 1000 + i)
    return grf(shape, -3.0, 1000 + i, device="cpu").astype(np.float32)


@dataclass(frozen=True)
class ServeRequest:
    rid: int
    arrival_s: float  # seconds from stream start
    side: int  # cubic grid side
    seed: int
    threshold: float


def serve_stream(rate_hz: float = 200.0, duration_s: float = 10.0, lo: int = 32, hi: int = 384,
                 seed: int = 11) -> list[ServeRequest]:
    """Open-loop Poisson arrivals at ``rate_hz``; cubic sides log-uniform in
    [lo, hi]; thresholds U(-2, 2) (fields are unit-variance GRFs)."""
    rng = np.random.default_rng(seed)
    out: list[ServeRequest] = []
    t = 0.0
    rid = 0
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        thr = float(rng.uniform(-2.0, 2.0))
        out.append(ServeRequest(rid, t, side, 5000 + rid, thr))
        rid += 1
    return out
