"""The seeded synthetic inputs have the recipe stated for them (CPU only).

The generators hold none of the merge-tree arithmetic; these tests pin that
each produces what its docstring says: determinism per seed, value ranges,
standardisation, the power-spectrum slope of the Gaussian random fields
(fitted over the radially averaged spectrum), the quantisation levels, the
lognormal transform, and the batch and serving streams."""

from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2301_10838_gb300 import fields


def test_white_noise_is_seeded_uniform_float32():
    a = fields.white_noise((16, 20, 24), 3)
    b = fields.white_noise((16, 20, 24), 3)
    c = fields.white_noise((16, 20, 24), 4)
    assert a.dtype == np.float32 and a.shape == (16, 20, 24)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(float(a.mean()) - 0.5) < 0.01 and abs(float(a.var()) - 1 / 12) < 0.005


def _spectral_slope(g):
    """Least-squares slope of log P(|k|) against log |k| over radial bins."""
    n = g.shape[0]
    p = np.abs(np.fft.fftn(g)) ** 2
    k = np.sqrt(sum(np.meshgrid(*(np.fft.fftfreq(n) ** 2,) * 3, indexing="ij")))
    edges = np.linspace(1.5 / n, 0.45, 20)
    ks, ps = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (k >= lo) & (k < hi)
        if m.any():
            ks.append(float(k[m].mean()))
            ps.append(float(p[m].mean()))
    return float(np.polyfit(np.log(ks), np.log(ps), 1)[0])


@pytest.mark.parametrize("slope", [-2.0, -2.5, -3.0])
def test_grf_spectrum_and_standardisation(slope):
    g = fields.grf((64, 64, 64), slope, seed=2)
    assert abs(float(g.mean())) < 1e-9 and abs(float(g.std(ddof=1)) - 1.0) < 1e-9  # torch standardises with n - 1
    assert abs(_spectral_slope(g) - slope) < 0.15
    assert np.array_equal(g, fields.grf((64, 64, 64), slope, seed=2))


def test_quantize_levels_and_range():
    g = fields.grf((32, 32, 32), -3.0, seed=5)
    q = fields.quantize(g, levels=64)
    assert q.dtype == np.float32 and float(q.min()) == 0.0 and float(q.max()) == 1.0
    vals = np.unique(q)
    assert len(vals) <= 64
    assert np.allclose(vals * 63, np.rint(vals * 63), atol=1e-4)  # on the grid of 63rds


def test_lognormal_is_exp_of_a_unit_grf():
    f = fields.lognormal((48, 48, 48), seed=3, sigma=0.8, slope=-2.0)
    assert f.dtype == np.float32 and float(f.min()) > 0.0
    g = np.log(f.astype(np.float64)) / 0.8
    assert abs(float(g.mean())) < 1e-5 and abs(float(g.std(ddof=1)) - 1.0) < 1e-5
    assert np.allclose(g, fields.grf((48, 48, 48), -2.0, seed=3), atol=1e-5)


def test_named_fields():
    assert fields.named_field("white64", seed=1).shape == (64, 64, 64)
    q = fields.named_field("grf256q12", seed=1, side=32)
    assert q.shape == (32, 32, 32) and len(np.unique(q)) <= 4096
    assert fields.named_field("lognorm1024", seed=1, side=24).shape == (24, 24, 24)
    with pytest.raises(KeyError):
        fields.named_field("nope")


def test_batch_shapes_are_log_uniform_and_uneven():
    shapes = fields.batch_shapes(512, 16, 128, seed=7)
    assert shapes == fields.batch_shapes(512, 16, 128, seed=7)
    sides = np.array(shapes)
    assert sides.min() >= 16 and sides.max() <= 128
    logs = np.log(sides.astype(np.float64))
    mid = (math.log(16) + math.log(128)) / 2
    assert abs(float(logs.mean()) - mid) < 0.05  # log-uniform: mean at the middle of the log range
    assert any(a != b for a, b, _ in shapes) and any(s[2] % 2 == 1 for s in shapes)
    assert fields.batch_field(3, (5, 6, 7)).dtype == np.float32  # white half
    assert fields.batch_field(300, (8, 9, 10)).dtype == np.float32  # GRF half


def test_serve_stream_is_poisson_at_the_rate():
    reqs = fields.serve_stream(rate_hz=200.0, duration_s=10.0, lo=32, hi=384, seed=11)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 10.0
    assert abs(len(reqs) - 2000) < 4 * math.sqrt(2000)  # Poisson count
    gaps = np.diff(t)
    assert abs(float(gaps.mean()) - 1 / 200) < 0.0005 and abs(float(gaps.std() / gaps.mean()) - 1.0) < 0.1
    sides = np.array([r.side for r in reqs])
    assert sides.min() >= 32 and sides.max() <= 384
    thr = np.array([r.threshold for r in reqs])
    assert thr.min() >= -2.0 and thr.max() <= 2.0
