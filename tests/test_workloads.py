"""The seeded input recipes (paper_2006_16861_gb300/workloads.py) against their
stated definitions: the generator, the field statistics, the speed models,
the absorbing layer, the sources and the configuration sizes."""
import math

import numpy as np
import pytest

from paper_2006_16861_gb300 import workloads as W

M64 = (1 << 64) - 1


def splitmix64_ref(seed, count):
    """splitmix64 from its published definition, in Python integers."""
    out, state = [], seed & M64
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2006168611, (1 << 64) - 5])
def test_splitmix64_matches_definition(seed):
    got = [int(v) for v in W.splitmix64(seed, 17)]
    assert got == splitmix64_ref(seed, 17)


def test_uniform_and_normal_samples():
    u = W.uniform01(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = W.white_noise(8, (400, 500))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert np.array_equal(W.white_noise(8, (400, 500)), z)       # seeded: reproducible
    assert not np.array_equal(W.white_noise(9, (400, 500)), z)


def test_gaussian_smoothing_is_a_normalised_truncated_convolution():
    """An impulse is smoothed into the normalised Gaussian kernel truncated at
    4 sigma (zero padding at the borders)."""
    f = np.zeros(61)
    f[30] = 1.0
    g = W.gaussian_smooth(f, 3.0)
    x = np.arange(61) - 30
    ker = np.where(np.abs(x) <= 12, np.exp(-0.5 * (x / 3.0) ** 2), 0.0)
    assert np.allclose(g, ker / ker.sum(), atol=1e-14)
    assert g.sum() == pytest.approx(1.0, abs=1e-13)


def test_random_field_is_zero_mean_unit_std():
    g = W.gaussian_random_field(3, (120, 140), 6.0)
    assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.0, abs=1e-12)


def test_heterogeneous_2d_model():
    p = W.config_2d_heterogeneous(201, layer=10, T=3)
    assert p.c_cell.shape == (202, 202) and p.R_node.shape == (201, 201)
    assert p.c_cell.min() >= 1.5 and p.c_cell.max() <= 4.5
    assert p.h == pytest.approx(1 / 200)
    ppw = 2 * math.pi * p.c_cell.min() / (p.omega * p.h)
    assert ppw == pytest.approx(8.0, rel=1e-12)                      # 8 points per wavelength
    F = np.zeros_like(p.F)
    F[100, 100] = 1 / p.h ** 2                                       # centre source, 1/h^2
    assert np.array_equal(p.F, F)


def test_layered_3d_model():
    p = W.config_3d_layered(40, layer=4, T=2)
    c = p.c_cell
    nz = c.shape[0]
    for q, base in enumerate((1.5, 2.5, 3.5, 4.5)):
        z0 = int(math.ceil(q * nz / 4)) + 1
        z1 = int((q + 1) * nz / 4) - 1
        sl = c[z0:z1]
        assert sl.size and np.all(np.abs(sl / base - 1.0) <= 0.1 * 6)   # 10 % perturbation
        assert abs(np.median(sl) / base - 1.0) < 0.05


def test_absorbing_layer_profile():
    w, R0, n = 5, 7.0, (16, 13)
    R = W.damping_profile(2, n, w, R0)
    assert np.all(R[w:n[0] - w, w:n[1] - w] == 0.0)                  # interior undamped
    assert R[0, 0] == pytest.approx(2 * R0)                          # corner: both axes, depth w
    assert R[0, 6] == pytest.approx(R0)                              # face: one axis, depth w
    assert R[2, 6] == pytest.approx(R0 * ((w - 2) / w) ** 2)
    assert np.allclose(R, R[::-1, ::-1])                             # symmetric on all faces


def test_seeded_sources_and_batched_configuration():
    F = W.seeded_sources(5, 3, (30, 31, 32), 0.1, 6, 4)
    assert F.shape == (6, 30, 31, 32)
    for f in F:
        idx = np.argwhere(f != 0)
        assert len(idx) == 1
        i = idx[0]
        assert np.all(i >= 4) and np.all(i <= np.array((30, 31, 32)) - 1 - 4)
    setup = W.config_batched(n3=24, nsrc=3, ninst=5, side_lo=40, side_hi=60)
    assert len(setup.probs) == 6 and setup.F[0].shape == (3, 24, 24, 24)
    assert all(40 <= p.n[0] <= 60 and p.n[0] == p.n[1] for p in setup.probs[1:])
    again = W.config_batched(n3=24, nsrc=3, ninst=5, side_lo=40, side_hi=60)
    assert all(np.array_equal(a.c_cell, b.c_cell) for a, b in zip(setup.probs, again.probs))


def test_periods_follow_the_side_in_wavelengths():
    p = W.config_2d_heterogeneous(1001)
    wl = 2 * math.pi * p.c_cell.min() / p.omega
    assert p.T == math.ceil(1.0 / wl - 1e-9) == 125
