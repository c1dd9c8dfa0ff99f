"""Seeded synthetic inputs for damped Helmholtz problems.

This module builds the *inputs* of a problem -- the grid, the wave speed per
cell c, the damping per node R, the physical angular frequency and the
right-hand side F -- and nothing of the method itself.  Both the CUDA path and
the CPU oracle are fed from here, so it must not hold any of the method's
arithmetic (no stencil, no recurrence, no parameter selection).

Problem statement (Stolk, Sec. 1, damped Helmholtz equation):
    -Delta U - (omega/c)^2 U + i omega R U = F,   zero Dirichlet data,
with e^{+i omega t} time dependence.

Grid reading: an ``n x n (x n)`` grid holds n unknown nodes per axis at
x_i = i*h, i = 0..n-1; the ring at i = -1 and i = n is a zero ghost ring.
c is given per cell (lower-corner index a = -1..n-1, stored at a+1), so it has
(n+1)^d values; R is given per node (n^d values).

Random fields: splitmix64 -> uniforms -> Box-Muller white noise, smoothed by a
separable Gaussian of standard deviation sigma = correlation length
(truncated at 4 sigma, zero padding), then normalised to zero mean and unit
standard deviation.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` outputs of the splitmix64 generator started at ``seed``.

    Published definition (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15;
    z = state; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB; return z ^ (z >> 31).
    """
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
             + k * np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def white_noise(seed: int, shape) -> np.ndarray:
    """Standard normal samples by the Box-Muller transform (cosine branch)."""
    count = int(np.prod(shape))
    u = uniform01(seed, 2 * count)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.reshape(shape)


def gaussian_smooth(field: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Separable Gaussian smoothing, kernel truncated at 4 sigma, zero padding.

    Each axis is convolved (linear, not circular) by FFT with the normalised
    kernel exp(-x^2 / (2 sigma^2)), x = -r..r, r = ceil(4 sigma).
    """
    r = max(1, int(math.ceil(4.0 * sigma_cells)))
    x = np.arange(-r, r + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (x / sigma_cells) ** 2)
    ker /= ker.sum()
    out = field.astype(np.float64)
    for ax in range(out.ndim):
        m = out.shape[ax]
        L = m + 2 * r
        nfft = 1 << (L - 1).bit_length()
        fk = np.fft.rfft(ker, nfft)
        fo = np.fft.rfft(out, nfft, axis=ax)
        shape = [1] * out.ndim
        shape[ax] = fk.shape[0]
        conv = np.fft.irfft(fo * fk.reshape(shape), nfft, axis=ax)
        out = np.take(conv, np.arange(r, r + m), axis=ax)
    return out


def gaussian_random_field(seed: int, shape, corr_len_cells: float) -> np.ndarray:
    """Zero-mean, unit-std smooth Gaussian field on ``shape``."""
    g = gaussian_smooth(white_noise(seed, shape), corr_len_cells)
    g -= g.mean()
    s = g.std()
    return g / s if s > 0 else g


def layer_depth(n: int, w: int) -> np.ndarray:
    """Distance into an absorbing layer of ``w`` cells on both ends of an axis.

    d(i) = max(0, w - min(i, n-1-i)) for nodes i = 0..n-1.
    """
    i = np.arange(n)
    return np.maximum(0, w - np.minimum(i, n - 1 - i)).astype(np.float64)


def damping_profile(ndim: int, n, w: int, R0: float) -> np.ndarray:
    """R(x) = R0 * sum over axes of (d_axis / w)^2 on all faces, per node."""
    n = list(n)
    R = np.zeros(n, dtype=np.float64)
    for ax in range(ndim):
        d = (layer_depth(n[ax], w) / w) ** 2
        shape = [1] * ndim
        shape[ax] = n[ax]
        R = R + R0 * d.reshape(shape)
    return R


def point_source(ndim: int, n, h: float, pos=None, amplitude=None) -> np.ndarray:
    """Complex right-hand side with one nonzero entry 1/h^d (default at the centre node)."""
    n = list(n)
    F = np.zeros(n, dtype=np.complex128)
    if pos is None:
        pos = tuple((m - 1) // 2 for m in n)
    F[tuple(pos)] = (1.0 / h ** ndim) if amplitude is None else amplitude
    return F


def random_rhs(seed: int, n) -> np.ndarray:
    """Dense complex right-hand side with standard normal real and imaginary parts."""
    n = list(n)
    z = white_noise(seed, [2] + n)
    return z[0] + 1j * z[1]


@dataclasses.dataclass
class Problem:
    """Inputs of one damped Helmholtz problem (host arrays, float64/complex128)."""
    name: str
    ndim: int
    n: tuple
    h: float
    c_cell: np.ndarray      # shape tuple(m + 1 for m in n)
    R_node: np.ndarray      # shape n
    omega: float            # physical angular frequency
    F: np.ndarray           # complex128, shape n
    T: int                  # periods per preconditioner application
    rho: float = 0.25       # window parameter

    @property
    def N(self) -> int:
        return int(np.prod(self.n))


def periods_for(n_side: int, h: float, c_min: float, omega: float) -> int:
    """T = ceil(side length in wavelengths at the slowest speed)."""
    wavelength = 2.0 * math.pi * c_min / omega
    return max(1, int(math.ceil((n_side - 1) * h / wavelength - 1e-9)))


def config_2d_constant(n: int = 101, ppw: float = 10.0, layer: int = 20,
                       T: int | None = None, rho: float = 0.25) -> Problem:
    """2-D unit square, constant c = 1, n x n nodes, h = 1/(n-1), ``ppw`` points per
    wavelength, ``layer``-cell absorbing layer with R0 = 2 omega, centre point source.
    n = 101 is the 101x101, h = 0.01, omega = 2 pi 10 case."""
    h = 1.0 / (n - 1)
    omega = 2.0 * math.pi / (ppw * h)
    c = np.ones((n + 1, n + 1))
    R = damping_profile(2, (n, n), layer, 2.0 * omega)
    F = point_source(2, (n, n), h)
    if T is None:
        T = periods_for(n, h, 1.0, omega)
    return Problem(f"2d_const_{n}", 2, (n, n), h, c, R, omega, F, T, rho)


def config_2d_heterogeneous(n: int = 1001, layer: int = 40, seed: int = 2006168611,
                            corr_len: float = 0.05, ppw: float = 8.0,
                            T: int | None = None, rho: float = 0.25) -> Problem:
    """2-D unit square, n x n nodes, h = 1/(n-1); c = clip(3 + 0.75 g, 1.5, 4.5) with g a
    Gaussian random field of correlation length ``corr_len``; omega for ``ppw`` points per
    wavelength at the minimum c; ``layer``-cell absorbing layer (R0 = 2 omega); one
    point source at the centre."""
    h = 1.0 / (n - 1)
    g = gaussian_random_field(seed, (n + 1, n + 1), corr_len / h)
    c = np.clip(3.0 + 0.75 * g, 1.5, 4.5)
    cmin = float(c.min())
    omega = 2.0 * math.pi * cmin / (ppw * h)
    R = damping_profile(2, (n, n), layer, 2.0 * omega)
    F = point_source(2, (n, n), h)
    if T is None:
        T = periods_for(n, h, cmin, omega)
    return Problem(f"2d_grf_{n}", 2, (n, n), h, c, R, omega, F, T, rho)


def layered_speed(n: int, seed: int, corr_len: float,
                  layers=(1.5, 2.5, 3.5, 4.5), perturb: float = 0.1) -> np.ndarray:
    """3-D speed per cell: 4 horizontal layers along axis 0 (depth quartiles of the cell
    centres) times (1 + perturb * g), g a unit Gaussian random field."""
    h = 1.0 / (n - 1)
    m = n + 1
    centre = (np.arange(m) - 0.5) * h           # cell a (stored a+1) centre at (a+0.5)h
    q = np.clip(np.floor(centre * len(layers)).astype(int), 0, len(layers) - 1)
    base = np.asarray(layers, dtype=np.float64)[q]
    g = gaussian_random_field(seed, (m, m, m), corr_len / h)
    return base[:, None, None] * (1.0 + perturb * g)


def config_3d_layered(n: int = 256, layer: int = 24, seed: int = 2006168612,
                      corr_len: float = 0.05, ppw: float = 8.0,
                      T: int | None = None, rho: float = 0.25) -> Problem:
    """3-D unit cube, n^3 nodes, h = 1/(n-1); 4 layers [1.5, 2.5, 3.5, 4.5] times a 10%
    Gaussian perturbation; omega for ``ppw`` points per wavelength at the minimum c;
    ``layer``-cell absorbing layer (R0 = 2 omega); centre point source."""
    h = 1.0 / (n - 1)
    c = layered_speed(n, seed, corr_len)
    cmin = float(c.min())
    omega = 2.0 * math.pi * cmin / (ppw * h)
    R = damping_profile(3, (n, n, n), layer, 2.0 * omega)
    F = point_source(3, (n, n, n), h)
    if T is None:
        T = periods_for(n, h, cmin, omega)
    return Problem(f"3d_layered_{n}", 3, (n, n, n), h, c, R, omega, F, T, rho)


@dataclasses.dataclass
class InversionSetup:
    """Sources, receivers and data for a receiver-misfit problem."""
    prob: Problem               # the model the misfit is evaluated at
    F: np.ndarray               # (nsrc, *n) complex right-hand sides
    rec_idx: np.ndarray         # int64 node linear indices of the receivers
    c_true: np.ndarray          # per-cell speed the data would come from


def seeded_sources(seed: int, ndim: int, n, h: float, nsrc: int, margin: int) -> np.ndarray:
    """nsrc point sources (amplitude 1/h^d) at seeded uniform node positions at
    least `margin` nodes from every face."""
    n = list(n)
    u = uniform01(seed, nsrc * ndim).reshape(nsrc, ndim)
    F = np.zeros([nsrc] + n, dtype=np.complex128)
    for s in range(nsrc):
        pos = tuple(int(margin + u[s, a] * (n[a] - 2 * margin)) for a in range(ndim))
        F[(s,) + pos] = 1.0 / h ** ndim
    return F


def top_row_receivers(n, row: int, margin: int) -> np.ndarray:
    """Linear node indices of the receivers on row `row` (axis 0) of a 2-D grid,
    columns margin .. n1 - 1 - margin."""
    cols = np.arange(margin, n[1] - margin)
    return (row * n[1] + cols).astype(np.int64)


def gaussian_blob(n_cells, h: float, centre, sigma: float, amplitude: float) -> np.ndarray:
    """1 + amplitude * exp(-|x - centre|^2 / (2 sigma^2)) at the cell centres."""
    axes = [(np.arange(m) - 0.5) * h for m in n_cells]
    grids = np.meshgrid(*axes, indexing="ij")
    r2 = sum((g - c0) ** 2 for g, c0 in zip(grids, centre))
    return 1.0 + amplitude * np.exp(-0.5 * r2 / sigma ** 2)


def config_adjoint(n: int = 512, nsrc: int = 8, layer: int = 20, seed: int = 2006168615,
                   corr_len: float = 0.05, ppw: float = 8.0, T: int | None = None,
                   rho: float = 0.25) -> InversionSetup:
    """2-D n x n model with a smooth random c (clip(3 + 0.75 g, 1.5, 4.5)), omega for
    `ppw` points per wavelength at min c, `layer`-cell absorbing layer (R0 = 2 omega),
    `nsrc` seeded point sources, receivers on the first row inside the top absorbing
    layer, and a 'true' model c * (1 + 5% Gaussian blob, sigma 0.1, at the centre)."""
    h = 1.0 / (n - 1)
    g = gaussian_random_field(seed, (n + 1, n + 1), corr_len / h)
    c = np.clip(3.0 + 0.75 * g, 1.5, 4.5)
    cmin = float(c.min())
    omega = 2.0 * math.pi * cmin / (ppw * h)
    R = damping_profile(2, (n, n), layer, 2.0 * omega)
    F = seeded_sources(seed + 1, 2, (n, n), h, nsrc, layer + 2)
    if T is None:
        T = periods_for(n, h, cmin, omega)
    prob = Problem(f"2d_adjoint_{n}", 2, (n, n), h, c, R, omega, F[0], T, rho)
    c_true = c * gaussian_blob((n + 1, n + 1), h, (0.5, 0.5), 0.1, 0.05)
    rec = top_row_receivers((n, n), layer, layer)
    return InversionSetup(prob, F, rec, c_true)


@dataclasses.dataclass
class BatchSetup:
    """Independent systems run as one batch: instance i is the problem probs[i]
    with the right-hand sides F[i] (shape (nrhs_i, *n_i))."""
    probs: list
    F: list


def config_batched(n3: int = 128, nsrc: int = 32, ninst: int = 64, side_lo: int = 200,
                   side_hi: int = 1000, seed: int = 2006168614, ppw: float = 8.0,
                   rho: float = 0.25) -> BatchSetup:
    """The 3-D layered model at n3^3 (absorbing layer 24 cells per 256, so the same
    physical width) with `nsrc` seeded point sources as right-hand sides, plus
    `ninst` 2-D instances whose sides are drawn uniformly from [side_lo, side_hi]:
    smooth random c = clip(3 + 0.75 g, 1.5, 4.5) (correlation length 0.05, own
    seed per instance), omega for `ppw` points per wavelength at its min c, an
    absorbing layer of 4 % of the side (R0 = 2 omega) and a centre point source."""
    layer3 = max(2, int(round(24 * n3 / 256)))
    p3 = config_3d_layered(n3, layer=layer3, seed=seed - 2, ppw=ppw, rho=rho)
    F3 = seeded_sources(seed, 3, p3.n, p3.h, nsrc, layer3 + 2)
    probs, Fs = [p3], [F3]
    u = uniform01(seed + 1, ninst)
    for i in range(ninst):
        side = side_lo + int(u[i] * (side_hi - side_lo + 1))
        side = min(side, side_hi)
        layer = max(4, int(round(0.04 * (side - 1))))
        p = config_2d_heterogeneous(side, layer=layer, seed=seed + 100 + i, ppw=ppw, rho=rho)
        probs.append(p)
        Fs.append(p.F[None].astype(np.complex128))
    return BatchSetup(probs, Fs)


def config_3d_paper_shape(shape=(106, 200, 200), ppw: float = 6.0, T: int = 25, layer: int = 16,
                          seed: int = 2006168616, corr_len: float = 0.05,
                          rho: float = 0.25) -> Problem:
    """The size of the paper's smallest 3-D example (200 x 200 x 106 nodes, depth
    along axis 0) at 6 points per wavelength and T = 25, with the 4-layer model of
    config_3d_layered standing in for the unavailable SEG/EAGE salt model (h from
    the longest side, layers by depth, 10 % Gaussian perturbation);
    ``layer``-cell absorbing layer (R0 = 2 omega) and a centre point source."""
    n = tuple(int(m) for m in shape)
    h = 1.0 / (max(n) - 1)
    cells = tuple(m + 1 for m in n)
    depth = (np.arange(cells[0]) - 0.5) / (n[0] - 1)
    layers = np.asarray((1.5, 2.5, 3.5, 4.5))
    q = np.clip(np.floor(depth * len(layers)).astype(int), 0, len(layers) - 1)
    g = gaussian_random_field(seed, cells, corr_len / h)
    c = layers[q][:, None, None] * (1.0 + 0.1 * g)
    cmin = float(c.min())
    omega = 2.0 * math.pi * cmin / (ppw * h)
    R = damping_profile(3, n, layer, 2.0 * omega)
    F = point_source(3, n, h)
    return Problem("3d_paper_shape", 3, n, h, c, R, omega, F, T, rho)
