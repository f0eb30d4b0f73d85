"""Seeded synthetic inputs for multi-coil Cartesian SENSE.

This module only draws inputs: ellipse phantoms, coil sensitivity maps,
Cartesian line masks, complex Gaussian noise and the instance mix of the
uneven-batching workload.  It holds none of the reconstruction arithmetic
(no transform, no encoding operator), so the FP64 oracle and the CUDA
library can both be fed from it without sharing any of the method.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.

Readings (the paper, arXiv 1807.11830, prints no phantom or coil model; its
case study, Sec. IV, uses scanner data that is not available):

* coordinates are normalised to [-1, 1) on each axis, centre at (n/2, n/2);
* an ellipse has centre U(-0.5, 0.5)^2, semi-axes U(0.1, 0.45), angle
  U(0, pi) and complex value a*exp(i phi), a ~ U(0.2, 1), phi ~ U(-pi, pi);
  overlapping ellipses add; cine frames scale every semi-axis by
  1 + 0.15 sin(2 pi t / 20);
* coil c has a Gaussian magnitude (sigma = 0.4 n) centred on a ring of
  radius n/2 around the image centre at angle 2 pi c / C, times a linear
  phase ramp pi((x - n/2) cos th + (y - n/2) sin th)/n; the maps are then
  divided pointwise by sqrt(sum_c |S_c|^2), in float64;
* k-space is stored uncentred (DC at row 0), so the fully sampled centre
  lines are rows {0 .. Lc/2-1} and {ny-Lc/2 .. ny-1}; the remaining L-Lc rows
  are drawn uniformly without replacement from the others; lines are sorted;
* complex Gaussian noise of level sigma has real and imaginary parts
  N(0, sigma^2/2) each, so E|n|^2 = sigma^2.
"""
from dataclasses import dataclass

import numpy as np

BASE_SEED = 1807


def rng_for(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    theta: float
    value: complex


def draw_ellipses(count, rng):
    out = []
    for _ in range(count):
        cx, cy = rng.uniform(-0.5, 0.5, size=2)
        a, b = rng.uniform(0.1, 0.45, size=2)
        theta = rng.uniform(0.0, np.pi)
        amp = rng.uniform(0.2, 1.0)
        phi = rng.uniform(-np.pi, np.pi)
        out.append(Ellipse(cx, cy, a, b, theta, amp * np.exp(1j * phi)))
    return out


def _grid(ny, nx):
    v = (np.arange(ny) - ny / 2.0) / (ny / 2.0)
    u = (np.arange(nx) - nx / 2.0) / (nx / 2.0)
    return np.meshgrid(u, v)  # U[y][x], V[y][x]


def render(ellipses, ny, nx, scale=1.0):
    U, V = _grid(ny, nx)
    img = np.zeros((ny, nx), np.complex128)
    for e in ellipses:
        du, dv = U - e.cx, V - e.cy
        c, s = np.cos(e.theta), np.sin(e.theta)
        p = (du * c + dv * s) / (e.a * scale)
        q = (-du * s + dv * c) / (e.b * scale)
        img[p * p + q * q <= 1.0] += e.value
    return img


def phantom(ny, nx, count, rng, frames=1, period=None):
    """[frames][ny][nx] complex128; with ``period`` the semi-axes of every
    ellipse follow 1 + 0.15 sin(2 pi t / period)."""
    ells = draw_ellipses(count, rng)
    out = np.empty((frames, ny, nx), np.complex128)
    for t in range(frames):
        scale = 1.0 if period is None else 1.0 + 0.15 * np.sin(2.0 * np.pi * t / period)
        out[t] = render(ells, ny, nx, scale)
    return out


def sensitivities(coils, ny, nx):
    """[coils][ny][nx] complex128 with sum_c |S_c|^2 == 1 (float64)."""
    n = float(max(ny, nx))
    sigma = 0.4 * n
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    S = np.empty((coils, ny, nx), np.complex128)
    for c in range(coils):
        th = 2.0 * np.pi * c / coils
        cx = nx / 2.0 + (nx / 2.0) * np.cos(th)
        cy = ny / 2.0 + (ny / 2.0) * np.sin(th)
        mag = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * sigma * sigma))
        ph = np.pi * ((x - nx / 2.0) * np.cos(th) + (y - ny / 2.0) * np.sin(th)) / n
        S[c] = mag * np.exp(1j * ph)
    S /= np.sqrt(np.sum(np.abs(S) ** 2, axis=0))[None]
    return S


def centre_rows(ny, n_centre):
    h = n_centre // 2
    return sorted(set(range(0, h)) | set(range(ny - (n_centre - h), ny)))


def mask_lines(ny, L, n_centre, frames, rng):
    """[frames][L] int32, sorted, each frame drawn afresh."""
    if not (0 <= n_centre <= L <= ny):
        raise ValueError("need 0 <= n_centre <= L <= ny")
    centre = centre_rows(ny, n_centre)
    rest = np.array([r for r in range(ny) if r not in set(centre)], np.int64)
    out = np.empty((frames, L), np.int32)
    for f in range(frames):
        extra = rng.choice(rest, size=L - len(centre), replace=False) if L > len(centre) else []
        out[f] = np.sort(np.concatenate([np.array(centre, np.int64), np.asarray(extra, np.int64)]))
    return out


def full_lines(ny, frames):
    return np.tile(np.arange(ny, dtype=np.int32), (frames, 1))


def centred_lines(lines, ny):
    """The same sampled frequencies in centred k-space indexing (DC at ny/2):
    row k becomes (k + ny/2) mod ny, sorted per frame."""
    return np.sort((np.asarray(lines, np.int64) + ny // 2) % ny, axis=1).astype(np.int32)


def complex_noise(shape, sigma, rng):
    s = sigma / np.sqrt(2.0)
    return rng.normal(0.0, s, size=shape) + 1j * rng.normal(0.0, s, size=shape)


def lines_for_acceleration(n, R):
    return int(round(n / R))


def centre_for(n):
    return max(8, n // 16)


@dataclass
class Problem:
    """One SENSE instance: the true images, the maps, the lines and the
    noise to add to E x.  k-space itself is made by whichever forward
    operator the caller trusts (the oracle in tests)."""
    name: str
    x_true: np.ndarray   # [F][ny][nx] complex128
    S: np.ndarray        # [C][ny][nx] complex128
    lines: np.ndarray    # [F][L] int32
    noise: np.ndarray    # [F][C][L][nx] complex128
    iters: int

    @property
    def shape(self):
        F, ny, nx = self.x_true.shape
        return dict(frames=F, coils=self.S.shape[0], ny=ny, nx=nx, lines=self.lines.shape[1])


def single_slice_64(seed=BASE_SEED + 0, noise_sigma=1e-3):
    """64x64, 10 ellipses, 4 coils, 8 centre lines + random lines to 33 %,
    noise 1e-3, 10 CG iterations."""
    rng = rng_for(seed)
    n, C = 64, 4
    x = phantom(n, n, 10, rng)
    S = sensitivities(C, n, n)
    L = int(round(0.33 * n))
    lines = mask_lines(n, L, 8, 1, rng)
    nz = complex_noise((1, C, L, n), noise_sigma, rng)
    return Problem("single-slice 64x64 C4 L21", x, S, lines, nz, 10)


def cine_256(seed=BASE_SEED + 1, frames=20, noise_sigma=1e-3):
    """256x256 x 20 frames, radii modulated by sin(2 pi t/20), 12 coils,
    acceleration 4 (L = 64, 16 centre lines, fresh lines per frame), 30 CG
    iterations."""
    rng = rng_for(seed)
    n, C = 256, 12
    x = phantom(n, n, 10, rng, frames=frames, period=20)
    S = sensitivities(C, n, n)
    lines = mask_lines(n, lines_for_acceleration(n, 4), 16, frames, rng)
    nz = complex_noise((frames, C, lines.shape[1], n), noise_sigma, rng)
    return Problem("cine 256x256 F%d C12 R4" % frames, x, S, lines, nz, 30)


def slices_320(seed=BASE_SEED + 2, frames=16, noise_sigma=1e-3):
    """320x320 x 16 slices, 32 coils, acceleration 3 (L = 107, 24 centre
    lines), 50 CG iterations."""
    rng = rng_for(seed)
    n, C = 320, 32
    x = phantom(n, n, 10, rng, frames=frames)
    S = sensitivities(C, n, n)
    lines = mask_lines(n, lines_for_acceleration(n, 3), 24, frames, rng)
    nz = complex_noise((frames, C, lines.shape[1], n), noise_sigma, rng)
    return Problem("slices 320x320 F%d C32 R3" % frames, x, S, lines, nz, 50)


MIX_SIZES = (128, 192, 256, 384)
MIX_ACCEL = (2, 3, 4, 6)


def paper_160(seed=BASE_SEED + 5, frames=16, noise_sigma=1e-3):
    """The shapes of the timed reconstruction of Sec. IV-B (16 cine frames of
    160x160, 8 coils, fully sampled Cartesian k-space), with 10-ellipse
    phantoms; it feeds the 2D inverse FFT + root-sum-of-squares and the
    Eq. 1 combine."""
    rng = rng_for(seed)
    n, C = 160, 8
    x = phantom(n, n, 10, rng, frames=frames, period=frames)
    S = sensitivities(C, n, n)
    lines = full_lines(n, frames)
    nz = complex_noise((frames, C, n, n), noise_sigma, rng)
    return Problem("paper 160x160 F%d C8 full" % frames, x, S, lines, nz, 0)


def draw_mix(count=512, seed=BASE_SEED + 3):
    """Instance shapes of the uneven-batching workload: n from
    {128,192,256,384}, coils U{8..32}, frames U{1..30}, R from {2,3,4,6}."""
    rng = rng_for(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(MIX_SIZES))
        C = int(rng.integers(8, 33))
        F = int(rng.integers(1, 31))
        R = int(rng.choice(MIX_ACCEL))
        out.append(dict(n=n, coils=C, frames=F, accel=R, lines=lines_for_acceleration(n, R),
                        centre=centre_for(n)))
    return out


def mix_instance(spec, seed):
    """Materialise one instance of the mix (phantom, maps, lines, noise)."""
    rng = rng_for(seed)
    n, C, F = spec["n"], spec["coils"], spec["frames"]
    x = phantom(n, n, 10, rng, frames=F, period=20 if F > 1 else None)
    S = sensitivities(C, n, n)
    lines = mask_lines(n, spec["lines"], spec["centre"], F, rng)
    nz = complex_noise((F, C, spec["lines"], n), 1e-3, rng)
    return Problem("mix n%d C%d F%d R%d" % (n, C, F, spec["accel"]), x, S, lines, nz, 20)


def poisson_arrivals(rate_hz, count, seed):
    """Arrival times (s) of a Poisson stream: exponential gaps of mean 1/rate."""
    rng = rng_for(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))


def random_complex(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
