"""Pins of the oracle's centred k-space convention (CPU only).

With `centred`, every transform of the oracle is fftshift . F . ifftshift
along each axis: DC and the image centre sit at index floor(n/2), and line
indices address that centred k-space (the paper leaves the convention open;
the uncentred one is the default).  The pins:
  * the textbook formula written out, X[k] = sum_j x[j] e^{-2 pi i (k-h)(j-h)/n}
    / sqrt(n) with h = floor(n/2), by brute force for odd and even n;
  * numpy's fftshift(fft2(ifftshift(.), norm="ortho"));
  * the adjoint identity and E^H E = I under full sampling with sum|S|^2 = 1;
  * for even n the modulation identities F_c = (-1)^{n/2} D F D,
    D = diag((-1)^i), lifted to E, E^H, E^H E and CG.  These are the route
    the CUDA library takes, so they pin the reading both sides share.
"""
import numpy as np
import pytest

import oracle
from paper_1807_11830_gb300 import synth


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def centred_dft_matrix(n):
    h = n // 2
    k = np.arange(n)[:, None] - h
    j = np.arange(n)[None, :] - h
    return np.exp(-2j * np.pi * k * j / n) / np.sqrt(n)


def _problem(ny, nx, C, F, L, seed):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(4, L), F, rng)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return x, S, lines, y


def checker(ny, nx):
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return np.where((yy + xx) % 2 == 0, 1.0, -1.0)


def kspace_signs(lines, nx):
    """(-1)^(ky + kx) for compacted k-space [F][C][L][nx]."""
    sy = np.where(lines % 2 == 0, 1.0, -1.0)  # [F][L]
    sx = np.where(np.arange(nx) % 2 == 0, 1.0, -1.0)
    return sy[:, None, :, None] * sx[None, None, None, :]


@pytest.mark.parametrize("ny,nx", [(1, 1), (3, 5), (4, 6), (5, 4), (7, 7), (8, 12)])
def test_centred_fft2_brute_force(ny, nx):
    rng = np.random.default_rng(ny * 31 + nx)
    x = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    expect = centred_dft_matrix(ny) @ x @ centred_dft_matrix(nx).T
    assert rel(oracle.fft2(x, centred=True), expect) < 1e-13
    back = oracle.fft2(expect, inverse=True, centred=True)
    assert rel(back, x) < 1e-13


@pytest.mark.parametrize("ny,nx", [(16, 16), (20, 12), (64, 96), (160, 160), (15, 9)])
def test_centred_fft2_matches_library(ny, nx):
    rng = np.random.default_rng(ny + 7 * nx)
    x = rng.standard_normal((2, ny, nx)) + 1j * rng.standard_normal((2, ny, nx))
    lib = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x, axes=(-2, -1)), norm="ortho"), axes=(-2, -1))
    assert rel(oracle.fft2(x, centred=True), lib) < 1e-12
    libi = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(x, axes=(-2, -1)), norm="ortho"), axes=(-2, -1))
    assert rel(oracle.fft2(x, inverse=True, centred=True), libi) < 1e-12


def test_centred_dc_at_centre():
    # a constant image has all its energy at the centred DC bin (h, h)
    n = 8
    x = np.ones((n, n), complex)
    X = oracle.fft2(x, centred=True)
    expect = np.zeros((n, n), complex)
    expect[n // 2, n // 2] = n
    assert rel(X, expect) < 1e-14


@pytest.mark.parametrize("shape", [(16, 12, 3, 7, 2), (20, 20, 2, 20, 1)])
def test_centred_adjoint_identity_and_full_sampling(shape):
    ny, nx, C, L, F = shape
    x, S, lines, y = _problem(ny, nx, C, F, L, 300 + ny)
    Ex = oracle.forward(x, S, lines, centred=True)
    EHy = oracle.adjoint(y, S, lines, centred=True)
    lhs = np.vdot(Ex, y)
    rhs = np.vdot(x, EHy)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Ex) * np.linalg.norm(y)
    full = synth.full_lines(ny, F)
    xx = oracle.normal(x, S, full, centred=True)
    assert rel(xx, x) < 1e-12  # sum|S|^2 = 1 and every line sampled: E^H E = I


@pytest.mark.parametrize("shape", [(16, 12, 3, 7, 2), (32, 20, 4, 11, 2), (12, 8, 2, 12, 1)])
def test_centred_equals_modulated_uncentred(shape):
    ny, nx, C, L, F = shape
    x, S, lines, y = _problem(ny, nx, C, F, L, 400 + ny + nx)
    D = checker(ny, nx)
    Dk = kspace_signs(lines, nx)
    c = (-1.0) ** (ny // 2 + nx // 2)
    # E_c x = c D_k E (D x)
    assert rel(oracle.forward(x, S, lines, centred=True), c * Dk * oracle.forward(D * x, S, lines)) < 1e-12
    # E_c^H y = c D E^H (D_k y)
    assert rel(oracle.adjoint(y, S, lines, centred=True), c * D * oracle.adjoint(Dk * y, S, lines)) < 1e-12
    # E_c^H E_c = D E^H E D
    assert rel(oracle.normal(x, S, lines, centred=True), D * oracle.normal(D * x, S, lines)) < 1e-12
    # RSS of centred k-space = RSS of the modulated k-space (signs on the image side drop out)
    assert rel(oracle.rss(y, lines, ny, centred=True), oracle.rss(c * Dk * y, lines, ny)) < 1e-12


def test_centred_cg_iterates_are_modulated():
    ny, nx, C, L, F = 16, 12, 4, 8, 2
    x, S, lines, _ = _problem(ny, nx, C, F, L, 555)
    y = oracle.forward(x, S, lines, centred=True)
    D = checker(ny, nx)
    Dk = kspace_signs(lines, nx)
    c = (-1.0) ** (ny // 2 + nx // 2)
    for K, tol in [(5, 0.0), (40, 1e-6)]:
        xc, ic, rc, sc = oracle.cg(y, S, lines, K, tol, centred=True)
        xu, iu, ru, su = oracle.cg(c * Dk * y, S, lines, K, tol)
        assert rel(xc, D * xu) < 1e-10
        np.testing.assert_array_equal(ic, iu)
        np.testing.assert_array_equal(sc, su)
        assert np.allclose(rc, ru, rtol=1e-8, atol=1e-14)
