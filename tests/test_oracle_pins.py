"""Pins of the FP64 oracle to facts outside itself (CPU only).

The paper (arXiv 1807.11830) prints no numeric result of its reconstruction,
so every pin here comes from mathematics: hand-derived DFT values, closed
forms, a library transform (numpy.fft with norm="ortho") for the special
cases that reduce to it, the adjoint identity, Hermitian/PSD structure, the
exact identity of Eq. 1 under full sampling with sum|S|^2 = 1, and a dense
Krylov-space solve for CG.  Each is chosen so that a plausible slip in the
oracle (a dropped conjugate, a flipped sign, a wrong index or scale) fails
at least one of them; tests/test_oracle_mutations.py checks that claim by
planting such slips in a copy of the oracle.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1807_11830_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIZES = [1, 2, 3, 4, 5, 6, 8, 12, 15, 16, 20, 24, 40, 48, 64, 80, 120, 128, 144, 160, 192, 240, 256, 288, 320, 384]


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def _parse_cplx_list(s):
    out = []
    for tok in s.split():
        re_, im_ = tok.split(",")
        out.append(complex(float(re_), float(im_)))
    return np.array(out)


def golden_dft_cases():
    cases = []
    with open(os.path.join(GOLDEN, "dft_small.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n, xin, xout = [p.strip() for p in line.split("|")]
            cases.append((int(n), _parse_cplx_list(xin), _parse_cplx_list(xout)))
    return cases


@pytest.mark.parametrize("n,x,expect", golden_dft_cases())
def test_dft_hand_values(n, x, expect):
    assert len(x) == n
    np.testing.assert_allclose(oracle.dft(x), expect, atol=1e-15, rtol=0)
    np.testing.assert_allclose(oracle.fft(x), expect, atol=1e-15, rtol=0)
    # inverse undoes forward
    np.testing.assert_allclose(oracle.fft(oracle.fft(x), inverse=True), x, atol=1e-14, rtol=0)


@pytest.mark.parametrize("n", SIZES)
def test_fft_equals_direct_dft(n):
    rng = synth.rng_for(100 + n)
    x = synth.random_complex(n, rng)
    for inv in (False, True):
        assert rel(oracle.fft(x, inv), oracle.dft(x, inv)) <= 1e-13


@pytest.mark.parametrize("n", [4, 7, 12, 64, 160, 384])
def test_fft_matches_library(n):
    rng = synth.rng_for(200 + n)
    x = synth.random_complex(n, rng)
    assert rel(oracle.fft(x), np.fft.fft(x, norm="ortho")) <= 1e-13
    assert rel(oracle.fft(x, True), np.fft.ifft(x, norm="ortho")) <= 1e-13


@pytest.mark.parametrize("ny,nx", [(8, 8), (12, 20), (64, 64), (192, 128), (320, 320)])
def test_fft2_matches_library(ny, nx):
    rng = synth.rng_for(300 + ny + nx)
    img = synth.random_complex((2, ny, nx), rng)
    assert rel(oracle.fft2(img), np.fft.fft2(img, norm="ortho")) <= 1e-13
    assert rel(oracle.fft2(img, True), np.fft.ifft2(img, norm="ortho")) <= 1e-13


def test_fft2_brute_force_tiny():
    # O(n^4) sum written as nested Python loops on a 6x4 image.
    rng = synth.rng_for(7)
    ny, nx = 6, 4
    img = synth.random_complex((ny, nx), rng)
    out = np.zeros((ny, nx), complex)
    for ky in range(ny):
        for kx in range(nx):
            acc = 0j
            for yy in range(ny):
                for xx in range(nx):
                    acc += img[yy, xx] * np.exp(-2j * np.pi * (ky * yy / ny + kx * xx / nx))
            out[ky, kx] = acc / np.sqrt(ny * nx)
    assert rel(oracle.fft2(img), out) <= 1e-13


@pytest.mark.parametrize("n", [64, 192, 320])
def test_parseval_delta_constant_ramp(n):
    rng = synth.rng_for(400 + n)
    img = synth.random_complex((n, n), rng)
    k = oracle.fft2(img)
    assert abs(np.linalg.norm(k) - np.linalg.norm(img)) <= 1e-12 * np.linalg.norm(img)
    # delta at the origin -> constant 1/n
    d = np.zeros((n, n), complex)
    d[0, 0] = 1.0
    np.testing.assert_allclose(oracle.fft2(d), np.full((n, n), 1.0 / n), atol=1e-14)
    # constant c -> c * n * delta
    c = 0.3 - 0.7j
    out = oracle.fft2(np.full((n, n), c))
    expect = np.zeros((n, n), complex)
    expect[0, 0] = c * n
    np.testing.assert_allclose(out, expect, atol=1e-11)
    # shifted delta -> pure phase ramp exp(-2 pi i (ky y0 + kx x0)/n)/n
    y0, x0 = 3, n - 5
    d = np.zeros((n, n), complex)
    d[y0, x0] = 1.0
    ky, kx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ramp = np.exp(-2j * np.pi * (ky * y0 + kx * x0) / n) / n
    np.testing.assert_allclose(oracle.fft2(d), ramp, atol=1e-13)


def _small_problem(ny, nx, C, L, F, seed, n_centre=4):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(n_centre, L), F, rng)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return x, S, lines, y


def test_forward_is_masked_library_fft2():
    x, S, lines, _ = _small_problem(16, 12, 3, 7, 2, 11)
    y = oracle.forward(x, S, lines)
    for f in range(2):
        for c in range(3):
            full = np.fft.fft2(S[c] * x[f], norm="ortho")
            np.testing.assert_allclose(y[f, c], full[lines[f], :], atol=1e-13)


def test_adjoint_is_zero_filled_library_ifft2():
    x, S, lines, y = _small_problem(16, 12, 3, 7, 2, 12)
    out = oracle.adjoint(y, S, lines)
    for f in range(2):
        acc = np.zeros((16, 12), complex)
        for c in range(3):
            z = np.zeros((16, 12), complex)
            z[lines[f], :] = y[f, c]
            acc += np.conj(S[c]) * np.fft.ifft2(z, norm="ortho")
        np.testing.assert_allclose(out[f], acc, atol=1e-13)


SHAPES = [  # (ny, nx, C, L, F): the workload shapes at reduced frame counts
    (64, 64, 4, 21, 1),
    (256, 256, 12, 64, 1),
    (320, 320, 4, 107, 1),
    (192, 128, 5, 48, 2),
    (384, 384, 2, 64, 1),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_adjoint_identity(shape):
    ny, nx, C, L, F = shape
    x, S, lines, y = _small_problem(ny, nx, C, L, F, 13 + ny)
    Ex = oracle.forward(x, S, lines)
    Ehy = oracle.adjoint(y, S, lines)
    lhs = np.vdot(Ex, y)    # <Ex, y>
    rhs = np.vdot(x, Ehy)   # <x, E^H y>
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Ex) * np.linalg.norm(y)


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_normal_hermitian_psd(shape):
    ny, nx, C, L, F = shape
    u, S, lines, _ = _small_problem(ny, nx, C, L, F, 21 + ny)
    v = synth.random_complex(u.shape, synth.rng_for(22 + ny))
    Au = oracle.normal(u, S, lines)
    Av = oracle.normal(v, S, lines)
    a = np.vdot(u, Av)
    b = np.conj(np.vdot(v, Au))
    assert abs(a - b) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(Av)
    quad = np.vdot(u, Au)
    assert abs(quad.imag) <= 1e-12 * abs(quad.real)
    assert quad.real >= 0.0


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_normal_equals_collapsed_form(shape):
    ny, nx, C, L, F = shape
    x, S, lines, _ = _small_problem(ny, nx, C, L, F, 31 + ny)
    a = oracle.normal(x, S, lines)
    b = oracle.normal_collapsed(x, S, lines)
    assert rel(a, b) <= 1e-12


def test_normal_equals_adjoint_of_forward():
    x, S, lines, _ = _small_problem(64, 64, 4, 21, 2, 41)
    assert rel(oracle.normal(x, S, lines), oracle.adjoint(oracle.forward(x, S, lines), S, lines)) == 0.0


@pytest.mark.parametrize("n,C", [(64, 4), (160, 8)])
def test_full_sampling_is_identity(n, C):
    """Eq. 1 with every line sampled and sum|S|^2 = 1: E^H E = I, so the
    adjoint of noiseless k-space returns the image and CG recovers it in one
    step with a zero residual."""
    rng = synth.rng_for(50 + n)
    S = synth.sensitivities(C, n, n)
    np.testing.assert_allclose(np.sum(np.abs(S) ** 2, axis=0), 1.0, atol=1e-14)
    lines = synth.full_lines(n, 2)
    x = synth.phantom(n, n, 10, rng, frames=2)
    assert rel(oracle.normal(x, S, lines), x) <= 1e-12
    y = oracle.forward(x, S, lines)
    assert rel(oracle.adjoint(y, S, lines), x) <= 1e-12
    # one step, fixed count: x1 = b = x
    x1, iters, resid, _ = oracle.cg(y, S, lines, max_iter=1)
    assert rel(x1, x) <= 1e-12 and list(iters) == [1, 1] and np.all(resid <= 1e-12)
    # with a stopping tolerance the residual test ends the solve after step 1
    xs, iters, resid, status = oracle.cg(y, S, lines, max_iter=5, tol=1e-10)
    assert rel(xs, x) <= 1e-12
    assert list(iters) == [1, 1]
    assert list(status) == [oracle.CG_CONVERGED] * 2
    assert np.all(resid <= 1e-12)


def _dense_normal(S, lines, ny, nx):
    n = ny * nx
    A = np.zeros((n, n), complex)
    for j in range(n):
        e = np.zeros((1, ny, nx), complex)
        e.ravel()[j] = 1.0
        A[:, j] = oracle.normal(e, S, lines).ravel()
    return A


def test_cg_against_dense_krylov_solves():
    """Tiny 8x8, 3 coils, R=2.  A = E^H E is built column by column; each CG
    iterate x_k must be the A-norm minimiser over span{b, Ab, ..., A^{k-1} b}
    (solved densely), and after many steps CG matches the dense solve of the
    normal equations."""
    ny = nx = 8
    rng = synth.rng_for(61)
    # generic random maps: the smooth ring model makes A an exact projector
    # at this size, and CG would finish in one step
    S = synth.random_complex((3, ny, nx), rng)
    lines = synth.mask_lines(ny, 4, 2, 1, rng)
    y = synth.random_complex((1, 3, 4, nx), rng)
    A = _dense_normal(S, lines, ny, nx)
    b = oracle.adjoint(y, S, lines).ravel()
    assert np.allclose(A, A.conj().T, atol=1e-13)
    for k in (1, 2, 3, 5, 8):
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        c = np.linalg.solve(Q.conj().T @ A @ Q, Q.conj().T @ b)
        xk_dense = Q @ c
        xk, iters, _, _ = oracle.cg(y, S, lines, max_iter=k)
        assert iters[0] == k
        assert rel(xk.ravel(), xk_dense) <= 1e-8, k
    # converged solve vs dense least squares (A may be singular: compare the
    # minimum-norm solution, which CG from x0 = 0 reaches in exact arithmetic)
    x_ls = np.linalg.lstsq(A, b, rcond=1e-12)[0]
    xc, _, resid, _ = oracle.cg(y, S, lines, max_iter=200, tol=1e-13)
    assert rel(xc.ravel(), x_ls) <= 1e-8
    assert rel(A @ xc.ravel(), b) <= 1e-10


@pytest.mark.parametrize("lam", [0.0625, 1.5])
def test_regularised_cg_against_dense_solves(lam):
    """Tikhonov-regularised CG solves (A + lam I) x = b with A = E^H E built
    densely: each iterate is the (A + lam I)-norm minimiser over the Krylov
    space of A + lam I, and the converged iterate is the dense solve (the
    shifted matrix is positive definite, so the solution is unique)."""
    ny = nx = 8
    rng = synth.rng_for(62)
    S = synth.random_complex((3, ny, nx), rng)
    lines = synth.mask_lines(ny, 4, 2, 1, rng)
    y = synth.random_complex((1, 3, 4, nx), rng)
    A = _dense_normal(S, lines, ny, nx) + lam * np.eye(ny * nx)
    b = oracle.adjoint(y, S, lines).ravel()
    for k in (1, 3, 6):
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        xk_dense = Q @ np.linalg.solve(Q.conj().T @ A @ Q, Q.conj().T @ b)
        xk, iters, _, _ = oracle.cg(y, S, lines, max_iter=k, lam=lam)
        assert iters[0] == k
        assert rel(xk.ravel(), xk_dense) <= 1e-8, k
    xc, _, _, status = oracle.cg(y, S, lines, max_iter=300, tol=1e-13, lam=lam)
    assert rel(xc.ravel(), np.linalg.solve(A, b)) <= 1e-9


def test_regularised_cg_limits():
    x, S, lines, y = _small_problem(16, 16, 3, 6, 2, 73)
    # lam = 0 is plain CG-SENSE
    a = oracle.cg(y, S, lines, 5)
    b = oracle.cg(y, S, lines, 5, lam=0.0)
    assert rel(a[0], b[0]) == 0.0
    # a dominant lam: one step gives x = (rho0 / (rho0 lam + <b, A b>)) b -> b / lam
    lam = 1e8
    xb = oracle.adjoint(y, S, lines)
    x1, _, _, _ = oracle.cg(y, S, lines, 1, lam=lam)
    assert rel(x1 * lam, xb) <= 1e-7


def _dense_coupled(S, lines, ny, nx, lam, lam_t):
    """Stacked dense matrix of E^H E + lam I + lam_t (L (x) I) over F frames,
    L the cyclic second difference 2 I - shift - shift^T."""
    F = lines.shape[0]
    n = ny * nx
    A = np.zeros((F * n, F * n), complex)
    for f in range(F):
        A[f * n:(f + 1) * n, f * n:(f + 1) * n] = _dense_normal(S, lines[f:f + 1], ny, nx) + lam * np.eye(n)
    Lt = 2 * np.eye(F) - np.roll(np.eye(F), 1, axis=1) - np.roll(np.eye(F), -1, axis=1)
    return A + lam_t * np.kron(Lt, np.eye(n))


@pytest.mark.parametrize("F,lam,lam_t", [(3, 0.0, 0.5), (4, 0.125, 2.0), (2, 0.0, 0.25)])
def test_temporal_cg_against_dense_solves(F, lam, lam_t):
    """Temporally regularised CG couples the frames: one CG on the stacked
    system.  Each iterate is the minimiser over the stacked Krylov space and
    the converged iterate is the dense solve."""
    ny = nx = 6
    rng = synth.rng_for(64 + F)
    S = synth.random_complex((2, ny, nx), rng)
    lines = synth.mask_lines(ny, 3, 2, F, rng)
    y = synth.random_complex((F, 2, 3, nx), rng)
    A = _dense_coupled(S, lines, ny, nx, lam, lam_t)
    assert np.allclose(A, A.conj().T, atol=1e-12)
    b = oracle.adjoint(y, S, lines).ravel()
    for k in (1, 2, 5):
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        xk_dense = Q @ np.linalg.solve(Q.conj().T @ A @ Q, Q.conj().T @ b)
        xk, iters, _, _ = oracle.cg(y, S, lines, max_iter=k, lam=lam, lam_t=lam_t)
        assert list(iters) == [k] * F
        assert rel(xk.ravel(), xk_dense) <= 1e-8, k
    xc, iters, resid, status = oracle.cg(y, S, lines, max_iter=400, tol=1e-13, lam=lam, lam_t=lam_t)
    assert len(set(iters)) == 1 and len(set(status)) == 1 and len(set(resid)) == 1
    x_ls = np.linalg.lstsq(A, b, rcond=1e-12)[0]
    assert rel(xc.ravel(), x_ls) <= 1e-8


def test_temporal_cg_special_cases():
    x, S, lines, y = _small_problem(12, 12, 3, 5, 1, 75)
    # one frame: the cyclic difference vanishes, the plain per-frame CG results
    a = oracle.cg(y, S, lines, 6, lam=0.25)
    b = oracle.cg(y, S, lines, 6, lam=0.25, lam_t=3.0)
    assert rel(b[0], a[0]) <= 1e-12
    # frames with identical data and masks: the solution is constant in time,
    # so the temporal term does not change it
    F = 3
    yy = np.repeat(y, F, axis=0)
    ll = np.repeat(lines, F, axis=0)
    c = oracle.cg(yy, S, ll, 8, lam_t=5.0)
    d = oracle.cg(yy, S, ll, 8)
    assert rel(c[0], d[0]) <= 1e-10


def test_cg_frames_independent_and_zero_rhs():
    x, S, lines, y = _small_problem(32, 32, 3, 12, 3, 71)
    y[1] = 0.0
    xs, iters, resid, status = oracle.cg(y, S, lines, max_iter=7)
    assert iters[1] == 0 and status[1] == oracle.CG_CONVERGED and resid[1] == 0.0
    assert np.all(xs[1] == 0)
    for f in (0, 2):
        xf, itf, rf, sf = oracle.cg(y[f:f + 1], S, lines[f:f + 1], max_iter=7)
        np.testing.assert_array_equal(xf[0], xs[f])
        assert itf[0] == iters[f] == 7 and sf[0] == oracle.CG_MAXITER


def test_cg_residual_monotone_reaches_tolerance():
    p = synth.single_slice_64()
    y = oracle.forward(p.x_true, p.S, p.lines) + p.noise
    x, iters, resid, status = oracle.cg(y, p.S, p.lines, max_iter=200, tol=1e-4)
    assert status[0] == oracle.CG_CONVERGED and resid[0] <= 1e-4
    # the recursive residual equals the true residual of the normal equations
    b = oracle.adjoint(y, p.S, p.lines)
    true_res = np.linalg.norm(b - oracle.normal(x, p.S, p.lines)) / np.linalg.norm(b)
    assert abs(true_res - resid[0]) <= 1e-6


def test_rss_closed_forms():
    """RSS of fully sampled single-coil k-space F2(x) is |x|; with maps
    summing to one in square, RSS of F2(S_c x) is |x| too."""
    rng = synth.rng_for(81)
    n = 32
    x = synth.random_complex((2, n, n), rng)
    lines = synth.full_lines(n, 2)
    y1 = oracle.fft2(x)[:, None]
    np.testing.assert_allclose(oracle.rss(y1, lines, n), np.abs(x), atol=1e-13)
    S = synth.sensitivities(5, n, n)
    yc = oracle.forward(x, S, lines)
    np.testing.assert_allclose(oracle.rss(yc, lines, n), np.abs(x), atol=1e-13)
    # with a partial mask RSS equals sqrt(sum_c |zero-filled library ifft2|^2)
    lines_p = synth.mask_lines(n, 10, 4, 2, rng)
    yp = synth.random_complex((2, 3, 10, n), rng)
    expect = np.zeros((2, n, n))
    for f in range(2):
        for c in range(3):
            z = np.zeros((n, n), complex)
            z[lines_p[f]] = yp[f, c]
            expect[f] += np.abs(np.fft.ifft2(z, norm="ortho")) ** 2
    np.testing.assert_allclose(oracle.rss(yp, lines_p, n), np.sqrt(expect), atol=1e-13)


def _bf16_golden():
    out = []
    with open(os.path.join(GOLDEN, "bf16_cases.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                a, b = line.split()
                out.append((int(a, 16), int(b, 16)))
    return out


def test_bf16_rne_hand_cases():
    cases = _bf16_golden()
    f32 = np.array([a for a, _ in cases], np.uint32).view(np.float32)
    got = oracle.bf16_rne(f32)
    np.testing.assert_array_equal(got, np.array([b for _, b in cases], np.uint16))


def test_bf16_rne_matches_library_cast():
    torch = pytest.importorskip("torch")
    rng = synth.rng_for(91)
    v = np.concatenate([rng.standard_normal(200000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 200000),
                        rng.standard_normal(1000).astype(np.float32)])
    ours = oracle.bf16_rne(v)
    lib = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, lib)


def test_lines_validation():
    x, S, lines, y = _small_problem(16, 16, 2, 5, 1, 95)
    bad = lines.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(ValueError):
        oracle.adjoint(y, S, bad)
    bad = lines.copy()
    bad[0, -1] = 16
    with pytest.raises(ValueError):
        oracle.forward(x, S, bad)
