"""Plant plausible slips in a copy of the oracle and check that the pins in
test_oracle_pins.py catch each one (CPU only).

Each mutant is the oracle source with one textual edit, built into a
temporary directory; the pins run against it through the oracle's own
loader and at least one of them must fail.  The committed oracle itself is
never modified.
"""
import os
import subprocess

import pytest

import oracle
import tests.test_oracle_centred as centred
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sense_oracle.cpp")

MUTANTS = {
    # adjoint forgets the conjugate of the maps
    "adjoint_no_conj": ("xf[i] += std::conj(Sc[i]) * z[i];", "xf[i] += Sc[i] * z[i];"),
    # twiddles of the recursive FFT take the wrong sign
    "fft_twiddle_sign": ("acc += sub[(size_t)r * m + k] * unit_root((long long)r * kk, n, dir);",
                         "acc += sub[(size_t)r * m + k] * unit_root((long long)r * kk, n, -dir);"),
    # twiddle exponent uses k instead of k + m s
    "fft_twiddle_index": ("unit_root((long long)r * kk, n, dir)", "unit_root((long long)r * k, n, dir)"),
    # 2D transform loses its 1/sqrt(n) scale
    "fft_no_scale": ("for (int j = 0; j < n; ++j) data[(long)j * stride] = tmp_out[j] * s;",
                     "for (int j = 0; j < n; ++j) data[(long)j * stride] = tmp_out[j];"),
    # forward keeps row l instead of row lines[l]
    "forward_line_index": ("t[(long)ln[l] * nx + k]", "t[(long)l * nx + k]"),
    # CG beta inverted
    "cg_beta_inverted": ("double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    # CG residual update with the wrong sign
    "cg_residual_sign": ("r[i] -= alpha * q[i];", "r[i] += alpha * q[i];"),
    # CG uses the imaginary part of <p, q> as well (a conj slip in re_dot)
    "dot_conj_slip": ("s += a[i].real() * b[i].real() + a[i].imag() * b[i].imag();",
                      "s += a[i].real() * b[i].real() - a[i].imag() * b[i].imag();"),
    # bf16 ties always round up
    "bf16_ties_up": ("(dropped == 0x8000u && (kept & 1u))", "(dropped == 0x8000u)"),
    # direct DFT index slip
    "dft_index": ("in[(long)j * stride] * unit_root((long long)j * k, n, dir)",
                  "in[(long)j * stride] * unit_root((long long)j * (k + 1), n, dir)"),
    # temporal difference adds a neighbour instead of subtracting it
    "temporal_neighbour_sign": ("(2.0 * pf[i] - pm[i] - pn[i])", "(2.0 * pf[i] - pm[i] + pn[i])"),
    # Tikhonov term with the wrong sign
    "cg_lambda_sign": ("q[i] += lambda * p[i];", "q[i] -= lambda * p[i];"),
    # centred transform forgets the output fftshift
    "centred_no_fftshift": ("  if (centred) rotate_strided(n, v, stride, n / 2);  // fftshift\n", "\n"),
    # centred transform shifts the input the wrong way (differs for odd n)
    "centred_shift_direction": ("rotate_strided(n, v, stride, -(n / 2));  // ifftshift",
                                "rotate_strided(n, v, stride, n / 2);  // ifftshift"),
    # RSS sums magnitudes instead of squared magnitudes
    "rss_abs_not_square": ("acc[i] += std::norm(z[i]);", "acc[i] += std::abs(z[i]);"),
    # RSS forgets the square root
    "rss_no_sqrt": ("out[f * npix + i] = std::sqrt(acc[i]);", "out[f * npix + i] = acc[i];"),
    # column-wise normal operator forgets the mask
    "collapsed_no_mask": ("          if (!sampled[r]) col[r] = 0.0;\n", "\n"),
    # column-wise normal operator applies the second transform in the forward direction
    "collapsed_second_forward": ("        fft1_strided(ny, +1, col.data(), 1, a, b);\n"
                                 "        for (int r = 0; r < ny; ++r) of[(long)r * nx + j]",
                                 "        fft1_strided(ny, -1, col.data(), 1, a, b);\n"
                                 "        for (int r = 0; r < ny; ++r) of[(long)r * nx + j]"),
}

QUICK_PINS = [
    lambda: [pins.test_dft_hand_values(*c) for c in pins.golden_dft_cases()],
    lambda: [pins.test_fft_equals_direct_dft(n) for n in (6, 12, 64)],
    lambda: pins.test_fft2_matches_library(12, 20),
    lambda: pins.test_parseval_delta_constant_ramp(64),
    pins.test_forward_is_masked_library_fft2,
    pins.test_adjoint_is_zero_filled_library_ifft2,
    lambda: pins.test_adjoint_identity(pins.SHAPES[0]),
    lambda: pins.test_full_sampling_is_identity(64, 4),
    pins.test_cg_against_dense_krylov_solves,
    pins.test_bf16_rne_hand_cases,
    lambda: [centred.test_centred_fft2_brute_force(*sh) for sh in [(3, 5), (4, 6), (7, 7)]],
    lambda: centred.test_centred_adjoint_identity_and_full_sampling((16, 12, 3, 7, 2)),
    lambda: pins.test_regularised_cg_against_dense_solves(0.0625),
    lambda: pins.test_temporal_cg_against_dense_solves(3, 0.0, 0.5),
    pins.test_rss_closed_forms,
    lambda: pins.test_normal_equals_collapsed_form(pins.SHAPES[0]),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor vanished from the oracle: %s" % name
    mutant = tmp_path / "mutant.cpp"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", str(mutant), "-o", str(lib)],
                   check=True)
    saved = oracle._LIB
    oracle._LIB = oracle._load(str(lib))
    caught = []
    try:
        for i, pin in enumerate(QUICK_PINS):
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                caught.append(i)
    finally:
        oracle._LIB = saved
    assert caught, "no pin caught mutant %s" % name
