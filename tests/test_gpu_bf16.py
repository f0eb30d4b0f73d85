"""BF16 storage of k-space and maps: parity and error against the oracle.

In BF16 storage S and y are held as bfloat16 (re, im) pairs; transforms,
coil sums and CG vectors stay FP32 and the CG inner products FP64.  Two
comparisons separate storage error from arithmetic error:
  * against the oracle fed the same bf16-rounded inputs ("quantised-input"),
    gated at the FP32 tolerances (1e-5 per operator, 1e-4 on CG images);
  * against the oracle fed the exact inputs, reported and bounded loosely
    (bf16 keeps 8 significant bits, so ~2^-9 relative per stored value).
The forward operator stores its result in bf16, so there the GPU result is
compared with the oracle's FP64 result rounded by the oracle's own RNE, to
within one bf16 ulp per component.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1807_11830_gb300 import sense, synth
from tests.gpu_util import (CG_TOL, OP_TOL, c64, ensure_built, gpu_adjoint, gpu_cg, gpu_forward, gpu_normal, rel)

pytestmark = pytest.mark.gpu
BF = sense.STORE_BF16


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def q(a):
    return oracle.quantize_c64_bf16(a)


def test_conversion_kernel_matches_oracle_rne():
    rng = synth.rng_for(11)
    a = (synth.random_complex(300001, rng) * 10.0 ** rng.integers(-20, 20, 300001)).astype(np.complex64)
    a[:4] = [np.inf, -np.inf + 1j, 0.0, -0.0]
    got = sense.to_bf16_pairs(c64(a))
    torch.cuda.synchronize()
    bits = got.view(torch.int16).cpu().numpy().view(np.uint16).reshape(-1)
    expect = oracle.bf16_rne(a.view(np.float32))
    np.testing.assert_array_equal(bits, expect)


def _problem(ny, nx, C, L, F, seed):
    rng = synth.rng_for(seed)
    S = synth.sensitivities(C, ny, nx)
    lines = synth.mask_lines(ny, L, min(8, L), F, rng)
    x = synth.random_complex((F, ny, nx), rng)
    y = synth.random_complex((F, C, L, nx), rng)
    return x, S, lines, y


SHAPES = [(64, 64, 4, 21, 2), (320, 320, 6, 107, 1), (192, 128, 5, 48, 2), (256, 256, 12, 64, 1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_adjoint_bf16(shape):
    _, S, lines, y = _problem(*shape, seed=500 + sum(shape))
    got = gpu_adjoint(y, S, lines, BF)
    assert rel(got, oracle.adjoint(q(y), q(S), lines)) <= OP_TOL
    assert rel(got, oracle.adjoint(y, S, lines)) <= 1e-2


@pytest.mark.parametrize("shape", SHAPES)
def test_normal_bf16(shape):
    x, S, lines, _ = _problem(*shape, seed=600 + sum(shape))
    x32 = x.astype(np.complex64).astype(np.complex128)
    got = gpu_normal(x, S, lines, BF)
    assert rel(got, oracle.normal(x32, q(S), lines)) <= OP_TOL
    assert rel(got, oracle.normal(x32, S, lines)) <= 1e-2


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_forward_bf16_output_rounding(shape):
    x, S, lines, _ = _problem(*shape, seed=700 + sum(shape))
    x32 = x.astype(np.complex64).astype(np.complex128)
    got = gpu_forward(x, S, lines, BF)
    exact = oracle.forward(x32, q(S), lines)
    rounded = q(exact)
    # Per component: within one bf16 ulp of the rounded oracle value, plus
    # the FP32 arithmetic error before rounding, which is absolute (set by
    # the array's largest values), not relative to each element.
    floor = 1e-5 * np.max(np.abs(exact))
    for part in (np.real, np.imag):
        g, r = part(got).ravel(), part(rounded).ravel()
        ulp = np.abs(r) * 2.0 ** -7
        assert np.all(np.abs(g - r) <= ulp + floor)
        # away from the floor the two roundings agree to the bit almost always
        big = np.abs(r) > 1e3 * floor
        assert np.mean(g[big] == r[big]) > 0.99
    assert rel(got, exact) <= 2.0 ** -8
