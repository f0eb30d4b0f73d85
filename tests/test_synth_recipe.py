"""The seeded input generators follow the stated recipe (CPU only).

Every workload is synthetic, so the inputs are only as good as their
generators.  These tests hold them to the recipe of each configuration:
coil maps normalised so that sum_c |S_c|^2 = 1, the Gaussian-ring magnitude
and its phase ramp, line masks (sorted, in range, centre rows always
sampled, fresh per frame, L = round(n / R)), the phantom's value ranges and
cine modulation, the noise level, the uneven-batch distribution and the
Poisson arrival process.  Draws are reproducible from their seeds.
"""
import numpy as np
import pytest

from paper_1807_11830_gb300 import synth


@pytest.mark.parametrize("coils,ny,nx", [(4, 64, 64), (12, 32, 48), (1, 16, 16)])
def test_sensitivities_normalised_ring(coils, ny, nx):
    S = synth.sensitivities(coils, ny, nx)
    assert S.shape == (coils, ny, nx)
    np.testing.assert_allclose(np.sum(np.abs(S) ** 2, axis=0), 1.0, rtol=0, atol=1e-12)
    if coils > 1:
        # coil c is strongest near its ring point at angle 2 pi c / C
        for c in range(coils):
            th = 2 * np.pi * c / coils
            cy = int(np.clip(round(ny / 2 + (ny / 2) * np.sin(th)), 0, ny - 1))
            cx = int(np.clip(round(nx / 2 + (nx / 2) * np.cos(th)), 0, nx - 1))
            assert np.argmax(np.abs(S[:, cy, cx])) == c


def test_sensitivity_phase_ramp():
    C, n = 3, 32
    S = synth.sensitivities(C, n, n)
    # the normalisation is real and positive, so the phase is the ramp itself
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    for c in range(C):
        th = 2 * np.pi * c / C
        ramp = np.pi * ((x - n / 2) * np.cos(th) + (y - n / 2) * np.sin(th)) / n
        np.testing.assert_allclose(np.angle(S[c] * np.exp(-1j * ramp)), 0.0, atol=1e-12)


@pytest.mark.parametrize("ny,L,nc,F", [(64, 21, 8, 1), (256, 64, 16, 20), (320, 107, 24, 4), (16, 16, 4, 2),
                                       (12, 5, 5, 3)])
def test_mask_lines(ny, L, nc, F):
    lines = synth.mask_lines(ny, L, nc, F, synth.rng_for(5))
    assert lines.shape == (F, L) and lines.dtype == np.int32
    centre = set(synth.centre_rows(ny, nc))
    assert len(centre) == nc
    assert centre == set(range(nc // 2)) | set(range(ny - (nc - nc // 2), ny))  # DC at row 0
    for f in range(F):
        row = lines[f]
        assert np.all(np.diff(row) > 0) and row[0] >= 0 and row[-1] < ny
        assert centre <= set(row.tolist())
    if F > 1 and L - nc >= 4 and L < ny:
        assert any(not np.array_equal(lines[0], lines[f]) for f in range(1, F))  # fresh per frame
    with pytest.raises(ValueError):
        synth.mask_lines(ny, nc - 1, nc, 1, synth.rng_for(1))


def test_centred_lines_are_the_same_frequencies():
    lines = synth.mask_lines(64, 20, 8, 3, synth.rng_for(9))
    c = synth.centred_lines(lines, 64)
    for f in range(3):
        assert np.all(np.diff(c[f]) > 0)
        np.testing.assert_array_equal(np.sort((c[f] - 32) % 64), lines[f])


def test_configuration_shapes():
    p0 = synth.single_slice_64()
    assert p0.shape == dict(frames=1, coils=4, ny=64, nx=64, lines=21) and p0.iters == 10
    p1 = synth.cine_256(frames=3)
    assert p1.shape == dict(frames=3, coils=12, ny=256, nx=256, lines=64) and p1.iters == 30
    assert set(synth.centre_rows(256, 16)) <= set(p1.lines[0].tolist())
    p4 = synth.paper_160(frames=2)
    assert p4.shape == dict(frames=2, coils=8, ny=160, nx=160, lines=160)
    np.testing.assert_array_equal(p4.lines, synth.full_lines(160, 2))
    assert synth.lines_for_acceleration(320, 3) == 107 and synth.lines_for_acceleration(256, 4) == 64
    assert [synth.centre_for(n) for n in (128, 192, 256, 384)] == [8, 12, 16, 24]


def test_phantom_values_and_cine_modulation():
    rng = synth.rng_for(3)
    ells = synth.draw_ellipses(200, rng)
    amps = np.array([abs(e.value) for e in ells])
    phases = np.array([np.angle(e.value) for e in ells])
    assert amps.min() >= 0.2 and amps.max() <= 1.0
    assert phases.min() >= -np.pi and phases.max() <= np.pi
    assert all(0.1 <= e.a <= 0.45 and 0.1 <= e.b <= 0.45 and -0.5 <= e.cx <= 0.5 for e in ells)
    x = synth.phantom(32, 32, 1, synth.rng_for(4), frames=20, period=20)
    support = (np.abs(x) > 0).sum(axis=(1, 2))
    # semi-axes scale with 1 + 0.15 sin(2 pi t / 20): largest near t = 5, smallest near t = 15
    assert support[5] > support[0] > support[15]
    assert np.array_equal(x[0] != 0, synth.phantom(32, 32, 1, synth.rng_for(4), frames=1)[0] != 0)


def test_noise_level():
    n = synth.complex_noise((400, 500), 1e-3, synth.rng_for(11))
    assert abs(np.mean(np.abs(n) ** 2) / 1e-6 - 1.0) < 0.02
    assert abs(np.var(n.real) / 0.5e-6 - 1.0) < 0.03 and abs(np.var(n.imag) / 0.5e-6 - 1.0) < 0.03


def test_mix_distribution_and_reproducibility():
    mix = synth.draw_mix(512)
    assert len(mix) == 512
    assert {m["n"] for m in mix} == set(synth.MIX_SIZES)
    assert {m["accel"] for m in mix} == set(synth.MIX_ACCEL)
    assert min(m["coils"] for m in mix) >= 8 and max(m["coils"] for m in mix) <= 32
    assert min(m["frames"] for m in mix) >= 1 and max(m["frames"] for m in mix) <= 30
    assert all(m["lines"] == round(m["n"] / m["accel"]) and m["centre"] == synth.centre_for(m["n"]) for m in mix)
    assert synth.draw_mix(512) == mix  # same seed, same draw
    a = synth.mix_instance(mix[0], 77)
    b = synth.mix_instance(mix[0], 77)
    np.testing.assert_array_equal(a.x_true, b.x_true)
    np.testing.assert_array_equal(a.lines, b.lines)
    assert a.lines.shape == (mix[0]["frames"], mix[0]["lines"])


def test_poisson_arrivals():
    t = synth.poisson_arrivals(800.0, 20000, seed=5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(np.mean(gaps) * 800.0 - 1.0) < 0.03
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.05  # exponential: coefficient of variation 1
