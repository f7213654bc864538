"""The seeded input generators (synth/) on CPU: the recipe the tests, the
bench and the oracle runs share (point sources, wavenumber profiles of MP 2-B,
the layered model, the ragged sizes) and its seeding."""
import numpy as np
import pytest

import synth


def test_point_sources():
    b = synth.point_source(16, 12, 0.25)
    assert b.shape == (13, 17) and b[6, 8] == 16.0 and np.count_nonzero(b) == 1
    with pytest.raises(ValueError):
        synth.point_source(16, 12, 0.25, i=0)
    r = synth.source_row(64, 32, 1 / 64, 8)
    assert r.shape == (8, 33, 65)
    for s in range(8):
        assert np.count_nonzero(r[s]) == 1
        assert r[s, 31, int(round((s + 0.5) / 8 * 64))] == 64.0 ** 2   # first row below the top boundary


def test_wavenumber_profiles():
    sm = synth.chi_smooth(40, 30, 3)
    assert sm.shape == (31, 41) and sm.min() == 0.0 and sm.max() == 1.0
    sh = synth.chi_sharp(63, 47, 4)
    assert sh.shape == (48, 64) and 0.0 <= sh.min() and sh.max() <= 1.0
    # constant on a 16 x 16 partition: 64 / 16 = 4 columns and 48 / 16 = 3 rows per block
    assert len(np.unique(sh)) <= 256
    assert np.array_equal(sh[:, 0], sh[:, 3]) and not np.array_equal(sh[:, 0], sh[:, 4])
    assert np.array_equal(sh[0], sh[2]) and not np.array_equal(sh[0], sh[3])
    kf = synth.k_field(sh, 10.0, 20.0)
    assert 10.0 <= kf.min() and kf.max() <= 20.0
    assert np.array_equal(synth.chi_sharp(63, 47, 4), sh) and not np.array_equal(synth.chi_sharp(63, 47, 5), sh)


def test_layered_model_and_perturbation():
    v = synth.layered_velocity(184, 60, 50.0, 7)
    assert v.shape == (61, 185)
    assert 1500.0 * 0.85 <= v.min() and v.max() <= 5500.0 * 1.15
    assert np.median(v[-1]) > np.median(v[0])            # faster with depth
    assert np.array_equal(v, synth.layered_velocity(184, 60, 50.0, 7))
    p = synth.smooth_perturbation(64, 48, 2)
    assert p.min() == -1.0 and abs(p.max() - 1.0) < 1e-15


def test_ragged_sizes_coarsen_to_small_grids():
    ns = synth.ragged_sizes(32, 3)
    assert ns == synth.ragged_sizes(32, 3) and len(ns) == 32
    for n in ns:
        assert 128 <= n <= 1024
        while n % 2 == 0 and n > 7:
            n //= 2
        assert 4 <= n <= 7, n


def test_random_vectors_are_seeded():
    a = synth.random_complex((5, 7), 1)
    assert a.dtype == np.complex128 and np.array_equal(a, synth.random_complex((5, 7), 1))
    assert not np.array_equal(a, synth.random_complex((5, 7), 2))
