"""Seeded input generators: quadrature moments, folding, masks (CPU)."""

import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I


@pytest.mark.parametrize("q", [I.circle_quadrature(16), I.circle_quadrature(32),
                               I.sphere_quadrature(24, 12), I.projected_quadrature(48, 12),
                               I.projected_quadrature(48, 12, fold=False)])
def test_quadrature_second_moment(q):
    # d_ang * sum_s w_s p p^T = identity in the plane (3D: in space): this makes
    # the flux weights K_o reproduce kappa_bulk for a uniform gradient
    d = q.angular_dim
    assert abs(q.weights.sum() - 1.0) < 1e-14
    for a in range(2):
        assert abs(d * np.sum(q.weights * q.dirs[:, a] ** 2) - 1.0) < 1e-13
    assert abs(np.sum(q.weights * q.dirs[:, 0] * q.dirs[:, 1])) < 1e-14


@pytest.mark.parametrize("q", [I.circle_quadrature(16), I.sphere_quadrature(24, 12),
                               I.projected_quadrature(48, 12)])
def test_quadrature_symmetric(q):
    # every direction has its mirror images and its reverse (walls conserve flux)
    for flip in ([-1, 1, 1], [1, -1, 1], [-1, -1, 1]):
        f = q.dirs * np.array(flip)
        for v, w in zip(f, q.weights):
            k = np.argmin(np.abs(q.dirs - v).sum(1))
            assert np.abs(q.dirs[k] - v).max() < 1e-12 and abs(q.weights[k] - w) < 1e-15


def test_no_grazing_directions():
    for q in (I.circle_quadrature(16), I.sphere_quadrature(24, 12), I.projected_quadrature(48, 12)):
        assert np.all(np.abs(q.dirs[:, 0]) > 1e-6) and np.all(np.abs(q.dirs[:, 1]) > 1e-6)


def test_mfp_bins():
    k, lam = I.mfp_bins(8)
    assert abs(k.sum() - 150.0) < 1e-12
    assert abs(lam[0] - 1e-9) < 1e-21 and abs(lam[-1] - 1e-5) < 1e-17
    assert np.all(np.diff(np.log(lam)) > 0)


def test_config_sizes():
    w1 = I.config1()
    assert w1.mask.shape == (1, 32, 32) and w1.n_ordinates == 128
    assert abs(w1.porosity - 0.2) < 0.01
    w2 = I.config2()
    assert w2.n_ordinates == 8640 and abs(w2.porosity - 0.25) < 0.005
    w3 = I.config3()
    assert w3.mask.shape == (32, 64, 64) and w3.n_ordinates == 8640
    w5 = I.config5()
    assert w5.s.shape == (1, 128, 128) and 0.5 <= w5.s.min() and w5.s.max() <= 2.0


def test_batch_geometries_seeded():
    a = I.config4(8)
    b = I.config4(8)
    for x, y in zip(a, b):
        assert np.array_equal(x.mask, y.mask)
        assert 48 <= x.shape[0] <= 192 and x.shape[0] % 16 == 0
        assert 0.03 < x.porosity < 0.45
