"""Pins of the oracle's A, E, T channels and likelihood inner products (CPU only).

The A, E, T map is fixed by its action on three independent X, Y, Z patterns (each row's
coefficients and signs), and cross-checked by orthonormality; the inner products by the
white-noise loss written directly in X, Y, Z (the loss of the differentiation workload),
by per-channel weights and by linearity in the data.
"""
import math

import numpy as np
import pytest

import oracle


def _series(seed, n=257):
    return np.random.default_rng(seed).normal(size=(3, n))


def test_aet_on_its_three_eigenpatterns():
    s = np.linspace(-2.0, 3.0, 11)
    z = np.zeros_like(s)
    # X = Y = Z: only T, with the norm of (1, 1, 1)
    np.testing.assert_allclose(oracle.aet(np.stack([s, s, s])), np.stack([z, z, math.sqrt(3) * s]), atol=1e-15)
    # X = -Z, Y = 0: only A, and A has the sign of Z - X
    np.testing.assert_allclose(oracle.aet(np.stack([s, z, -s])), np.stack([-math.sqrt(2) * s, z, z]), atol=1e-15)
    # X = Z = -Y/2: only E, with E > 0 for X > 0
    np.testing.assert_allclose(oracle.aet(np.stack([s, -2 * s, s])), np.stack([z, math.sqrt(6) * s, z]),
                               atol=1e-15)


def test_aet_is_orthonormal():
    x = _series(1)
    a = oracle.aet(x)
    assert abs(np.sum(a * a) - np.sum(x * x)) <= 1e-14 * np.sum(x * x)
    y = _series(2)
    assert abs(np.sum(oracle.aet(y) * a) - np.sum(y * x)) <= 1e-13 * math.sqrt(np.sum(x * x) * np.sum(y * y))


def test_like_equals_white_noise_loss_in_xyz():
    h, d = _series(3), _series(4)
    sigma = 0.7
    w = (1 / sigma**2,) * 3
    dh, hh = oracle.like_inner(h, oracle.aet(d), w)
    _, dd = oracle.like_inner(d, oracle.aet(d), w)
    loss_xyz = 0.5 * np.sum((h - d) ** 2) / sigma**2
    assert abs(0.5 * (dd + hh - 2 * dh) - loss_xyz) <= 1e-12 * loss_xyz


def test_channel_weights_select_channels():
    s = np.sin(np.arange(64) * 0.3)
    z = np.zeros_like(s)
    h_a = np.stack([s, z, -s])  # pure A
    d = oracle.aet(_series(5, 64))
    dh, hh = oracle.like_inner(h_a, d, (0.0, 1.0, 1.0))
    assert dh == 0.0 and hh == 0.0
    dh, hh = oracle.like_inner(h_a, d, (2.0, 0.0, 0.0))
    a = -math.sqrt(2) * s
    assert dh == pytest.approx(2.0 * np.dot(d[0], a), rel=1e-14)
    assert hh == pytest.approx(2.0 * np.dot(a, a), rel=1e-14)


def test_like_is_linear_in_the_data():
    h, d1, d2 = _series(6), _series(7), _series(8)
    w = (1.0, 2.0, 0.5)
    a, _ = oracle.like_inner(h, d1, w)
    b, _ = oracle.like_inner(h, d2, w)
    c, _ = oracle.like_inner(h, 3.0 * d1 - d2, w)
    assert c == pytest.approx(3.0 * a - b, rel=1e-12, abs=1e-12)
