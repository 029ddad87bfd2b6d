"""Pins of the oracle's learned-probe network (plain numpy): the periodic
convolution against scipy's wrap-mode correlation, shift equivariance, the
width-1 layer as a matrix product, and the BF16 decoding."""
import numpy as np
import pytest

import oracle

scipy_nd = pytest.importorskip("scipy.ndimage")


def test_bf16_decoding():
    bits = np.array([0x3F80, 0xC000, 0x3F00, 0x0000, 0x4049], dtype=np.uint16)
    v = oracle.bf16_to_f64(bits)
    assert v[:4].tolist() == [1.0, -2.0, 0.5, 0.0]
    assert abs(v[4] - 3.140625) < 1e-12          # 0x4049 = 3.140625 exactly


def test_periodic_conv_is_wrap_correlation():
    g = np.random.default_rng(1)
    x = g.standard_normal((3, 37))
    W = g.standard_normal((2, 3, 5))
    b = g.standard_normal(2)
    y = oracle.periodic_conv1d(x, W, b)
    ref = np.zeros((2, 37))
    for o in range(2):
        ref[o] = b[o] + sum(scipy_nd.correlate1d(x[i], W[o, i], mode="wrap") for i in range(3))
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_periodic_conv_shift_equivariant_and_width_one():
    g = np.random.default_rng(2)
    x = g.standard_normal((4, 20))
    W = g.standard_normal((3, 4, 5))
    y = oracle.periodic_conv1d(x, W, np.zeros(3))
    assert np.allclose(oracle.periodic_conv1d(np.roll(x, 3, axis=1), W, np.zeros(3)), np.roll(y, 3, axis=1))
    W1 = g.standard_normal((6, 4, 1))
    assert np.allclose(oracle.periodic_conv1d(x, W1, np.ones(6)), W1[:, :, 0] @ x + 1.0)


def test_learned_probe_layout():
    """Output channel j(N+1)+t is time block t of column j."""
    n, N, m = 8, 2, 2
    Np1 = N + 1
    traj = np.arange(Np1 * n, dtype=np.float64).reshape(Np1, n)
    mask = np.zeros((Np1, n))
    W = [np.zeros((64, 2 * Np1, 5)), np.zeros((64, 64, 5)), np.zeros((64, 64, 5)), np.zeros((m * Np1, 64, 1))]
    b = [np.zeros(64), np.zeros(64), np.zeros(64), np.arange(m * Np1, dtype=np.float64)]
    S = oracle.learned_probes(traj, 8.0, mask, W, b, m)
    assert S.shape == (m, Np1 * n)
    for j in range(m):
        for t in range(Np1):
            assert np.all(S[j, t * n:(t + 1) * n] == j * Np1 + t)
