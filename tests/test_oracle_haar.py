"""Pins of the oracle's Haar transform (Eq. 1.2, mu = Omega beta; Results:
level-L Haar) against a hand-derived example, orthonormality, perfect
reconstruction and the explicit basis-function definition."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import haar

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_derived_2x2():
    g = json.load(open(os.path.join(GOLD, "haar_2x2.json")))
    img = np.array(g["image"])
    beta = haar.analysis(img, g["levels"])
    np.testing.assert_allclose(beta, g["coefficients"], atol=1e-15)
    np.testing.assert_allclose(haar.synthesis(beta, 2, 2, 1), img, atol=1e-15)


@pytest.mark.parametrize("nx,ny,L", [(8, 8, 3), (48, 40, 3), (64, 32, 2), (16, 48, 4)])
def test_orthonormal_and_perfect_reconstruction(nx, ny, L):
    Om = haar.basis_matrix(nx, ny, L)
    N = nx * ny
    assert abs(Om.T @ Om - sp.identity(N)).max() < 1e-14
    rng = np.random.default_rng(nx + ny + L)
    x = rng.standard_normal((ny, nx))
    b = haar.analysis(x, L)
    np.testing.assert_allclose(haar.synthesis(b, nx, ny, L), x, atol=1e-13)
    # Parseval
    assert abs(np.dot(b, b) - np.sum(x * x)) < 1e-10 * np.sum(x * x)
    # butterfly synthesis == explicit basis (two independent codings)
    beta = rng.standard_normal(N)
    np.testing.assert_allclose(Om @ beta, haar.synthesis(beta, nx, ny, L).ravel(), atol=1e-13)
    np.testing.assert_allclose(Om.T @ x.ravel(), b, atol=1e-13)


def test_constant_image_lives_in_approximations():
    nx, ny, L = 32, 16, 3
    b = haar.analysis(np.full((ny, nx), 0.7), L)
    n_a = (nx >> L) * (ny >> L)
    np.testing.assert_allclose(b[:n_a], 0.7 * 2 ** L, atol=1e-13)
    np.testing.assert_allclose(b[n_a:], 0.0, atol=1e-13)


def test_basis_function_shapes():
    # the level-2 'v' detail of block (by=1, bx=2) of a 16x16 image is
    # +1/4 on the left half (x = 8..9), -1/4 on the right (x = 10..11),
    # rows y = 4..7, zero elsewhere
    nx = ny = 16
    L = 3
    planes = haar.layout(nx, ny, L)
    (lvl, t, off, r, c), = [p for p in planes if p[0] == 2 and p[1] == 1]
    z = off + 1 * c + 2
    e = np.zeros(nx * ny)
    e[z] = 1.0
    img = haar.synthesis(e, nx, ny, L)
    want = np.zeros((ny, nx))
    want[4:8, 8:10] = 0.25
    want[4:8, 10:12] = -0.25
    np.testing.assert_allclose(img, want, atol=1e-15)
    # and the level-1 'h' detail of block (by=0, bx=0): +1/2 on row 0, -1/2 on row 1
    (lvl, t, off, r, c), = [p for p in planes if p[0] == 1 and p[1] == 0]
    e[:] = 0
    e[off] = 1.0
    want = np.zeros((ny, nx))
    want[0, 0:2] = 0.5
    want[1, 0:2] = -0.5
    np.testing.assert_allclose(haar.synthesis(e, nx, ny, L), want, atol=1e-15)
