"""Pins for the block-assembly oracle (75 statements of affine combinations, Listing 2 shape)."""
import numpy as np
import pytest

import oracle
from paper_2306_13002_gb300 import inputs

DYADIC = (0.5, 2.0, 4.0, 0.25, 0.5)          # dt, q1, q2, q3, q4 -> t1 = 1, t2 = 2


def closed_form(A, B, G, halo=1):
    """The block body with t1 = 1, t2 = 2, q3 = 1/4, q4 = 1/2 written as whole-array shifts."""
    h = halo
    Am, A0, Ap = A[:, h - 1:-h - 1, h:-h, h:-h], A[:, h:-h, h:-h, h:-h], A[:, h + 1:A.shape[1] - h + 1, h:-h, h:-h]
    Bm, B0, Bp = B[:, h - 1:-h - 1, h:-h, h:-h], B[:, h:-h, h:-h, h:-h], B[:, h + 1:B.shape[1] - h + 1, h:-h, h:-h]
    g = G[h:-h, h:-h, h:-h]
    eye = np.eye(5).reshape(25, 1, 1, 1)
    L = -2.0 * Am - Bm - 0.25 * g * eye
    D = 2.0 * B0 - A0 + eye * (1.0 + 0.5 * g)
    W = 2.0 * Ap - Bp - 0.25 * g * eye
    return np.concatenate([L, D, W])


def _int_fields(nx, ny, nz, halo=1, seed=0):
    rng = np.random.default_rng(seed)
    sh = (nz + 2 * halo, ny + 2 * halo, nx + 2 * halo)
    A = rng.integers(-64, 64, size=(25,) + sh).astype(np.float64)
    B = rng.integers(-64, 64, size=(25,) + sh).astype(np.float64)
    G = rng.integers(1, 16, size=sh).astype(np.float64)
    return A, B, G


@pytest.fixture
def orc():
    return oracle.default()


def test_block_closed_form_exact_on_integers(orc):
    A, B, G = _int_fields(5, 4, 6)
    np.testing.assert_array_equal(orc.block(A, B, G, prm=DYADIC), closed_form(A, B, G))


def test_block_zero_blocks_give_identity_structure(orc):
    A = np.zeros((25, 5, 4, 6))
    B = np.zeros_like(A)
    G = np.full((5, 4, 6), 2.0)
    out = orc.block(A, B, G, prm=DYADIC)
    eye = np.eye(5).reshape(25)
    for q in range(25):
        assert np.all(out[q] == -0.5 * eye[q])
        assert np.all(out[25 + q] == eye[q] * 2.0)
        assert np.all(out[50 + q] == -0.5 * eye[q])


def test_block_general_params_within_rounding(orc):
    A, B, G = inputs.block_fields(4, 3, 5)
    dt, q1, q2, q3, q4 = 0.013, 1.7, 2.3, 0.61, 0.37
    out = orc.block(A, B, G, prm=(dt, q1, q2, q3, q4))
    t1, t2 = dt * q1, dt * q2
    h = 1
    eye = np.eye(5).reshape(25, 1, 1, 1)
    g = G[h:-h, h:-h, h:-h]
    L = -t2 * A[:, :-2, h:-h, h:-h] - t1 * B[:, :-2, h:-h, h:-h] - t1 * q3 * g * eye
    D = 2 * t1 * B[:, 1:-1, h:-h, h:-h] - q4 * t2 * A[:, 1:-1, h:-h, h:-h] + eye * (1 + 2 * t1 * q3 * g)
    W = t2 * A[:, 2:, h:-h, h:-h] - t1 * B[:, 2:, h:-h, h:-h] - t1 * q3 * g * eye
    np.testing.assert_allclose(out, np.concatenate([L, D, W]), rtol=1e-14, atol=1e-15)


def test_block_translation_and_padding(orc):
    A, B, G = inputs.block_fields(5, 4, 6, seed=3)
    out = orc.block(A, B, G)
    np.testing.assert_array_equal(orc.block(A[:, 1:], B[:, 1:], G[1:]), out[:, 1:])
    Ap, Bp, Gp = (inputs.pad_rows(x, x.shape[-1] + 3) for x in (A, B, G))
    np.testing.assert_array_equal(orc.block(Ap, Bp, Gp), out)
