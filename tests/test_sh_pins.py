"""Pins of the real spherical-harmonic colour basis (degrees 0-3) used for the
view-dependent colour (Sec. 3: each Gaussian carries SH colour coefficients).

Both oracles (the C oracle's basis and the gradient oracle's PyTorch basis)
are checked against what the mathematics fixes, not against each other:
- the definition of the real basis through associated Legendre functions
  (scipy's ``lpmv``, with its Condon-Shortley phase removed so that every
  normalisation constant is positive), in l-major order, m = -l..l, with
  sin(|m| phi) for m < 0 and cos(m phi) for m > 0, where phi is the azimuth of
  (x, y) and theta the polar angle from z;
- orthonormality on the sphere, by a product rule exact for these degrees
  (Gauss-Legendre in cos(theta) x trapezoid in phi);
- each |x|^l Y_lm(x/|x|) is a harmonic polynomial: its Laplacian, taken by
  central differences (exact for polynomials up to degree 3), vanishes.
A dropped term, a swapped constant or a wrong polynomial (3z^2 - 1 against
5z^2 - 3, say) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle

LM = [(l, m) for l in range(4) for m in range(-l, l + 1)]


def _grad_oracle_basis(v):
    import torch
    from oracle import grad as G
    return G._sh_basis(torch.as_tensor(v, dtype=torch.float64), 3).numpy()


BASES = {"c_oracle": oracle.sh_basis, "grad_oracle": _grad_oracle_basis}


def _legendre_real_sh(v):
    """Real SH from associated Legendre functions (textbook definition)."""
    v = np.asarray(v, np.float64)
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    phi = np.arctan2(y, x)
    out = np.zeros((v.shape[0], 16))
    for k, (l, m) in enumerate(LM):
        am = abs(m)
        norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
        P = sps.lpmv(am, l, z) * (-1.0) ** am           # remove the Condon-Shortley phase
        if m == 0:
            out[:, k] = norm * P
        elif m > 0:
            out[:, k] = math.sqrt(2.0) * norm * P * np.cos(am * phi)
        else:
            out[:, k] = math.sqrt(2.0) * norm * P * np.sin(am * phi)
    return out


def _unit(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("which", list(BASES))
def test_sh_basis_matches_legendre_definition(which):
    v = _unit(500, 1)
    # include the poles and the coordinate axes, where the azimuth is degenerate
    v = np.concatenate([v, np.eye(3), -np.eye(3)])
    got = BASES[which](v)
    want = _legendre_real_sh(v)
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("which", list(BASES))
def test_sh_basis_orthonormal_on_the_sphere(which):
    # Y_i Y_j has degree <= 6: 8 Gauss-Legendre nodes in cos(theta) and 16 azimuths are exact
    ct, wt = np.polynomial.legendre.leggauss(8)
    phi = np.arange(16) * (2 * math.pi / 16)
    C, PH = np.meshgrid(ct, phi, indexing="ij")
    S = np.sqrt(1 - C * C)
    v = np.stack([S * np.cos(PH), S * np.sin(PH), C], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(16, 2 * math.pi / 16)[None, :]).reshape(-1)
    Y = BASES[which](v)
    gram = (Y * w[:, None]).T @ Y
    assert np.abs(gram - np.eye(16)).max() < 1e-12


@pytest.mark.parametrize("which", list(BASES))
def test_sh_basis_harmonic_homogeneous_polynomials(which):
    basis = BASES[which]
    deg = np.array([l for l, _ in LM])
    rng = np.random.default_rng(3)
    pts = rng.normal(size=(40, 3))
    pts *= (0.7 + 0.6 * rng.random((40, 1))) / np.linalg.norm(pts, axis=1, keepdims=True)

    def P(x):  # homogeneous extension |x|^l Y_lm(x/|x|)
        r = np.linalg.norm(x, axis=1, keepdims=True)
        return basis(x / r) * r ** deg[None, :]

    h = 1e-2
    lap = np.zeros((pts.shape[0], 16))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lap += (P(pts + e) + P(pts - e) - 2 * P(pts)) / (h * h)
    scale = np.abs(P(pts)).max(0) + 1.0
    assert (np.abs(lap).max(0) / scale).max() < 1e-8
    # homogeneity: scaling the point by c scales P by c^l (a check of the extension itself)
    assert np.allclose(P(2.0 * pts), P(pts) * 2.0 ** deg[None, :], rtol=1e-12, atol=1e-12)
    # and each degree-l function is not identically zero
    assert (np.abs(P(pts)).max(0) > 1e-3).all()
