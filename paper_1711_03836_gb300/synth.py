"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by
the oracle's tests.

This module only draws inputs; it contains none of the operator's arithmetic
(no hopping term, clover term or solver).  Recipes:

* links: U = exp(i eps A) with A = sum_a w_a lambda_a / 2, w_a ~ N(0, 1), drawn
  with numpy's PCG64 ``default_rng(seed)`` in lex order (site, mu, a); the
  exponential is torch's multithreaded matrix_exp on the CPU (scaling and
  squaring), then U is projected back onto SU(3) (Gram-Schmidt on rows 1-2,
  row 3 = conj(row1 x row2)).
* U(1) angles A_mu(x) ~ N(0, sigma^2), i.i.d.
* spinors: real and imaginary parts ~ N(0, 1), i.i.d. per component.

Site lex = x + Lx*(y + Ly*(z + Lz*t)); a field of one parity is indexed by
lex/2.  Layouts: links [V][4][3][3] complex128, U(1) [V][4] float64, spinors
[V/2][4][3] complex128.
"""
from __future__ import annotations

import numpy as np


def _gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


GELL_MANN = _gell_mann()


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def check_dims(dims) -> None:
    if len(dims) != 4 or any(int(d) < 2 or int(d) % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even numbers >= 2, got {dims}")


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Project [..., 3, 3] matrices onto SU(3): Gram-Schmidt rows 1-2, row 3 = conj(r1 x r2)."""
    r1 = U[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = U[..., 1, :]
    r2 = r2 - np.sum(r1.conj() * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.cross(r1, r2).conj()
    return np.stack([r1, r2, r3], axis=-2)


def su3_near_identity(n: int, eps: float, rng: np.random.Generator) -> np.ndarray:
    """n matrices exp(i eps A), A Gaussian traceless Hermitian, reunitarised."""
    import torch

    w = rng.standard_normal((n, 8))
    H = np.einsum("na,aij->nij", w, GELL_MANN / 2)
    U = torch.linalg.matrix_exp(torch.from_numpy(1j * eps * H)).numpy()
    return reunitarise(U)


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """Links [V][4][3][3] = reunitarised exp(i eps A), drawn in lex order (site, mu, a)."""
    check_dims(dims)
    n = volume(dims) * 4
    rng = np.random.default_rng(seed)
    U = np.empty((n, 3, 3), np.complex128)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        U[s:e] = su3_near_identity(e - s, eps, rng)
    return U.reshape(volume(dims), 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    check_dims(dims)
    U = np.zeros((volume(dims), 4, 3, 3), np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def random_su3(n: int, seed: int) -> np.ndarray:
    """n Haar-random SU(3) matrices (QR of a complex Gaussian, phases fixed, det set to 1)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[:, None, None]


def u1_field(dims, sigma: float, seed: int) -> np.ndarray:
    """U(1) angles A_mu(x) ~ N(0, sigma^2), shape [V][4]."""
    check_dims(dims)
    return np.random.default_rng(seed).normal(0.0, sigma, (volume(dims), 4))


def gaussian_spinor(n_sites: int, seed: int) -> np.ndarray:
    """[n][4][3] complex, Re and Im ~ N(0,1) i.i.d."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n_sites, 4, 3, 2))
    return z[..., 0] + 1j * z[..., 1]


def point_source(n_sites: int, site: int, spin: int, colour: int) -> np.ndarray:
    """Unit source at one half-lattice site, spin and colour."""
    b = np.zeros((n_sites, 4, 3), np.complex128)
    b[site, spin, colour] = 1.0
    return b


def lex_coords(dims) -> np.ndarray:
    """[V][4] integer coordinates (x, y, z, t) of every lex site."""
    V = volume(dims)
    lex = np.arange(V)
    c = np.empty((V, 4), np.int64)
    c[:, 0] = lex % dims[0]
    c[:, 1] = (lex // dims[0]) % dims[1]
    c[:, 2] = (lex // (dims[0] * dims[1])) % dims[2]
    c[:, 3] = lex // (dims[0] * dims[1] * dims[2])
    return c


def half_sites(dims, parity: int) -> np.ndarray:
    """lex index of each half-lattice site of the given parity, in half-index order."""
    c = lex_coords(dims)
    lex = np.arange(volume(dims))
    par = c.sum(axis=1) % 2
    sel = lex[par == parity]
    assert np.all(sel // 2 == np.arange(len(sel)))
    return sel


def z2_noise(n_sites: int, seed: int) -> np.ndarray:
    """Complex Z2 x Z2 noise [n][4][3]: each component (+-1 +- i)/sqrt(2), so that
    E[eta eta^dag] = 1 (the noise of stochastic trace estimates)."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, 2, (n_sites, 4, 3, 2)) * 2 - 1
    return (s[..., 0] + 1j * s[..., 1]) / np.sqrt(2.0)
