"""Shared test helpers: closed forms, plane waves, gauge transforms, dense matrices.

These helpers build test inputs and expected values from mathematics the
operator must satisfy; none of them calls the CUDA library.
"""
from __future__ import annotations

import numpy as np

from paper_1711_03836_gb300 import synth


def vdot(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def pauli():
    return [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]


def chiral_gammas():
    """gamma_1..4 of the chiral basis, typed from its definition."""
    g = []
    for s in pauli():
        m = np.zeros((4, 4), complex)
        m[:2, 2:] = -1j * s
        m[2:, :2] = 1j * s
        g.append(m)
    m = np.zeros((4, 4), complex)
    m[:2, 2:] = np.eye(2)
    m[2:, :2] = np.eye(2)
    g.append(m)
    return g


def gamma5_apply(psi):
    out = psi.copy()
    out[:, 2:, :] *= -1
    return out


def plane_wave(dims, n, u, t_bc):
    """psi(x) = exp(i p.x) u on the full lattice, p_i = 2 pi n_i / L_i, and
    p_4 = (2 pi n_4 + pi) / L_t for an antiperiodic time direction."""
    c = synth.lex_coords(dims)
    p = np.array([2 * np.pi * n[k] / dims[k] for k in range(4)])
    if t_bc < 0:
        p[3] += np.pi / dims[3]
    phase = np.exp(1j * (c @ p))
    return phase[:, None, None] * u[None, :, :], p


def free_dirac_symbol(p, mu_chem, gammas):
    """D(p) = a - i gamma.b with a = 2 sum cos p'_mu, b_mu = 2 sin p'_mu and
    p'_4 = p_4 - i mu (the chemical potential shifts p_4 into the complex plane)."""
    pc = p.astype(complex).copy()
    pc[3] -= 1j * mu_chem
    a = 2 * np.sum(np.cos(pc))
    b = 2 * np.sin(pc)
    return a * np.eye(4) - 1j * sum(b[m] * gammas[m] for m in range(4)), a, b


def gauge_transform(dims, U, A, G, theta, charge):
    """U'_mu(x) = G(x) U_mu(x) G(x+mu)^dag and A'_mu(x) = A_mu(x) + theta(x+mu) - theta(x)."""
    c = synth.lex_coords(dims)
    V = synth.volume(dims)
    Up = np.empty_like(U)
    Ap = None if A is None else np.empty_like(A)
    for mu in range(4):
        cc = c.copy()
        cc[:, mu] = (cc[:, mu] + 1) % dims[mu]
        fwd = cc[:, 0] + dims[0] * (cc[:, 1] + dims[1] * (cc[:, 2] + dims[2] * cc[:, 3]))
        Up[:, mu] = G @ U[:, mu] @ G[fwd].conj().transpose(0, 2, 1)
        if A is not None:
            Ap[:, mu] = A[:, mu] + theta[fwd] - theta
    return Up, Ap


def dense(apply, n_sites):
    """Dense matrix of a linear map on [n_sites][4][3] complex fields."""
    n = n_sites * 12
    M = np.empty((n, n), complex)
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        M[:, j] = np.ravel(apply(e.reshape(n_sites, 4, 3)))
    return M


def abelian_background(dims, mu, nu, m, c, dep_on):
    """U(3) background with U_nu(x) = diag(exp(i phi c_a x_mu)) (dep_on='mu') or
    U_mu(x) = diag(exp(i phi c_a x_nu)) (dep_on='nu'), every other link 1,
    phi = 2 pi m / L (L the extent of the coordinate it depends on)."""
    U = synth.unit_gauge(dims)
    co = synth.lex_coords(dims)
    c = np.asarray(c, float)
    if dep_on == "mu":
        phi = 2 * np.pi * m / dims[mu]
        ph = np.exp(1j * phi * co[:, mu][:, None] * c[None, :])
        U[:, nu] = 0
        U[:, nu, [0, 1, 2], [0, 1, 2]] = ph
    else:
        phi = 2 * np.pi * m / dims[nu]
        ph = np.exp(1j * phi * co[:, nu][:, None] * c[None, :])
        U[:, mu] = 0
        U[:, mu, [0, 1, 2], [0, 1, 2]] = ph
    return U, phi


def two_plane_background(dims, c12, c34, m):
    """Constant abelian field strength in the planes (0,1) and (2,3) at once:
    U_1(x) = diag(exp(i phi c12_a x_0)), U_3(x) = diag(exp(i phi' c34_a x_2)),
    every other link 1. Every plaquette of the other four planes is 1."""
    U, phi = abelian_background(dims, 0, 1, m, c12, "mu")
    U34, phi34 = abelian_background(dims, 2, 3, m, c34, "mu")
    U[:, 3] = U34[:, 3]
    return U, phi, phi34


def pack_clover(dims, A_even, A_odd):
    """The canonical clover field [V][2][36] (lex site order) of per-parity
    [V/2][12][12] matrices: per site and chirality block (spin components 0, 1
    and 2, 3) the 6 real diagonal entries, then the 15 complex entries above the
    diagonal row by row (re, im). A re-layout of the matrices, no arithmetic."""
    c = synth.lex_coords(dims)
    V = synth.volume(dims)
    par = c.sum(axis=1) % 2
    h = np.arange(V) // 2
    A = np.where((par == 0)[:, None, None], A_even[h], A_odd[h])
    out = np.empty((V, 2, 36))
    iu = np.triu_indices(6, 1)
    for b in range(2):
        B = A[:, 6 * b:6 * b + 6, 6 * b:6 * b + 6]
        out[:, b, :6] = np.real(np.diagonal(B, axis1=1, axis2=2))
        up = B[:, iu[0], iu[1]]
        out[:, b, 6::2] = up.real
        out[:, b, 7::2] = up.imag
    return out
