"""The seeded input generators follow their stated recipes: links in SU(3) near
the identity at the requested spread, reproducible by seed and independent of
the chunking; Gell-Mann generators normalised tr(l_a l_b) = 2 delta_ab; U(1)
angles, Gaussian spinors and Haar SU(3) with the moments of their
distributions; lex coordinates and half-lattice indexing consistent."""
import numpy as np
import pytest

from paper_1711_03836_gb300 import synth


def test_gell_mann_normalisation():
    lam = synth.GELL_MANN
    assert np.abs(lam - np.conj(np.swapaxes(lam, -1, -2))).max() == 0
    assert np.abs(np.trace(lam, axis1=-2, axis2=-1)).max() < 1e-15
    gram = np.einsum("aij,bji->ab", lam, lam)
    assert np.abs(gram - 2 * np.eye(8)).max() < 1e-14


@pytest.mark.parametrize("eps", [0.05, 0.2])
def test_gauge_field_su3_and_spread(eps):
    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, eps, 3)
    assert U.shape == (synth.volume(dims), 4, 3, 3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # |U - 1|_F^2 = eps^2 sum_a w_a^2 tr((l_a/2)^2) + O(eps^4): mean 4 eps^2
    d2 = np.sum(np.abs(U - np.eye(3)) ** 2, axis=(-2, -1))
    assert abs(d2.mean() / (4 * eps ** 2) - 1) < 0.05 + eps ** 2


def test_gauge_field_reproducible_and_chunk_independent():
    dims = (2, 4, 2, 4)
    a = synth.gauge_field(dims, 0.3, 11)
    b = synth.gauge_field(dims, 0.3, 11, chunk=7)
    c = synth.gauge_field(dims, 0.3, 12)
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() > 0.1


def test_reunitarise_projects_onto_su3():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((50, 3, 3)) + 1j * rng.standard_normal((50, 3, 3))
    U = synth.reunitarise(M)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    V = synth.random_su3(20, 1)
    assert np.abs(synth.reunitarise(V) - V).max() < 1e-14  # SU(3) is left alone


def test_random_su3_haar_moments():
    U = synth.random_su3(20000, 2)
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    # Haar measure: E|U_ij|^2 = 1/3, E U_ij = 0
    p = np.abs(U) ** 2
    assert np.abs(p.mean(axis=0) - 1 / 3).max() < 0.01
    assert np.abs(U.mean(axis=0)).max() < 0.02


def test_u1_spinor_and_point_source():
    dims = (8, 8, 8, 8)
    A = synth.u1_field(dims, 0.1, 4)
    assert A.shape == (synth.volume(dims), 4)
    assert abs(A.mean()) < 0.002 and abs(A.std() / 0.1 - 1) < 0.01
    z = synth.gaussian_spinor(20000, 5)
    assert z.shape == (20000, 4, 3)
    assert abs(np.mean(np.abs(z) ** 2) / 2 - 1) < 0.01
    assert abs(np.mean(z.real * z.imag)) < 0.01
    b = synth.point_source(10, 3, 2, 1)
    assert b[3, 2, 1] == 1 and np.count_nonzero(b) == 1


def test_lex_coords_and_half_sites():
    dims = (4, 2, 6, 8)
    c = synth.lex_coords(dims)
    lex = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * (c[:, 2] + dims[2] * c[:, 3]))
    assert np.array_equal(lex, np.arange(synth.volume(dims)))
    for par in (0, 1):
        s = synth.half_sites(dims, par)
        assert len(s) == synth.volume(dims) // 2
        assert np.all(c[s].sum(axis=1) % 2 == par)
    assert np.array_equal(np.sort(np.concatenate([synth.half_sites(dims, 0), synth.half_sites(dims, 1)])),
                          np.arange(synth.volume(dims)))
    with pytest.raises(ValueError):
        synth.check_dims((4, 4, 3, 4))
