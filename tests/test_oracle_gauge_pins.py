"""Pins of the oracle's stout smearing and clover log det.

Stout smearing (the singly iterated stout links of the QCD+QED fermion action,
Eq. 5; Morningstar and Peardon 2004) is checked against a closed form on
diagonal (abelian) SU(3) fields, where every matrix commutes and each link
phase moves by the imaginary part of its staple sum; against gauge covariance;
and against the group property of the result. The clover log det (Eq. 2) is
checked against the closed form of a constant abelian field strength.
"""
import numpy as np
import pytest

import oracle
from paper_1711_03836_gb300 import synth
from helpers import abelian_background, gauge_transform, two_plane_background


def _neighbour(dims, mu, d):
    """lex index of x + d mu-hat for every lex site x (periodic)."""
    c = synth.lex_coords(dims)
    c[:, mu] = (c[:, mu] + d) % dims[mu]
    return c[:, 0] + dims[0] * (c[:, 1] + dims[1] * (c[:, 2] + dims[2] * c[:, 3]))


def test_stout_rho_zero_and_unit_gauge():
    dims = (4, 2, 4, 6)
    U = synth.gauge_field(dims, 0.3, 2)
    assert np.array_equal(oracle.stout(dims, U, 0.0, 1), U)
    one = synth.unit_gauge(dims)
    assert np.abs(oracle.stout(dims, one, 0.2, 2) - one).max() < 1e-15


@pytest.mark.parametrize("rho", [0.1, 0.25])
def test_stout_abelian_closed_form(rho):
    """Diagonal links diag(e^{i theta_a}), sum_a theta_a = 0: the smeared phase is
    theta_a + Im w_a - (1/3) sum_b Im w_b with w_a = rho e^{-i theta_a(x,mu)} times
    the sum of the staple phases."""
    dims = (4, 6, 2, 4)
    rng = np.random.default_rng(11)
    V = synth.volume(dims)
    th = rng.normal(0, 0.7, (V, 4, 3))
    th -= th.mean(axis=2, keepdims=True)
    U = np.zeros((V, 4, 3, 3), complex)
    for a in range(3):
        U[:, :, a, a] = np.exp(1j * th[:, :, a])
    w = np.zeros((V, 4, 3), complex)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            xpn, xpm, xmn = _neighbour(dims, nu, 1), _neighbour(dims, mu, 1), _neighbour(dims, nu, -1)
            xmn_pm = _neighbour(dims, mu, 1)[xmn]
            up = th[:, nu] + th[xpn, mu] - th[xpm, nu]
            lo = -th[xmn, nu] + th[xmn, mu] + th[xmn_pm, nu]
            w[:, mu] += np.exp(1j * up) + np.exp(1j * lo)
        w[:, mu] *= rho * np.exp(-1j * th[:, mu])
    q = w.imag - w.imag.mean(axis=2, keepdims=True)
    expect = np.zeros_like(U)
    for a in range(3):
        expect[:, :, a, a] = np.exp(1j * (th[:, :, a] + q[:, :, a]))
    got = oracle.stout(dims, U, rho, 1)
    assert np.abs(got - expect).max() < 1e-14


def test_stout_gauge_covariance_and_group():
    dims = (4, 4, 2, 6)
    U = synth.gauge_field(dims, 0.4, 7)
    G = synth.gauge_field(dims, 2.0, 8)[:, 0]
    Ug, _ = gauge_transform(dims, U, None, G, None, 0.0)
    S = oracle.stout(dims, U, 0.15, 2)
    Sg = oracle.stout(dims, Ug, 0.15, 2)
    expect, _ = gauge_transform(dims, S, None, G, None, 0.0)
    assert np.abs(Sg - expect).max() < 1e-13
    eye = np.eye(3)
    assert np.abs(S @ np.conj(np.swapaxes(S, -1, -2)) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(S) - 1).max() < 1e-14
    assert np.abs(S - U).max() > 1e-2  # smearing moved the links


def test_clover_logdet_closed_form():
    """Constant abelian field: A = 1 + i kappa c_SW sigma_{mu nu} x F, F = i diag(f_a),
    sigma_{mu nu} has eigenvalues +-1 twice, so det A(x) = prod_a (1 - (kappa c_SW f_a)^2)^2."""
    dims = (4, 6, 4, 8)
    c = (1.0, 2.0, 0.0)
    U, phi = abelian_background(dims, 0, 1, 1, c, "mu")
    kappa, csw = 0.13, 1.9
    p_ = oracle.params(dims, kappa=kappa, csw=csw)
    f = np.sin(phi * np.array(c))
    f -= f.mean()
    per_site = 2 * np.sum(np.log(1 - (kappa * csw * f) ** 2))
    for par in (0, 1):
        ld, neg = oracle.clover_logdet(p_, U, par)
        assert abs(ld - per_site * synth.volume(dims) / 2) < 1e-11 * abs(per_site * synth.volume(dims))
        assert neg == 0
    ld0, _ = oracle.clover_logdet(oracle.params(dims, kappa=kappa, csw=0.0), synth.gauge_field(dims, 0.3, 1), 0)
    assert ld0 == 0.0


def test_clover_logdet_two_planes_negative():
    """F_12 = i diag(g_a), F_34 = i diag(g'_a) commute, and so do sigma_12 and
    sigma_34 (eigenvalues +-1 each, every sign pair once per colour), so the 12x12
    clover matrix has eigenvalues 1 - kc (s g_a + s' g'_a) and
    det A(x) = prod_a (1 - kc^2 (g_a + g'_a)^2) (1 - kc^2 (g_a - g'_a)^2),
    independent of the gamma basis. With g = g' = (2/3, -1/3, -1/3) and kc = 1
    exactly one factor is negative: every site has det A(x) < 0."""
    dims = (4, 4, 4, 6)
    c = (1.0, 0.0, 0.0)
    U, phi, phi34 = two_plane_background(dims, c, c, 1)
    assert abs(phi - np.pi / 2) < 1e-15 and abs(phi34 - np.pi / 2) < 1e-15
    kappa, csw = 0.25, 4.0
    kc = kappa * csw
    g = np.sin(phi * np.array(c))
    g -= g.mean()
    gp = np.sin(phi34 * np.array(c))
    gp -= gp.mean()
    det_site = np.prod((1 - kc ** 2 * (g + gp) ** 2) * (1 - kc ** 2 * (g - gp) ** 2))
    assert det_site < 0
    p_ = oracle.params(dims, kappa=kappa, csw=csw)
    for par in (0, 1):
        ld, neg = oracle.clover_logdet(p_, U, par)
        n = synth.volume(dims) // 2
        assert abs(ld - n * np.log(abs(det_site))) < 1e-12 * n
        assert neg == n
    # a positive case of the same form: kc = 0.5 leaves every factor positive
    ld, neg = oracle.clover_logdet(oracle.params(dims, kappa=0.125, csw=4.0), U, 0)
    det_pos = np.prod((1 - 0.25 * (g + gp) ** 2) * (1 - 0.25 * (g - gp) ** 2))
    assert neg == 0 and abs(ld - synth.volume(dims) // 2 * np.log(det_pos)) < 1e-12 * synth.volume(dims)


# ---------------------------------------------------------------- stochastic traces

def _dense_full(op, Vh):
    n = Vh * 12
    M = np.empty((2 * n, 2 * n), complex)
    for j in range(2 * n):
        e = np.zeros(2 * n, complex)
        e[j] = 1
        y_e, y_o = op.full(e[:n].reshape(Vh, 4, 3), e[n:].reshape(Vh, 4, 3))
        M[:, j] = np.concatenate([y_e.ravel(), y_o.ravel()])
    return M


@pytest.mark.parametrize("mu_chem,charge", [(0.0, 0.0), (0.2, 2.0 / 3.0)])
def test_trace_samples_sum_to_dense_traces(mu_chem, charge):
    """Summed over every unit vector (exact probing), the three samples give
    Tr M^{-1}, Tr gamma_5 M^{-1} and Tr (M^dag M)^{-1} of the dense matrix; the
    adjoint operator is the dense conjugate transpose."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.4, 3)
    A = synth.u1_field(dims, 0.1, 4) if charge else None
    p_ = oracle.params(dims, kappa=0.12, csw=1.3, mu=mu_chem, t_bc=-1.0, charge=charge)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    n = Vh * 12
    M = _dense_full(op, Vh)
    rng = np.random.default_rng(5)
    xe, xo = [rng.standard_normal((Vh, 4, 3)) + 1j * rng.standard_normal((Vh, 4, 3)) for _ in range(2)]
    ye, yo = op.full_dagger(xe, xo)
    got = np.concatenate([ye.ravel(), yo.ravel()])
    assert np.abs(got - M.conj().T @ np.concatenate([xe.ravel(), xo.ravel()])).max() < 1e-12
    tot = np.zeros(3, complex)
    for j in range(2 * n):
        e = np.zeros(2 * n, complex)
        e[j] = 1
        tot += op.trace_samples(e[:n].reshape(Vh, 4, 3), e[n:].reshape(Vh, 4, 3), tol=1e-13)
    Mi = np.linalg.inv(M)
    G5 = np.kron(np.eye(2 * Vh), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    assert abs(tot[0] - np.trace(Mi)) < 1e-9 * abs(np.trace(Mi))
    assert abs(tot[1] - np.trace(G5 @ Mi)) < 1e-9 * np.abs(Mi).sum()
    sv = np.linalg.svd(M, compute_uv=False)
    assert abs(tot[2] - np.sum(sv ** -2.0)) < 1e-9 * np.sum(sv ** -2.0)
    # one Z2 noise vector, sample by sample: eta^dag M^-1 eta, eta^dag g5 M^-1 eta and
    # eta^dag (M^dag M)^-1 eta (not (M M^dag)^-1, which has the same trace)
    eta_e, eta_o = synth.z2_noise(Vh, 41), synth.z2_noise(Vh, 42)
    eta = np.concatenate([eta_e.ravel(), eta_o.ravel()])
    got = op.trace_samples(eta_e, eta_o, tol=1e-13)
    expect = [np.vdot(eta, Mi @ eta), np.vdot(eta, G5 @ Mi @ eta), np.vdot(eta, np.linalg.solve(M.conj().T @ M, eta))]
    for g, e in zip(got, expect):
        assert abs(g - e) < 1e-8 * abs(expect[2])
    assert abs(np.vdot(eta, np.linalg.solve(M @ M.conj().T, eta)) - expect[2]) > 1e-6 * abs(expect[2])


def test_z2_noise_moments():
    eta = synth.z2_noise(20000, 3)
    assert np.allclose(np.abs(eta), 1.0)
    flat = eta.reshape(-1, 12)
    C = flat.T @ flat.conj() / flat.shape[0]
    assert np.abs(C - np.eye(12)).max() < 0.03
