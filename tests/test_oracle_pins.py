"""Pins of the FP64 CPU oracle against what the action and the mathematics fix.

Each test checks the oracle against something other than itself: the Clifford
algebra, the free-field closed form of the hopping term (Eq. 1), gamma_5
hermiticity, adjointness, gauge covariance (Eq. 1, Eq. 5), an abelian
background with an analytic field strength (Eq. 2), dense linear algebra on
small lattices and the dense spectral form of the multishift sum.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle
from paper_1711_03836_gb300 import synth
from helpers import (abelian_background, chiral_gammas, dense, free_dirac_symbol, gamma5_apply,
                     gauge_transform, plane_wave, rel, vdot)


# ---------------------------------------------------------------- gamma matrices

def test_gamma_clifford_algebra():
    g = [oracle.gamma(k) for k in range(5)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2 * np.eye(4) * (m == n))
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3])
    for m, gm in enumerate(chiral_gammas()):
        assert np.allclose(g[m], gm)


# ---------------------------------------------------------------- free field (Eq. 1)

@pytest.mark.parametrize("dims,t_bc,mu_chem", [
    ((4, 6, 2, 8), -1.0, 0.0),
    ((4, 6, 2, 8), -1.0, 0.1),
    ((2, 4, 4, 6), +1.0, 0.25),
])
def test_free_field_plane_wave(dims, t_bc, mu_chem):
    """D_hop on exp(i p.x) u equals (a - i gamma.b) u exp(i p.x), on both parities."""
    rng = np.random.default_rng(7)
    U = synth.unit_gauge(dims)
    p_ = oracle.params(dims, kappa=0.1, mu=mu_chem, t_bc=t_bc)
    gam = chiral_gammas()
    for trial in range(3):
        n = rng.integers(0, 8, 4)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi, p = plane_wave(dims, n, u, t_bc)
        Dp, _, _ = free_dirac_symbol(p, mu_chem, gam)
        expect = np.einsum("st,xta->xsa", Dp, psi)
        for out_par in (0, 1):
            src = psi[synth.half_sites(dims, 1 - out_par)]
            got = oracle.dhop(p_, U, None, src, out_par)
            assert rel(got, expect[synth.half_sites(dims, out_par)]) < 1e-13


@pytest.mark.parametrize("mu_chem,kappa", [(0.0, 0.125), (0.15, 0.11)])
def test_free_field_full_operator(mu_chem, kappa):
    """Without clover term (c_SW = 0, A = 1) the full matrix on exp(i p.x) u is
    (1 - kappa (a - i gamma.b)) u exp(i p.x), on the even and odd halves."""
    dims = (4, 2, 6, 8)
    rng = np.random.default_rng(17)
    U = synth.unit_gauge(dims)
    p_ = oracle.params(dims, kappa=kappa, csw=0.0, mu=mu_chem, t_bc=-1.0)
    op = oracle.Operator(p_, U)
    gam = chiral_gammas()
    ev, od = synth.half_sites(dims, 0), synth.half_sites(dims, 1)
    for trial in range(3):
        n = rng.integers(0, 8, 4)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi, p = plane_wave(dims, n, u, -1.0)
        Dp, _, _ = free_dirac_symbol(p, mu_chem, gam)
        expect = np.einsum("st,xta->xsa", np.eye(4) - kappa * Dp, psi)
        y_e, y_o = op.full(psi[ev], psi[od])
        assert rel(y_e, expect[ev]) < 1e-13
        assert rel(y_o, expect[od]) < 1e-13


@pytest.mark.parametrize("mu_chem,kappa", [(0.0, 0.125), (0.1, 0.2)])
def test_free_field_mhat_spectrum(mu_chem, kappa):
    """Dense spectrum of Mhat on 4^4 (U=1, antiperiodic t) equals the closed form
    1 - kappa^2 (a -+ i sqrt(b.b))^2, three-fold per momentum of the full zone."""
    dims = (4, 4, 4, 4)
    p_ = oracle.params(dims, kappa=kappa, csw=1.0, mu=mu_chem, t_bc=-1.0)
    op = oracle.Operator(p_, synth.unit_gauge(dims))
    Vh = oracle.half_volume(p_)
    ev = np.linalg.eigvals(dense(op.mhat, Vh))
    expect = []
    for n in np.ndindex(*dims):
        p = np.array([2 * np.pi * n[k] / dims[k] for k in range(4)])
        p[3] += np.pi / dims[3]
        pc = p.astype(complex)
        pc[3] -= 1j * mu_chem
        a = 2 * np.sum(np.cos(pc))
        bb = np.sqrt(np.sum((2 * np.sin(pc)) ** 2))
        for lam in (a - 1j * bb, a + 1j * bb):
            expect += [1 - kappa ** 2 * lam ** 2] * 3
    expect = np.array(expect)
    assert len(expect) == len(ev)
    cost = np.abs(expect[:, None] - ev[None, :])
    r, c = linear_sum_assignment(cost)
    assert cost[r, c].max() < 1e-8


# ---------------------------------------------------------------- operator identities

def _random_setup(dims, mu_chem=0.0, charge=0.0, csw=1.0, kappa=0.13, seed=1):
    U = synth.gauge_field(dims, 0.3, seed)
    A = synth.u1_field(dims, 0.1, seed + 7) if charge else None
    p_ = oracle.params(dims, kappa=kappa, csw=csw, mu=mu_chem, t_bc=-1.0, charge=charge)
    return p_, U, A


@pytest.mark.parametrize("charge", [0.0, 2.0 / 3.0])
def test_gamma5_hermiticity(charge):
    """gamma_5 Mhat gamma_5 = Mhat^dagger at mu = 0, tested with the non-adjoint path only."""
    dims = (4, 4, 4, 8)
    p_, U, A = _random_setup(dims, charge=charge)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    x = synth.gaussian_spinor(Vh, 11)
    y = synth.gaussian_spinor(Vh, 12)
    lhs = vdot(x, gamma5_apply(op.mhat(gamma5_apply(y))))
    rhs = vdot(op.mhat(x), y)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    # the hopping term alone: <x, g5 D g5 y> = <D x, y> between the two parities
    xo = synth.gaussian_spinor(Vh, 13)
    lhs = vdot(xo, gamma5_apply(oracle.dhop(p_, U, A, gamma5_apply(y), 1)))
    rhs = vdot(oracle.dhop(p_, U, A, xo, 0), y)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13


def test_gamma5_hermiticity_chemical_potential():
    """gamma_5 Mhat(mu) gamma_5 = Mhat(-mu)^dagger."""
    dims = (4, 4, 4, 8)
    p_, U, A = _random_setup(dims, mu_chem=0.1, charge=-1.0 / 3.0)
    pm = oracle.params(dims, kappa=p_.kappa, csw=p_.csw, mu=-0.1, t_bc=-1.0, charge=p_.charge)
    op, opm = oracle.Operator(p_, U, A), oracle.Operator(pm, U, A)
    Vh = oracle.half_volume(p_)
    x, y = synth.gaussian_spinor(Vh, 21), synth.gaussian_spinor(Vh, 22)
    lhs = vdot(x, gamma5_apply(op.mhat(gamma5_apply(y))))
    rhs = vdot(opm.mhat(x), y)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    # and the identity is not trivially true: Mhat(mu) itself is not gamma_5-hermitian
    rhs_wrong = vdot(op.mhat(x), y)
    assert abs(lhs - rhs_wrong) / abs(rhs) > 1e-4


@pytest.mark.parametrize("mu_chem,charge", [(0.0, 0.0), (0.1, 2.0 / 3.0)])
def test_adjoint(mu_chem, charge):
    """<x, Mhat y> = <Mhat^dagger x, y> with the independently written adjoint."""
    dims = (4, 4, 4, 8)
    p_, U, A = _random_setup(dims, mu_chem=mu_chem, charge=charge)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    x, y = synth.gaussian_spinor(Vh, 31), synth.gaussian_spinor(Vh, 32)
    lhs = vdot(x, op.mhat(y))
    rhs = vdot(op.mhat(x, dagger=True), y)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    for par in (0, 1):
        lhs = vdot(x, oracle.dhop(p_, U, A, y, par))
        rhs = vdot(oracle.dhop(p_, U, A, x, 1 - par, dagger=True), y)
        assert abs(lhs - rhs) / abs(rhs) < 1e-13


@pytest.mark.parametrize("mu_chem,charge", [(0.0, 0.0), (0.1, -1.0 / 3.0)])
def test_gauge_covariance(mu_chem, charge):
    """Mhat[U^G, A^theta] (g psi) = g Mhat[U, A] psi with g = e^{iQ theta} G (clover rebuilt)."""
    dims = (4, 4, 6, 4)
    p_, U, A = _random_setup(dims, mu_chem=mu_chem, charge=charge, csw=1.7)
    V = synth.volume(dims)
    G = synth.random_su3(V, 99)
    theta = np.random.default_rng(5).uniform(-np.pi, np.pi, V)
    Up, Ap = gauge_transform(dims, U, A, G, theta, charge)
    even = synth.half_sites(dims, 0)
    g = G[even] * np.exp(1j * charge * theta[even])[:, None, None]
    psi = synth.gaussian_spinor(len(even), 41)
    gpsi = np.einsum("xab,xsb->xsa", g, psi)
    out = oracle.Operator(p_, U, A).mhat(psi)
    outp = oracle.Operator(p_, Up, Ap).mhat(gpsi)
    assert rel(outp, np.einsum("xab,xsb->xsa", g, out)) < 1e-13
    # a non-covariant change (links transformed, spinor not) must fail
    assert rel(outp, out) > 1e-2


# ---------------------------------------------------------------- clover term (Eq. 2)

@pytest.mark.parametrize("mu,nu", [(0, 1), (0, 3), (1, 2), (2, 3)])
@pytest.mark.parametrize("dep_on", ["mu", "nu"])
def test_clover_abelian_background(mu, nu, dep_on):
    """Constant abelian field: every mu-nu plaquette is diag(e^{+-i phi c}) so
    F = traceless part of +-i sin(phi c), A = 1 + i kappa c_SW sigma_{mu nu} F."""
    dims = (4, 6, 4, 8)
    c = (1.0, 2.0, 0.0)
    U, phi = abelian_background(dims, mu, nu, 1, c, dep_on)
    kappa, csw = 0.13, 1.9
    p_ = oracle.params(dims, kappa=kappa, csw=csw)
    sign = 1.0 if dep_on == "mu" else -1.0
    F = 1j * sign * np.sin(phi * np.array(c))
    F = np.diag(F - F.mean())
    g = chiral_gammas()
    sigma = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
    expect = np.eye(12) + 1j * kappa * csw * np.kron(sigma, F)
    for par in (0, 1):
        Am = oracle.clover_field(p_, U, par)
        assert np.abs(Am - expect[None]).max() < 1e-14


def test_clover_properties_random_field():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 3)
    p_ = oracle.params(dims, kappa=0.1355, csw=1.9)
    Am = oracle.clover_field(p_, U, 1)
    g5 = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    assert np.abs(Am - Am.conj().transpose(0, 2, 1)).max() < 1e-14      # Hermitian
    assert np.abs(Am @ g5 - g5 @ Am).max() < 1e-14                       # [A, gamma_5] = 0
    assert np.abs(Am - np.eye(12)).max() > 1e-3
    Ai = oracle.clover_invert(Am)
    assert np.abs(Am @ Ai - np.eye(12)).max() < 1e-13
    assert np.abs(Ai - np.linalg.inv(Am)).max() < 1e-13
    p0 = oracle.params(dims, kappa=0.1355, csw=0.0)
    assert np.abs(oracle.clover_field(p0, U, 0) - np.eye(12)).max() == 0


# ---------------------------------------------------------------- even-odd reduction

def test_schur_complement_dense():
    """Mhat equals A_ee - kappa^2 D_eo A_oo^{-1} D_oe formed from dense blocks."""
    dims = (4, 4, 4, 4)
    p_, U, A = _random_setup(dims, mu_chem=0.05, charge=2.0 / 3.0)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    Doe = dense(lambda v: oracle.dhop(p_, U, A, v, 1), Vh)
    Deo = dense(lambda v: oracle.dhop(p_, U, A, v, 0), Vh)
    Aee = dense(lambda v: oracle.clover_apply(oracle.clover_field(p_, U, 0), v), Vh)
    Aoo = dense(lambda v: oracle.clover_apply(oracle.clover_field(p_, U, 1), v), Vh)
    Mhat = Aee - p_.kappa ** 2 * Deo @ np.linalg.solve(Aoo, Doe)
    got = dense(op.mhat, Vh)
    assert np.abs(got - Mhat).max() < 1e-12
    got_dag = dense(lambda v: op.mhat(v, dagger=True), Vh)
    assert np.abs(got_dag - Mhat.conj().T).max() < 1e-12


def test_special_cases():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 4)
    Vh = synth.volume(dims) // 2
    psi = synth.gaussian_spinor(Vh, 5)
    # kappa = 0: Mhat = A_ee = 1 (clover term is proportional to kappa)
    p0 = oracle.params(dims, kappa=0.0, csw=1.0)
    assert rel(oracle.Operator(p0, U).mhat(psi), psi) < 1e-15
    # Q = 0 with a U(1) field equals no U(1) field
    pq = oracle.params(dims, kappa=0.12, csw=1.0, charge=0.0)
    A = synth.u1_field(dims, 0.1, 6)
    assert rel(oracle.Operator(pq, U, A).mhat(psi), oracle.Operator(pq, U).mhat(psi)) < 1e-15
    # the U(1) field does change the operator when Q != 0
    pq2 = oracle.params(dims, kappa=0.12, csw=1.0, charge=2.0 / 3.0)
    assert rel(oracle.Operator(pq2, U, A).mhat(psi), oracle.Operator(pq, U).mhat(psi)) > 1e-3


def test_site_sampling_matches_full():
    dims = (4, 4, 6, 8)
    p_, U, A = _random_setup(dims, mu_chem=0.1, charge=2.0 / 3.0, csw=1.9)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    psi = synth.gaussian_spinor(Vh, 51)
    sites = np.array([0, 1, 7, Vh // 2, Vh - 1])
    for dag in (False, True):
        assert rel(oracle.mhat_sites(p_, U, A, psi, sites, dag), op.mhat(psi, dag)[sites]) < 1e-14
        for par in (0, 1):
            assert rel(oracle.dhop_sites(p_, U, A, psi, par, sites, dag),
                       oracle.dhop(p_, U, A, psi, par, dag)[sites]) < 1e-14
    for par in (0, 1):
        Am = oracle.clover_field(p_, U, par)
        assert rel(oracle.clover_sites(p_, U, par, psi, sites), oracle.clover_apply(Am, psi)[sites]) < 1e-14
        assert rel(oracle.clover_sites(p_, U, par, psi, sites, inverse=True),
                   oracle.clover_apply(oracle.clover_invert(Am), psi)[sites]) < 1e-14


# ---------------------------------------------------------------- solvers

def test_cg_matches_dense_solve():
    dims = (4, 4, 4, 4)
    p_, U, A = _random_setup(dims, csw=1.0, kappa=0.125)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    b = synth.gaussian_spinor(Vh, 61)
    x, it = op.cg(b, tol=1e-10)
    assert 0 < it < 1000
    K = dense(op.mdagm, Vh)
    xd = np.linalg.solve(K, b.ravel())
    cond = np.linalg.cond(K)
    assert rel(x.ravel(), xd) < cond * 1e-10
    assert rel(op.mdagm(x), b) <= 1e-10 * 1.01


@pytest.mark.parametrize("mu_chem,charge", [(0.0, 0.0), (0.1, 2.0 / 3.0)])
def test_full_solve_matches_dense(mu_chem, charge):
    """The block-eliminated full solve equals a dense solve of M on 4^4, and the
    Schur complement of M's odd block is Mhat."""
    dims = (4, 4, 4, 4)
    p_, U, A = _random_setup(dims, mu_chem=mu_chem, charge=charge, csw=1.2, kappa=0.125)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    n = Vh * 12
    Mfull = np.empty((2 * n, 2 * n), complex)
    for j in range(2 * n):
        e = np.zeros(2 * n, complex)
        e[j] = 1
        y_e, y_o = op.full(e[:n].reshape(Vh, 4, 3), e[n:].reshape(Vh, 4, 3))
        Mfull[:, j] = np.concatenate([y_e.ravel(), y_o.ravel()])
    S = Mfull[:n, :n] - Mfull[:n, n:] @ np.linalg.solve(Mfull[n:, n:], Mfull[n:, :n])
    assert np.abs(S - dense(op.mhat, Vh)).max() < 1e-12
    b_e, b_o = synth.gaussian_spinor(Vh, 81), synth.gaussian_spinor(Vh, 82)
    x_e, x_o = op.solve_full(b_e, b_o, tol=1e-12)
    xd = np.linalg.solve(Mfull, np.concatenate([b_e.ravel(), b_o.ravel()]))
    got = np.concatenate([x_e.ravel(), x_o.ravel()])
    assert rel(got, xd) < np.linalg.cond(Mfull) * 1e-11
    y_e, y_o = op.full(x_e, x_o)
    assert rel(np.concatenate([y_e.ravel(), y_o.ravel()]), np.concatenate([b_e.ravel(), b_o.ravel()])) < 1e-10


def test_multishift_matches_spectral_sum():
    """sum_k alpha_k (Mhat^dag Mhat + sigma_k)^{-1} b equals the dense eigen-sum."""
    dims = (4, 4, 4, 4)
    p_, U, A = _random_setup(dims, csw=1.0, kappa=0.125)
    op = oracle.Operator(p_, U, A)
    Vh = oracle.half_volume(p_)
    b = synth.gaussian_spinor(Vh, 71)
    shifts = 10.0 ** (-4 + 4 * np.arange(10) / 9)
    xs = op.multishift(b, shifts, tol=1e-11)
    K = dense(op.mdagm, Vh)
    lam, W = np.linalg.eigh(K)
    bw = W.conj().T @ b.ravel()
    expect = W @ (bw * sum(0.1 / (lam + s) for s in shifts))
    got = sum(0.1 * x.ravel() for x in xs)
    assert rel(got, expect) < 1e-9
    for x, s in zip(xs, shifts):
        assert rel(op.mdagm(x, s), b) <= 1e-11 * 1.01
