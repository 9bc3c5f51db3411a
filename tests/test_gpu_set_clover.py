"""A clover field supplied by the caller (bq_set_clover) against the FP64 oracle.

The caller's field is the oracle's clover term (Eq. 2) plus a random Hermitian
perturbation of each chirality block, so it differs from the field the library
would build from the links; Mhat, Mhat^dag and Mhat^dag Mhat through the C ABI
must match the oracle's even-odd operator assembled on that same field.
"""
import numpy as np
import pytest

import oracle
from helpers import pack_clover
from paper_1711_03836_gb300 import synth

TOL = {"double": 1e-13, "single": 1e-6, "half": 5e-3}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bq():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_03836_gb300 import bqcd

    return bqcd


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def perturbed(Am, rng, size=0.05):
    """Am plus a random Hermitian matrix on each 6x6 chirality block (commutes with gamma_5)."""
    out = Am.copy()
    for b in range(2):
        X = rng.normal(size=(len(Am), 6, 6)) + 1j * rng.normal(size=(len(Am), 6, 6))
        out[:, 6 * b:6 * b + 6, 6 * b:6 * b + 6] += size * (X + X.conj().transpose(0, 2, 1))
    return out


def setup(bq, dims, prec, recon, kappa=0.1355, csw=1.9, mu=0.0):
    U = synth.gauge_field(dims, 0.2, 1)
    lat = bq.Lattice(dims, kappa, csw, mu, -1.0)
    bq.bq_set_gauge(lat.ctx, U)
    bq.bq_set_recon(lat.ctx, prec, recon)
    p = oracle.params(dims, kappa=kappa, csw=csw, mu=mu, t_bc=-1.0)
    return lat, U, p


def check_mhat(bq, lat, op, prec, seed=5):
    psi = synth.gaussian_spinor(lat.Vh, seed)
    src = lat.pack(psi, prec)
    out = lat.spinor(prec)
    errs = []
    for dag in (False, True):
        bq.bq_apply_mhat(lat.ctx, out, src, dag, prec)
        errs.append(rel(lat.unpack(out, prec), op.mhat(psi, dag)))
    bq.bq_apply_mdagm(lat.ctx, out, src, prec)
    errs.append(rel(lat.unpack(out, prec), op.mdagm(psi)))
    return max(errs)


@pytest.mark.parametrize("prec,recon,mu", [("double", 18, 0.0), ("single", 12, 0.1), ("half", 12, 0.0)])
def test_set_clover_perturbed_field(bq, prec, recon, mu):
    dims = (6, 4, 6, 10)
    lat, U, p = setup(bq, dims, prec, recon, mu=mu)
    op = oracle.Operator(p, U)
    built = (op.Aee, op.Aoo, op.Aoo_inv)
    rng = np.random.default_rng(11)
    Ae, Ao = perturbed(op.Aee, rng), perturbed(op.Aoo, rng)
    bq.bq_set_clover(lat.ctx, pack_clover(dims, Ae, Ao))
    op.Aee, op.Aoo, op.Aoo_inv = Ae, Ao, oracle.clover_invert(Ao)
    assert check_mhat(bq, lat, op, prec) < TOL[prec]
    # the perturbation is visible: the built field gives a different operator
    psi = synth.gaussian_spinor(lat.Vh, 5)
    op_built = oracle.Operator(p, U)
    assert rel(op.mhat(psi), op_built.mhat(psi)) > 1e-3
    # the caller's field stays when kappa changes (only the hopping coefficient moves)
    bq.bq_set_params(lat.ctx, 0.12, 1.9, mu, -1.0)
    p2 = oracle.params(dims, kappa=0.12, csw=1.9, mu=mu, t_bc=-1.0)
    op2 = oracle.Operator(p2, U)
    op2.Aee, op2.Aoo, op2.Aoo_inv = Ae, Ao, op.Aoo_inv
    assert check_mhat(bq, lat, op2, prec) < TOL[prec]
    # NULL goes back to the clover term built from the links
    bq.bq_set_params(lat.ctx, 0.1355, 1.9, mu, -1.0)
    bq.bq_set_clover(lat.ctx, None)
    op.Aee, op.Aoo, op.Aoo_inv = built
    assert check_mhat(bq, lat, op, prec) < TOL[prec]
    lat.close()


def test_set_clover_device_field_logdet_and_built_equivalence(bq):
    import torch

    dims = (8, 8, 8, 8)
    lat, U, p = setup(bq, dims, "double", 18)
    op = oracle.Operator(p, U)
    # the built field itself, passed in from device memory, gives the same operator
    packed = torch.from_numpy(pack_clover(dims, op.Aee, op.Aoo)).cuda()
    bq.bq_set_clover(lat.ctx, packed)
    assert check_mhat(bq, lat, op, "double") < TOL["double"]
    # a perturbed field: log det of both parities against dense slogdet of the 12x12 matrices
    rng = np.random.default_rng(3)
    Ae, Ao = perturbed(op.Aee, rng, 0.1), perturbed(op.Aoo, rng, 0.1)
    bq.bq_set_clover(lat.ctx, torch.from_numpy(pack_clover(dims, Ae, Ao)).cuda())
    for par, Am in ((0, Ae), (1, Ao)):
        ld, neg = bq.bq_clover_logdet(lat.ctx, par)
        sign, ref = np.linalg.slogdet(Am)
        assert abs(ld - np.sum(ref)) <= 1e-12 * max(1.0, abs(np.sum(ref))), par
        # block determinants are real (Hermitian blocks); count the negative ones
        nb = sum(int(np.sum(np.linalg.det(Am[:, 6 * b:6 * b + 6, 6 * b:6 * b + 6]).real < 0)) for b in range(2))
        assert neg == nb
    lat.close()


def test_set_clover_singular_block_falls_back(bq):
    dims = (4, 4, 4, 4)
    lat, U, p = setup(bq, dims, "double", 18)
    op = oracle.Operator(p, U)
    Ae, Ao = op.Aee.copy(), op.Aoo.copy()
    Ao[3, 6:, 6:] = 0.0  # one odd site's lower chirality block has no inverse
    with pytest.raises(bq.BqError) as e:
        bq.bq_set_clover(lat.ctx, pack_clover(dims, Ae, Ao))
    assert e.value.status == bq.BQ_ERR_CLOVER_SINGULAR
    # the context went back to the clover term built from the links
    assert check_mhat(bq, lat, op, "double") < TOL["double"]
    with pytest.raises(bq.BqError) as e:
        bq._check(bq._lib_handle().bq_set_clover(lat.ctx, None, 7), "bq_set_clover")
    assert e.value.status == bq.BQ_ERR_ARG
    lat.close()


def test_set_clover_in_batched_and_multishift_solves(bq):
    """A caller's clover field drives the solvers too: two systems in one batched
    mixed-precision CG (shared-memory tile mapping) and a two-shift multishift
    solve, each to a true residual <= 1e-10 of the oracle operator on that field."""
    dims = (6, 4, 6, 10)
    lat, U, p = setup(bq, dims, "single", 12)
    op = oracle.Operator(p, U)
    rng = np.random.default_rng(5)
    Ae, Ao = perturbed(op.Aee, rng), perturbed(op.Aoo, rng)
    bq.bq_set_clover(lat.ctx, pack_clover(dims, Ae, Ao))
    op.Aee, op.Aoo, op.Aoo_inv = Ae, Ao, oracle.clover_invert(Ao)
    bq.bq_set_batch_mapping(lat.ctx, -3)
    bs = [synth.gaussian_spinor(lat.Vh, 60 + i) for i in range(2)]
    xs = [np.empty_like(b) for b in bs]
    st = bq.bq_solve_cg_batch([lat.ctx] * 2, xs, bs, tol=1e-10, precision="single")
    for b, x, s in zip(bs, xs, st):
        assert s["converged"] and np.linalg.norm(op.mdagm(x) - b) / np.linalg.norm(b) <= 1e-10
    shifts = [0.01, 0.2]
    xm = [np.empty_like(bs[0]) for _ in shifts]
    bq.bq_solve_multishift_cg(lat.ctx, xm, bs[0], shifts, tol=1e-10, precision="single")
    for x, sh in zip(xm, shifts):
        assert np.linalg.norm(op.mdagm(x, sh) - bs[0]) / np.linalg.norm(bs[0]) <= 1e-10
    lat.close()
