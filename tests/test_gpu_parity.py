"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative 2-norm error per apply against the FP64 oracle):
FP64 1e-13, FP32 1e-6, FP16 storage with per-site scale 5e-3.
Small lattices are compared element by element on every site; they span
several 128-thread blocks and leave a ragged tail (V/2 = 720).
"""
import numpy as np
import pytest

import oracle
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


def make(bq, dims, kappa=0.1355, csw=1.9, mu=0.0, charge=0.0, eps=0.2, seed=1, recon=18, precision="double"):
    U = synth.gauge_field(dims, eps, seed)
    A = synth.u1_field(dims, 0.1, seed + 5) if charge else None
    lat = bq.Lattice(dims, kappa, csw, mu, -1.0, charge)
    bq.bq_set_gauge(lat.ctx, U)
    if A is not None:
        bq.bq_set_u1(lat.ctx, A)
    bq.bq_set_recon(lat.ctx, precision, recon)
    p = oracle.params(dims, kappa=kappa, csw=csw, mu=mu, t_bc=-1.0, charge=charge)
    return lat, U, A, p


CASES = [
    # (precision, recon, mu, charge)
    ("double", 18, 0.0, 0.0),
    ("double", 12, 0.1, 0.0),
    ("double", 18, 0.1, 2.0 / 3.0),
    ("single", 18, 0.0, -1.0 / 3.0),
    ("single", 12, 0.1, 0.0),
    ("half", 12, 0.0, 0.0),
    ("half", 18, 0.1, 2.0 / 3.0),
    ("single", 8, 0.1, 0.0),
    ("half", 8, 0.0, 0.0),
]


@pytest.mark.parametrize("prec,recon,mu,charge", CASES)
@pytest.mark.parametrize("dims", [(6, 4, 6, 10), (8, 8, 8, 8)])
def test_dhop_parity(bq, dims, prec, recon, mu, charge):
    lat, U, A, p = make(bq, dims, mu=mu, charge=charge, recon=recon, precision=prec)
    psi = synth.gaussian_spinor(lat.Vh, 3)
    src = lat.pack(psi, prec)
    out = lat.spinor(prec)
    for par in (0, 1):
        for dag in (False, True):
            bq.bq_apply_dhop(lat.ctx, out, src, par, dag, prec)
            got = lat.unpack(out, prec)
            ref = oracle.dhop(p, U, A, psi, par, dag)
            assert rel(got, ref) < TOL[prec], (par, dag)
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_clover_parity(bq, prec):
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims)
    psi = synth.gaussian_spinor(lat.Vh, 4)
    src = lat.pack(psi, prec)
    out = lat.spinor(prec)
    for par in (0, 1):
        Am = oracle.clover_field(p, U, par)
        for inv in (False, True):
            bq.bq_apply_clover(lat.ctx, out, src, par, inv, prec)
            ref = oracle.clover_apply(oracle.clover_invert(Am) if inv else Am, psi)
            assert rel(lat.unpack(out, prec), ref) < TOL[prec], (par, inv)
    lat.close()


@pytest.mark.parametrize("dims", [(6, 6, 6, 6), (6, 6, 6, 10)])
def test_clover_build_ragged_tail(bq, dims):
    """The clover build covers 32 sites per block (one warp per mu-nu plane);
    V = 1296 and 2160 leave a partly filled last block."""
    lat, U, A, p = make(bq, dims)
    assert lat.Vh * 2 % 32 != 0
    psi = synth.gaussian_spinor(lat.Vh, 6)
    src = lat.pack(psi, "double")
    out = lat.spinor("double")
    for par in (0, 1):
        Am = oracle.clover_field(p, U, par)
        for inv in (False, True):
            bq.bq_apply_clover(lat.ctx, out, src, par, inv, "double")
            ref = oracle.clover_apply(oracle.clover_invert(Am) if inv else Am, psi)
            assert rel(lat.unpack(out, "double"), ref) < TOL["double"], (par, inv)
    lat.close()


@pytest.mark.parametrize("prec,recon,mu,charge", CASES)
def test_mhat_parity(bq, prec, recon, mu, charge):
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, mu=mu, charge=charge, recon=recon, precision=prec)
    op = oracle.Operator(p, U, A)
    psi = synth.gaussian_spinor(lat.Vh, 5)
    src = lat.pack(psi, prec)
    out = lat.spinor(prec)
    for dag in (False, True):
        bq.bq_apply_mhat(lat.ctx, out, src, dag, prec)
        assert rel(lat.unpack(out, prec), op.mhat(psi, dag)) < TOL[prec], dag
    bq.bq_apply_mdagm(lat.ctx, out, src, prec)
    assert rel(lat.unpack(out, prec), op.mdagm(psi)) < TOL[prec]
    lat.close()


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6), (4, 2, 6, 2)])
def test_tiny_and_degenerate_extents(bq, dims):
    """Extent-2 directions: the forward and backward neighbour coincide."""
    lat, U, A, p = make(bq, dims, mu=0.1, charge=2.0 / 3.0, eps=0.5)
    op = oracle.Operator(p, U, A)
    psi = synth.gaussian_spinor(lat.Vh, 6)
    out = lat.spinor("double")
    bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi), 0, "double")
    assert rel(lat.unpack(out), op.mhat(psi)) < 1e-13
    lat.close()


def test_zero_and_point_sources(bq):
    dims = (4, 4, 4, 4)
    lat, U, A, p = make(bq, dims, precision="half", recon=12)
    op = oracle.Operator(p, U, A)
    for prec in ("double", "single", "half"):
        out = lat.spinor(prec)
        z = np.zeros((lat.Vh, 4, 3), np.complex128)
        bq.bq_apply_mhat(lat.ctx, out, lat.pack(z, prec), 0, prec)
        assert np.all(lat.unpack(out, prec) == 0)
        b = synth.point_source(lat.Vh, 0, 2, 1)
        bq.bq_apply_mhat(lat.ctx, out, lat.pack(b, prec), 0, prec)
        assert rel(lat.unpack(out, prec), op.mhat(b)) < TOL[prec]
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_cg_config1(bq, prec):
    """8^4, eps 0.3, kappa 0.125, c_SW 1.0, antiperiodic t: true FP64 residual <= 1e-10."""
    dims = (8, 8, 8, 8)
    lat, U, A, p = make(bq, dims, kappa=0.125, csw=1.0, eps=0.3, seed=1, recon=12 if prec != "double" else 18,
                        precision=prec)
    op = oracle.Operator(p, U)
    b = synth.gaussian_spinor(lat.Vh, 1001)
    x = np.empty_like(b)
    st = bq.bq_solve_cg(lat.ctx, x, b, tol=1e-10, precision=prec, delta=1e-3 if prec == "single" else 1e-1)
    assert st["converged"] == 1
    res = np.linalg.norm(op.mdagm(x) - b) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert abs(st["true_residual"] - res) < 1e-11
    xo, _ = op.cg(b, tol=1e-12)
    assert rel(x, xo) < 1e-8
    lat.close()


def test_cg_shift_and_device_buffers(bq):
    import torch

    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.13, csw=1.7, mu=0.0)
    op = oracle.Operator(p, U)
    b = synth.gaussian_spinor(lat.Vh, 77)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    # FP32 and FP16-storage inner iterations (the shifted <p, Ap> sums |p|^2 inside the fused launch)
    for prec, delta in (("single", 1e-3), ("half", 1e-1)):
        bq.bq_set_recon(lat.ctx, prec, 12)
        st = bq.bq_solve_cg(lat.ctx, xd, bd, tol=1e-10, precision=prec, shift=0.05, delta=delta)
        x = xd.cpu().numpy()
        res = np.linalg.norm(op.mdagm(x, 0.05) - b) / np.linalg.norm(b)
        assert res <= 1e-10 and st["converged"], (prec, res)
    lat.close()


def test_error_codes(bq):
    with pytest.raises(bq.BqError) as e:
        bq.bq_create((4, 4, 5, 4))
    assert e.value.status == bq.BQ_ERR_ARG
    lat = bq.Lattice((4, 4, 4, 4), 0.12)
    out, inp = lat.spinor(), lat.spinor()
    with pytest.raises(bq.BqError) as e:
        bq.bq_apply_mhat(lat.ctx, out, inp, 0, "double")
    assert e.value.status == bq.BQ_ERR_STATE
    bq.bq_set_gauge(lat.ctx, synth.gauge_field((4, 4, 4, 4), 0.2, 3))
    bq.bq_set_u1(lat.ctx, synth.u1_field((4, 4, 4, 4), 0.1, 4))
    for recon in (12, 8):
        with pytest.raises(bq.BqError) as e:
            bq.bq_set_recon(lat.ctx, "single", recon)
        assert e.value.status == bq.BQ_ERR_ARG
    with pytest.raises(bq.BqError) as e:
        bq.bq_apply_mhat(lat.ctx, out, out, 0, "double")
    assert e.value.status == bq.BQ_ERR_ARG
    b = synth.gaussian_spinor(lat.Vh, 1)
    x = np.empty_like(b)
    with pytest.raises(bq.BqError) as e:
        bq.bq_solve_cg(lat.ctx, x, b, tol=1e-10, max_iter=2)
    assert e.value.status == bq.BQ_ERR_NOT_CONVERGED
    lat.close()


def test_recon8_refusals(bq):
    """8-real links: no FP64 storage, and a field with |U00| = 1 (the unit gauge,
    where the storage is singular) is refused at link packing, not applied."""
    lat = bq.Lattice((4, 4, 4, 4), 0.12, 1.0)
    with pytest.raises(bq.BqError) as e:
        bq.bq_set_recon(lat.ctx, "double", 8)
    assert e.value.status == bq.BQ_ERR_ARG
    bq.bq_set_gauge(lat.ctx, synth.unit_gauge((4, 4, 4, 4)))
    bq.bq_set_recon(lat.ctx, "single", 8)
    src = lat.pack(synth.gaussian_spinor(lat.Vh, 2), "single")
    out = lat.spinor("single")
    with pytest.raises(bq.BqError) as e:
        bq.bq_apply_mhat(lat.ctx, out, src, 0, "single")
    assert e.value.status == bq.BQ_ERR_ARG and "8-real" in str(e.value)
    # the same context with a generic SU(3) field then works
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 5)
    bq.bq_set_gauge(lat.ctx, U)
    bq.bq_apply_mhat(lat.ctx, out, src, 0, "single")
    op = oracle.Operator(oracle.params(dims, kappa=0.12, csw=1.0, t_bc=-1.0), U)
    psi = lat.unpack(src, "single")
    assert rel(lat.unpack(out, "single"), op.mhat(psi)) < TOL["single"]
    lat.close()


@pytest.mark.parametrize("cfg", ["16^3x32 mu=0.1", "32^3x64"])
def test_full_size_sampled(bq, cfg):
    """Full-size lattices: the GPU applies Mhat on every site, the oracle
    recomputes 48 sampled even sites one by one."""
    if cfg.startswith("16"):
        dims, eps, kappa, csw, mu = (16, 16, 16, 32), 0.2, 0.1350, 1.7, 0.1
    else:
        dims, eps, kappa, csw, mu = (32, 32, 32, 64), 0.15, 0.1355, 1.9, 0.0
    U = synth.gauge_field(dims, eps, 1)
    lat = bq.Lattice(dims, kappa, csw, mu, -1.0)
    bq.bq_set_gauge(lat.ctx, U)
    bq.bq_set_recon(lat.ctx, "single", 12)
    bq.bq_set_recon(lat.ctx, "half", 12)
    p = oracle.params(dims, kappa=kappa, csw=csw, mu=mu, t_bc=-1.0)
    psi = synth.gaussian_spinor(lat.Vh, 9)
    rng = np.random.default_rng(0)
    sites = np.unique(np.concatenate([[0, lat.Vh - 1], rng.integers(0, lat.Vh, 46)]))
    for dag in (False, True):
        ref = oracle.mhat_sites(p, U, None, psi, sites, dag)
        for prec in ("double", "single", "half"):
            out = lat.spinor(prec)
            bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi, prec), dag, prec)
            got = lat.unpack(out, prec)[sites]
            assert rel(got, ref) < TOL[prec], (prec, dag)
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_multishift_cg(bq, prec):
    """10 shifts geometric over [1e-4, 1]: every x_k reaches a true FP64 residual
    <= 1e-10 and matches the oracle's independent per-shift CG."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.1350, csw=1.7, eps=0.2, recon=12 if prec != "double" else 18,
                        precision=prec)
    op = oracle.Operator(p, U)
    b = synth.gaussian_spinor(lat.Vh, 4242)
    shifts = 10.0 ** (-4 + 4 * np.arange(10) / 9)
    xs = [np.empty_like(b) for _ in shifts]
    st = bq.bq_solve_multishift_cg(lat.ctx, xs, b, shifts, tol=1e-10, precision=prec,
                                   delta=1e-3 if prec == "single" else 1e-1)
    assert st["converged"] == 1
    for k, s in enumerate(shifts):
        res = np.linalg.norm(op.mdagm(xs[k], s) - b) / np.linalg.norm(b)
        assert res <= 1e-10, (k, res)
        assert abs(st["residuals"][k] - res) < 1e-11
        xo, _ = op.cg(b, sigma=s, tol=1e-12)
        assert rel(xs[k], xo) < 1e-8
    # the rational sum of an RHMC term
    xsum = sum(0.1 * x for x in xs)
    osum = sum(0.1 * op.cg(b, sigma=s, tol=1e-12)[0] for s in shifts)
    assert rel(xsum, osum) < 1e-8
    lat.close()


def test_multishift_krylov_phase_alone(bq):
    """FP64 multishift: the shared Krylov space alone must already meet the
    tolerance for every shift, so the refinement phase adds no iterations beyond
    its residual check (shifted recurrences are exact in exact arithmetic)."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.1350, csw=1.7, eps=0.2)
    b = synth.gaussian_spinor(lat.Vh, 4243)
    shifts = [0.0, 0.01, 0.1, 1.0]
    xs = [np.empty_like(b) for _ in shifts]
    st1 = bq.bq_solve_multishift_cg(lat.ctx, xs, b, shifts, tol=1e-9, precision="double")
    x0 = np.empty_like(b)
    st0 = bq.bq_solve_cg(lat.ctx, x0, b, tol=1e-9, precision="double", check_every=8)
    # Krylov iterations are those of the smallest shift; refinement adds few (the true residual check)
    assert st1["iterations"] <= st0["iterations"] + 8 * len(shifts)
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_spinor_dot(bq, prec):
    dims = (6, 4, 6, 10)
    lat = bq.Lattice(dims, 0.13)
    a = synth.gaussian_spinor(lat.Vh, 1)
    b = synth.gaussian_spinor(lat.Vh, 2)
    na, nb = lat.pack(a, prec), lat.pack(b, prec)
    # the oracle side of this check is numpy's vdot on what the buffers hold
    ad, bd = lat.unpack(na, prec), lat.unpack(nb, prec)
    ref = np.vdot(ad.ravel(), bd.ravel())
    got = bq.bq_spinor_dot(lat.ctx, na, nb, prec)
    assert abs(got - ref) / abs(ref) < (1e-13 if prec == "double" else 1e-6)
    assert bq.bq_spinor_dot(lat.ctx, na, nb, prec) == got  # fixed reduction order
    lat.close()


DF64_CASES = [(18, 0.0, 0.0), (12, 0.1, 0.0), (18, 0.1, 2.0 / 3.0)]


@pytest.mark.parametrize("recon,mu,charge", DF64_CASES)
def test_df64_arith_parity(bq, recon, mu, charge):
    """FP64 storage with double-float arithmetic meets the FP64 tolerance (1e-13)."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, mu=mu, charge=charge, recon=recon, precision="double")
    bq.bq_set_fp64_arith(lat.ctx, "df64")
    op = oracle.Operator(p, U, A)
    psi = synth.gaussian_spinor(lat.Vh, 15)
    src = lat.pack(psi, "double")
    out = lat.spinor("double")
    for par in (0, 1):
        for dag in (False, True):
            bq.bq_apply_dhop(lat.ctx, out, src, par, dag, "double")
            assert rel(lat.unpack(out), oracle.dhop(p, U, A, psi, par, dag)) < 1e-13, (par, dag)
    for dag in (False, True):
        bq.bq_apply_mhat(lat.ctx, out, src, dag, "double")
        assert rel(lat.unpack(out), op.mhat(psi, dag)) < 1e-13, dag
    for par in (0, 1):
        for inv in (False, True):
            bq.bq_apply_clover(lat.ctx, out, src, par, inv, "double")
            Am = oracle.clover_field(p, U, par)
            ref = oracle.clover_apply(oracle.clover_invert(Am) if inv else Am, psi)
            assert rel(lat.unpack(out), ref) < 1e-13
    # values spanning many binades, exact zeros and a point source survive the float-pair split
    wide = psi * np.exp(np.random.default_rng(3).uniform(-30, 30, psi.shape))
    wide[::7] = 0
    bq.bq_apply_mhat(lat.ctx, out, lat.pack(wide, "double"), 0, "double")
    assert rel(lat.unpack(out), op.mhat(wide)) < 1e-13
    x = np.empty_like(psi)
    st = bq.bq_solve_cg(lat.ctx, x, psi, tol=1e-10, precision="single")
    assert st["converged"] and np.linalg.norm(op.mdagm(x) - psi) / np.linalg.norm(psi) <= 1e-10
    lat.close()


def test_df64_full_size_sampled(bq):
    dims = (32, 32, 32, 64)
    U = synth.gauge_field(dims, 0.15, 1)
    lat = bq.Lattice(dims, 0.1355, 1.9, 0.0, -1.0)
    bq.bq_set_gauge(lat.ctx, U)
    bq.bq_set_fp64_arith(lat.ctx, "df64")
    p = oracle.params(dims, kappa=0.1355, csw=1.9, mu=0.0, t_bc=-1.0)
    psi = synth.gaussian_spinor(lat.Vh, 19)
    sites = np.unique(np.concatenate([[0, lat.Vh - 1], np.random.default_rng(1).integers(0, lat.Vh, 30)]))
    out = lat.spinor("double")
    bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi), 0, "double")
    assert rel(lat.unpack(out)[sites], oracle.mhat_sites(p, U, None, psi, sites)) < 1e-13
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_batched_point_sources(bq, prec):
    """12 spin-colour point sources on one lattice in one batched solve: each
    solution reaches a true FP64 residual <= 1e-10 and equals the oracle CG."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.1350, csw=1.7, eps=0.2, recon=12 if prec != "double" else 18,
                        precision=prec)
    op = oracle.Operator(p, U)
    bs = [synth.point_source(lat.Vh, 0, s, c) for s in range(4) for c in range(3)]
    xs = [np.empty_like(b) for b in bs]
    stats = bq.bq_solve_cg_batch([lat.ctx] * 12, xs, bs, tol=1e-10, precision=prec,
                                 delta=1e-3 if prec == "single" else 1e-1)
    for b, x, st in zip(bs, xs, stats):
        res = np.linalg.norm(op.mdagm(x) - b) / np.linalg.norm(b)
        assert st["converged"] and res <= 1e-10, res
        assert abs(st["true_residual"] - res) < 1e-11
        xo, _ = op.cg(b, tol=1e-12)
        assert rel(x, xo) < 1e-8
    lat.close()


def test_batched_ragged_lattices(bq):
    """A ragged batch (different lattices, parameters, chemical potential and
    shift) in one batched solve, on device buffers."""
    import torch

    cases = [((8, 8, 8, 8), 0.125, 1.0, 0.0, 0.3), ((6, 4, 6, 10), 0.1350, 1.7, 0.1, 0.2), ((4, 4, 4, 4), 0.13, 1.9, 0.0, 0.2)]
    lats, ops, bs_d, xs_d, bs = [], [], [], [], []
    for i, (dims, kappa, csw, mu, eps) in enumerate(cases):
        lat, U, A, p = make(bq, dims, kappa=kappa, csw=csw, mu=mu, eps=eps, seed=10 + i, recon=12, precision="single")
        lats.append(lat)
        ops.append(oracle.Operator(p, U))
        b = synth.gaussian_spinor(lat.Vh, 500 + i)
        bs.append(b)
        bs_d.append(torch.from_numpy(b).cuda())
        xs_d.append(torch.empty_like(bs_d[-1]))
    stats = bq.bq_solve_cg_batch([l.ctx for l in lats], xs_d, bs_d, tol=1e-10, precision="single", shift=0.01)
    for op, b, x, st in zip(ops, bs, xs_d, stats):
        x = x.cpu().numpy()
        res = np.linalg.norm(op.mdagm(x, 0.01) - b) / np.linalg.norm(b)
        assert st["converged"] and res <= 1e-10, res
    for l in lats:
        l.close()


@pytest.mark.parametrize("nsys,mapping", [(1, 0), (3, 0), (3, -5)])
def test_cuda_graph_matches_eager(bq, nsys, mapping):
    """The graph-captured iteration gives bit-identical solutions, iteration
    counts and launch/byte counters to eager launches, and its event-timed
    hopping-term kernels are measured (also with the CG-fused tile launches of
    mapping -5)."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.1350, csw=1.7, eps=0.2, recon=12, precision="single")
    bq.bq_set_batch_mapping(lat.ctx, mapping)
    bs = [synth.gaussian_spinor(lat.Vh, 60 + i) for i in range(nsys)]
    # one solve first, so that the one-time field preparation is not counted below
    bq.bq_solve_cg_batch([lat.ctx] * nsys, [np.empty_like(b) for b in bs], bs, tol=1e-6, precision="single")
    runs = {}
    for graphs in (True, False):
        bq.bq_set_cuda_graphs(lat.ctx, graphs)
        xs = [np.empty_like(b) for b in bs]
        bq.bq_reset_counters(lat.ctx, timing=True)
        st = bq.bq_solve_cg_batch([lat.ctx] * nsys, xs, bs, tol=1e-10, precision="single", check_every=4)
        runs[graphs] = (xs, st, bq.bq_get_counters(lat.ctx))
    (xg, sg, cg), (xe, se, ce) = runs[True], runs[False]
    for a, b in zip(xg, xe):
        assert np.array_equal(a, b)
    assert [s["iterations"] for s in sg] == [s["iterations"] for s in se]
    assert cg["launches"] == ce["launches"]
    assert cg["dslash_launches"] == ce["dslash_launches"]
    assert np.allclose(np.array(cg["dslash_bytes"]), np.array(ce["dslash_bytes"]), rtol=1e-12)
    assert cg["dslash_ms"][1][1] > 0
    if nsys == 1 or mapping <= -3:  # the two A x - k D steps carry the fused CG vector work
        assert cg["dslash_ms"][1][3] > 0 and cg["dslash_ms"][1][4] > 0 and cg["dslash_launches"][1][2] == 0
    elif bq.bq_get_batch_mapping(lat.ctx) > -3:
        assert cg["dslash_ms"][1][2] > 0
    lat.close()


def test_config5_qed_48x96(bq):
    """48^3x96 QCD+QED: SU(3) links exp(i 0.15 A) times U(1) phases exp(-i Q A_mu),
    sigma_A = 0.1, kappa 0.1355, c_SW 1.9, flavours Q = +2/3 and -1/3. Sampled
    parity of Mhat at every precision, then 4 Gaussian sources per flavour solved
    in one batched FP16/FP32/FP64 solve, their residual re-checked on sampled
    sites by the oracle (Mhat^dag applied to the GPU's FP64 Mhat x)."""
    import torch

    dims = (48, 48, 48, 96)
    U = synth.gauge_field(dims, 0.15, 5)
    A = synth.u1_field(dims, 0.1, 6)
    Vh = synth.volume(dims) // 2
    rng = np.random.default_rng(3)
    sites = np.unique(np.concatenate([[0, Vh - 1], rng.integers(0, Vh, 22)]))
    lats = []
    for q in (2.0 / 3.0, -1.0 / 3.0):
        lat = bq.Lattice(dims, 0.1355, 1.9, 0.0, -1.0, q)
        bq.bq_set_gauge(lat.ctx, U)
        bq.bq_set_u1(lat.ctx, A)
        lats.append(lat)
        p = oracle.params(dims, kappa=0.1355, csw=1.9, mu=0.0, t_bc=-1.0, charge=q)
        psi = synth.gaussian_spinor(Vh, 31)
        ref = oracle.mhat_sites(p, U, A, psi, sites)
        for prec in ("double", "single", "half"):
            out = lat.spinor(prec)
            bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi, prec), 0, prec)
            assert rel(lat.unpack(out, prec)[sites], ref) < TOL[prec], (q, prec)
    # one batched mixed-precision solve: 4 sources per flavour
    bs = [torch.from_numpy(synth.gaussian_spinor(Vh, 700 + i)).cuda() for i in range(8)]
    xs = [torch.empty_like(b) for b in bs]
    ctxs = [lats[0].ctx] * 4 + [lats[1].ctx] * 4
    stats = bq.bq_solve_cg_batch(ctxs, xs, bs, tol=1e-10, precision="half", delta=1e-2, check_every=2)
    assert all(s["converged"] and s["true_residual"] <= 1e-10 for s in stats)
    for i in (0, 5):
        lat, q = (lats[0], 2.0 / 3.0) if i < 4 else (lats[1], -1.0 / 3.0)
        p = oracle.params(dims, kappa=0.1355, csw=1.9, mu=0.0, t_bc=-1.0, charge=q)
        y = lat.spinor("double")
        bq.bq_apply_mhat(lat.ctx, y, lat.pack(xs[i]), 0, "double")
        r = oracle.mhat_sites(p, U, A, lat.unpack(y), sites, dagger=True) - bs[i].cpu().numpy()[sites]
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bs[i].cpu().numpy())
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("cfg", ["32^3x64", "16^3x32 mu=0.1"])
def test_apply_error_report(bq, cfg, capsys):
    """States the per-apply error of every storage/arithmetic against the FP64
    oracle (sampled sites, Mhat), and checks it against the tolerances."""
    if cfg.startswith("32"):
        dims, eps, kappa, csw, mu = (32, 32, 32, 64), 0.15, 0.1355, 1.9, 0.0
    else:
        dims, eps, kappa, csw, mu = (16, 16, 16, 32), 0.2, 0.1350, 1.7, 0.1
    U = synth.gauge_field(dims, eps, 1)
    lat = bq.Lattice(dims, kappa, csw, mu, -1.0)
    bq.bq_set_gauge(lat.ctx, U)
    p = oracle.params(dims, kappa=kappa, csw=csw, mu=mu, t_bc=-1.0)
    psi = synth.gaussian_spinor(lat.Vh, 9)
    sites = np.unique(np.random.default_rng(2).integers(0, lat.Vh, 64))
    ref = oracle.mhat_sites(p, U, None, psi, sites)
    lines = []
    for prec, recon, arith in (("double", 18, "native"), ("double", 18, "df64"), ("double", 12, "df64"),
                               ("single", 18, None), ("single", 12, None), ("single", 8, None),
                               ("half", 18, None), ("half", 12, None), ("half", 8, None)):
        bq.bq_set_recon(lat.ctx, prec, recon)
        if arith:
            bq.bq_set_fp64_arith(lat.ctx, arith)
        out = lat.spinor(prec)
        bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi, prec), 0, prec)
        err = rel(lat.unpack(out, prec)[sites], ref)
        lines.append(f"APPLY-ERROR {cfg} {prec} r{recon} {arith or ''} {err:.3e}")
        assert err < TOL[prec]
    lat.close()
    with capsys.disabled():
        print("\n" + "\n".join(lines))


FULL_CASES = [
    # (method, precision, mu, charge, delta)
    ("bicgstab", "double", 0.1, 0.0, 1e-3),
    ("bicgstab", "single", 0.1, 2.0 / 3.0, 1e-3),
    ("bicgstab", "half", 0.0, 0.0, 1e-1),
    ("cg", "single", 0.1, 0.0, 1e-3),
    ("cg", "double", 0.0, -1.0 / 3.0, 1e-3),
]


@pytest.mark.parametrize("method,prec,mu,charge,delta", FULL_CASES)
def test_full_system_solve(bq, method, prec, mu, charge, delta):
    """M x = b on the whole lattice through the even-odd reduction: the FP64
    residual |b - M x| / |b| from the oracle's M meets tol and x matches the
    oracle's block-eliminated solution."""
    dims = (6, 4, 6, 10)
    recon = 12 if prec != "double" and not charge else 18
    lat, U, A, p = make(bq, dims, kappa=0.13, csw=1.7, mu=mu, charge=charge, recon=recon, precision=prec)
    op = oracle.Operator(p, U, A)
    b_e, b_o = synth.gaussian_spinor(lat.Vh, 501), synth.gaussian_spinor(lat.Vh, 502)
    x_e, x_o = np.empty_like(b_e), np.empty_like(b_o)
    st = bq.bq_solve_full(lat.ctx, x_e, x_o, b_e, b_o, method=method, tol=1e-10, precision=prec, delta=delta)
    y_e, y_o = op.full(x_e, x_o)
    bn = np.sqrt(np.linalg.norm(b_e) ** 2 + np.linalg.norm(b_o) ** 2)
    res = np.sqrt(np.linalg.norm(y_e - b_e) ** 2 + np.linalg.norm(y_o - b_o) ** 2) / bn
    assert st["converged"] == 1 and res <= 1e-10, (st, res)
    assert abs(st["true_residual"] - res) < 1e-11
    xo_e, xo_o = op.solve_full(b_e, b_o, tol=1e-12)
    assert rel(np.concatenate([x_e.ravel(), x_o.ravel()]), np.concatenate([xo_e.ravel(), xo_o.ravel()])) < 1e-8
    lat.close()


def test_full_system_device_buffers_and_zero_source(bq):
    import torch

    dims = (4, 4, 4, 6)
    lat, U, A, p = make(bq, dims, kappa=0.12, csw=1.0, mu=0.05)
    op = oracle.Operator(p, U)
    b_e, b_o = synth.gaussian_spinor(lat.Vh, 511), np.zeros((lat.Vh, 4, 3), np.complex128)
    dev = [torch.from_numpy(v).cuda() for v in (b_e, b_o)]
    xs = [torch.full_like(dev[0], 7.0), torch.full_like(dev[1], 7.0)]
    st = bq.bq_solve_full(lat.ctx, xs[0], xs[1], dev[0], dev[1], method="bicgstab", tol=1e-11)
    x_e, x_o = xs[0].cpu().numpy(), xs[1].cpu().numpy()
    y_e, y_o = op.full(x_e, x_o)
    res = np.sqrt(np.linalg.norm(y_e - b_e) ** 2 + np.linalg.norm(y_o) ** 2) / np.linalg.norm(b_e)
    assert st["converged"] and res <= 1e-11
    # b = 0 gives x = 0 without iterating
    z = np.zeros_like(b_e)
    x_e, x_o = np.ones_like(b_e), np.ones_like(b_e)
    st = bq.bq_solve_full(lat.ctx, x_e, x_o, z, z, method="cg")
    assert st["converged"] and st["iterations"] == 0 and not x_e.any() and not x_o.any()
    with pytest.raises(bq.BqError) as e:
        bq.bq_solve_full(lat.ctx, x_e, x_o, b_e, b_o, method="bicgstab", tol=1e-10, max_iter=2)
    assert e.value.status == bq.BQ_ERR_NOT_CONVERGED
    lat.close()


@pytest.mark.parametrize("rho,n_iter", [(0.1, 1), (0.125, 3)])
def test_stout_links_parity(bq, rho, n_iter):
    """Stout-smeared links of the hopping term against the oracle, element by element."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, eps=0.3)
    bq.bq_set_stout(lat.ctx, rho, n_iter)
    got = bq.bq_get_hop_links(lat.ctx, np.empty_like(U))
    expect = oracle.stout(dims, U, rho, n_iter)
    assert np.abs(got - expect).max() < 1e-13
    bq.bq_set_stout(lat.ctx, 0.0, 0)
    assert np.array_equal(bq.bq_get_hop_links(lat.ctx, np.empty_like(U)), U)
    lat.close()


@pytest.mark.parametrize("prec,recon,mu,charge", [("double", 18, 0.0, 0.0), ("double", 12, 0.1, 0.0),
                                                  ("single", 12, 0.0, 0.0), ("double", 18, 0.0, 2.0 / 3.0),
                                                  ("half", 18, 0.1, -1.0 / 3.0), ("single", 8, 0.1, 0.0),
                                                  ("half", 8, 0.0, 0.0)])
def test_stout_operator_parity(bq, prec, recon, mu, charge):
    """Mhat with stout-smeared hopping links and the clover term from the thin links."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, mu=mu, charge=charge, recon=recon, precision=prec)
    bq.bq_set_stout(lat.ctx, 0.1, 1)
    op = oracle.Operator(p, U, A, U_hop=oracle.stout(dims, U, 0.1, 1))
    psi = synth.gaussian_spinor(lat.Vh, 41)
    src, dst = lat.pack(psi, prec), lat.spinor(prec)
    for dag in (False, True):
        bq.bq_apply_mhat(lat.ctx, dst, src, dag, prec)
        assert rel(lat.unpack(dst, prec), op.mhat(psi, dag)) < TOL[prec]
    # a new gauge field is smeared again
    U2 = synth.gauge_field(dims, 0.25, 9)
    bq.bq_set_gauge(lat.ctx, U2)
    op2 = oracle.Operator(p, U2, A, U_hop=oracle.stout(dims, U2, 0.1, 1))
    bq.bq_apply_mhat(lat.ctx, dst, src, False, prec)
    assert rel(lat.unpack(dst, prec), op2.mhat(psi)) < TOL[prec]
    lat.close()


@pytest.mark.parametrize("dims,eps", [((6, 4, 6, 10), 0.3), ((8, 8, 8, 8), 0.6)])
def test_clover_logdet_parity(bq, dims, eps):
    lat, U, A, p = make(bq, dims, kappa=0.1355, csw=1.9, eps=eps)
    for par in (0, 1):
        ld, neg = bq.bq_clover_logdet(lat.ctx, par)
        ld_o, neg_o = oracle.clover_logdet(p, U, par)
        assert abs(ld - ld_o) <= 1e-12 * max(1.0, abs(ld_o)) + 1e-10, (ld, ld_o)
        assert neg == neg_o == 0
    lat.close()


def test_clover_logdet_two_planes_closed_form(bq):
    """Constant abelian fields in the planes 12 and 34 with g = g' =
    (2/3, -1/3, -1/3) and kappa c_SW = 1: per site one chirality block has
    det 1 and the other prod_a (1 - (2 kc g_a)^2) < 0 (the two blocks hold the
    sigma sign pairs (s, s') and (s, -s')), so every site contributes one
    negative block and log|det A(x)| = log|prod_a (1 - 4 kc^2 g_a^2)|."""
    from helpers import two_plane_background

    dims = (4, 4, 4, 6)
    c = (1.0, 0.0, 0.0)
    U, phi, _ = two_plane_background(dims, c, c, 1)
    kc = 1.0
    g = np.sin(phi * np.array(c))
    g -= g.mean()
    det_site = np.prod(1 - 4 * kc ** 2 * g ** 2)
    assert det_site < 0
    lat = bq.Lattice(dims, 0.25, 4.0, 0.0, -1.0, 0.0)
    bq.bq_set_gauge(lat.ctx, U)
    n = lat.Vh
    for par in (0, 1):
        ld, neg = bq.bq_clover_logdet(lat.ctx, par)
        assert abs(ld - n * np.log(abs(det_site))) < 1e-12 * n, (ld, n * np.log(abs(det_site)))
        assert neg == n
    lat.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_clover_rough_field_both_paths(bq, seed):
    """A rough field (eps 2) with kappa c_SW = 1: about a quarter of the 6x6
    blocks have an LDL^dag pivot below 0.1 of their largest entry and take the
    pivoted fallback of the inverse and of the log det, the rest the unpivoted
    fast path; most blocks have det < 0. The blocks' condition
    numbers reach 1e5, so the inverse is held to 1e-10 (1e5 x FP64 unit
    roundoff, with a factor 10 for the elimination's growth)."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.25, csw=4.0, eps=2.0, seed=seed)
    psi = synth.gaussian_spinor(lat.Vh, 7)
    src = lat.pack(psi, "double")
    out = lat.spinor("double")
    for par in (0, 1):
        Am = oracle.clover_field(p, U, par)
        bq.bq_apply_clover(lat.ctx, out, src, par, True, "double")
        assert rel(lat.unpack(out, "double"), oracle.clover_apply(oracle.clover_invert(Am), psi)) < 1e-10, par
        ld, neg = bq.bq_clover_logdet(lat.ctx, par)
        ld_o, neg_sites = oracle.clover_logdet(p, U, par)
        assert abs(ld - ld_o) <= 1e-12 * abs(ld_o), (ld, ld_o)
        # the library counts 6x6 chirality blocks with det < 0, the oracle 12x12 sites;
        # count the blocks of the oracle's clover matrices, and the sign of det A agrees
        neg_blocks = sum(int(np.sum(np.linalg.slogdet(Am[:, 6 * b:6 * b + 6, 6 * b:6 * b + 6])[0].real < 0))
                         for b in (0, 1))
        assert neg == neg_blocks and neg_blocks > 1000, (neg, neg_blocks)
        assert neg % 2 == neg_sites % 2
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single", "half"])
def test_block_multishift_cg(bq, prec):
    """Three right-hand sides (one of them zero) x four shifts: every solution
    against the oracle's CG of its own shifted system, and its FP64 residual."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.13, csw=1.7, mu=0.0, recon=12 if prec != "double" else 18,
                        precision=prec)
    op = oracle.Operator(p, U)
    bs = [synth.gaussian_spinor(lat.Vh, 800 + r) for r in range(2)] + [np.zeros((lat.Vh, 4, 3), np.complex128)]
    shifts = [0.002, 0.03, 0.3, 1.0]
    xs = [[np.empty_like(bs[0]) for _ in shifts] for _ in bs]
    st = bq.bq_solve_multishift_cg_block(lat.ctx, xs, bs, shifts, tol=1e-10, precision=prec,
                                         delta=1e-3 if prec != "half" else 1e-1)
    for r, b in enumerate(bs):
        assert st[r]["converged"] == 1
        for k, sh in enumerate(shifts):
            if not b.any():
                assert not xs[r][k].any()
                continue
            res = np.linalg.norm(op.mdagm(xs[r][k], sh) - b) / np.linalg.norm(b)
            assert res <= 1e-10 and abs(st[r]["residuals"][k] - res) < 1e-11, (r, k, res)
            xo, _ = op.cg(b, sh, tol=1e-12)
            assert rel(xs[r][k], xo) < 1e-8
    lat.close()


def test_block_multishift_matches_single_rhs(bq):
    """One right-hand side through the block solver equals the multishift solver's result
    within the solves' tolerance; device buffers."""
    import torch

    dims = (4, 4, 4, 6)
    lat, U, A, p = make(bq, dims, kappa=0.12, csw=1.0, mu=0.0)
    b = torch.from_numpy(synth.gaussian_spinor(lat.Vh, 71)).cuda()
    shifts = [0.01, 0.1, 1.0]
    xb = [[torch.empty_like(b) for _ in shifts]]
    xm = [torch.empty_like(b) for _ in shifts]
    bq.bq_solve_multishift_cg_block(lat.ctx, xb, [b], shifts, tol=1e-11, precision="single")
    bq.bq_solve_multishift_cg(lat.ctx, xm, b, shifts, tol=1e-11, precision="single")
    for k in range(len(shifts)):
        assert rel(xb[0][k].cpu().numpy(), xm[k].cpu().numpy()) < 1e-9
    lat.close()


@pytest.mark.parametrize("method,prec,mu", [("cg", "single", 0.1), ("bicgstab", "double", 0.1), ("cg", "half", 0.0)])
def test_full_system_adjoint_solve(bq, method, prec, mu):
    """M^dag x = b through the adjoint even-odd reduction, checked with the oracle's M^dag."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.12, csw=1.7, mu=mu, recon=12 if prec != "double" else 18, precision=prec)
    op = oracle.Operator(p, U)
    b_e, b_o = synth.gaussian_spinor(lat.Vh, 521), synth.gaussian_spinor(lat.Vh, 522)
    x_e, x_o = np.empty_like(b_e), np.empty_like(b_o)
    st = bq.bq_solve_full(lat.ctx, x_e, x_o, b_e, b_o, method=method, tol=1e-10, precision=prec,
                          delta=1e-1 if prec == "half" else 1e-3, dagger=True)
    y_e, y_o = op.full_dagger(x_e, x_o)
    bn = np.sqrt(np.linalg.norm(b_e) ** 2 + np.linalg.norm(b_o) ** 2)
    res = np.sqrt(np.linalg.norm(y_e - b_e) ** 2 + np.linalg.norm(y_o - b_o) ** 2) / bn
    assert st["converged"] == 1 and res <= 1e-10 and abs(st["true_residual"] - res) < 1e-11
    xo_e, xo_o = op.solve_full(b_e, b_o, tol=1e-12, dagger=True)
    assert rel(np.concatenate([x_e.ravel(), x_o.ravel()]), np.concatenate([xo_e.ravel(), xo_o.ravel()])) < 1e-8
    lat.close()


@pytest.mark.parametrize("prec,mu,charge", [("single", 0.0, 0.0), ("double", 0.1, 2.0 / 3.0)])
def test_trace_samples(bq, prec, mu, charge):
    """Per noise vector, the three trace samples against the oracle's (Z2 noise, four vectors)."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.13, csw=1.7, mu=mu, charge=charge, precision=prec)
    op = oracle.Operator(p, U, A)
    etas = [(synth.z2_noise(lat.Vh, 900 + 2 * n), synth.z2_noise(lat.Vh, 901 + 2 * n)) for n in range(4)]
    got, st = bq.bq_trace_samples(lat.ctx, [e for e, _ in etas], [o for _, o in etas], tol=1e-10, precision=prec)
    assert all(s_["converged"] for s_ in st) and max(s_["true_residual"] for s_ in st) <= 1e-10
    eta2 = 2 * lat.Vh * 12  # |eta|^2 of unit-modulus noise
    for n, (e, o) in enumerate(etas):
        ref = op.trace_samples(e, o, tol=1e-12)
        for k in range(3):
            # a solve to 1e-10 moves eta^dag x by at most cond(M) 1e-10 |eta|^2
            assert abs(got[n, k] - ref[k]) <= 1e-7 * abs(ref[k]) + 1e-8 * eta2, (n, k, got[n, k], ref[k])
    lat.close()


@pytest.mark.parametrize("mapping", [-1, -2, -3, -4, -5, 1, 2, 4, 8])
@pytest.mark.parametrize("prec", ["single", "half"])
def test_batched_rhs_mappings(bq, mapping, prec):
    """Every mapping of right-hand sides onto threads (forced, not autotuned):
    five Gaussian sources (a ragged last group for every mapping) against the oracle."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.1350, csw=1.7, eps=0.2, mu=0.1, recon=12, precision=prec)
    bq.bq_set_batch_mapping(lat.ctx, mapping)
    op = oracle.Operator(p, U)
    bs = [synth.gaussian_spinor(lat.Vh, 300 + i) for i in range(5)]
    xs = [np.empty_like(b) for b in bs]
    stats = bq.bq_solve_cg_batch([lat.ctx] * 5, xs, bs, tol=1e-10, precision=prec,
                                 delta=1e-3 if prec == "single" else 1e-1)
    for b, x, st in zip(bs, xs, stats):
        res = np.linalg.norm(op.mdagm(x) - b) / np.linalg.norm(b)
        assert st["converged"] and res <= 1e-10, res
    # block multishift with the same forced mapping
    shifts = [0.01, 0.5]
    xm = [[np.empty_like(bs[0]) for _ in shifts] for _ in bs[:3]]
    bq.bq_solve_multishift_cg_block(lat.ctx, xm, bs[:3], shifts, tol=1e-10, precision=prec,
                                    delta=1e-3 if prec == "single" else 1e-1)
    for r in range(3):
        for k, sh in enumerate(shifts):
            assert np.linalg.norm(op.mdagm(xm[r][k], sh) - bs[r]) / np.linalg.norm(bs[r]) <= 1e-10
    with pytest.raises(bq.BqError):
        bq.bq_set_batch_mapping(lat.ctx, 3 * 4)
    lat.close()


@pytest.mark.parametrize("prec", ["single", "half"])
@pytest.mark.parametrize("mapping", [-3, -5, -1])
def test_batched_cg_shift_fused_tiles(bq, mapping, prec):
    """Batched CG with a shift (FP32 and FP16-storage inner iteration): in the
    tile mappings the x / r update and <p, Ap> = |Mhat p|^2 + shift |p|^2 ride on
    the tile launches (the block-interleaved mapping runs the separate kernels);
    every system against the oracle."""
    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.1350, csw=1.7, eps=0.2, mu=0.1, recon=12, precision=prec)
    bq.bq_set_batch_mapping(lat.ctx, mapping)
    op = oracle.Operator(p, U)
    bs = [synth.gaussian_spinor(lat.Vh, 340 + i) for i in range(3)]
    xs = [np.empty_like(b) for b in bs]
    bq.bq_reset_counters(lat.ctx)
    stats = bq.bq_solve_cg_batch([lat.ctx] * 3, xs, bs, tol=1e-10, precision=prec, shift=0.05,
                                 delta=1e-3 if prec == "single" else 1e-1)
    c = bq.bq_get_counters(lat.ctx)
    pi = 1 if prec == "single" else 2
    fused = c["dslash_launches"][pi][3] > 0 and c["dslash_launches"][pi][4] > 0
    assert fused == (mapping <= -3) and (c["dslash_launches"][pi][2] == 0) == fused
    for b, x, st in zip(bs, xs, stats):
        res = np.linalg.norm(op.mdagm(x, 0.05) - b) / np.linalg.norm(b)
        assert st["converged"] and res <= 1e-10, res
    lat.close()


def test_next_rows_error_codes(bq):
    """Argument and state errors of the full-system, block multishift, stout,
    log det and trace entry points come back as status codes."""
    import ctypes

    lat = bq.Lattice((4, 4, 4, 4), 0.12, 1.0)
    z = np.zeros((lat.Vh, 4, 3), np.complex128)
    x_e, x_o = np.empty_like(z), np.empty_like(z)
    lib = bq._lib_handle()
    for call in (lambda: bq.bq_solve_full(lat.ctx, x_e, x_o, z, z),
                 lambda: bq.bq_clover_logdet(lat.ctx, 0),
                 lambda: bq.bq_get_hop_links(lat.ctx, np.empty((2 * lat.Vh, 4, 3, 3), np.complex128)),
                 lambda: bq.bq_trace_samples(lat.ctx, [z], [z])):
        with pytest.raises(bq.BqError) as e:
            call()
        assert e.value.status == bq.BQ_ERR_STATE
    bq.bq_set_gauge(lat.ctx, synth.gauge_field((4, 4, 4, 4), 0.2, 3))
    for bad in ((-0.1, 1), (1.5, 1), (0.1, -1), (0.1, 65)):
        with pytest.raises(bq.BqError) as e:
            bq.bq_set_stout(lat.ctx, *bad)
        assert e.value.status == bq.BQ_ERR_ARG
    with pytest.raises(bq.BqError) as e:
        bq.bq_clover_logdet(lat.ctx, 2)
    assert e.value.status == bq.BQ_ERR_ARG
    sp = bq.bq_solver_params(1e-10, 100, 0, 1e-3, 8, 0.0)
    st = bq.bq_solver_stats()
    p = z.ctypes.data
    assert lib.bq_solve_full(lat.ctx, p, p, p, p, 0, 7, 0, ctypes.byref(sp), ctypes.byref(st)) == bq.BQ_ERR_ARG
    assert lib.bq_solve_full(lat.ctx, p, p, p, p, 0, 0, 2, ctypes.byref(sp), ctypes.byref(st)) == bq.BQ_ERR_ARG
    assert lib.bq_solve_full(lat.ctx, None, p, p, p, 0, 0, 0, ctypes.byref(sp), ctypes.byref(st)) == bq.BQ_ERR_ARG
    sp_shift = bq.bq_solver_params(1e-10, 100, 0, 1e-3, 8, 0.5)
    assert lib.bq_solve_full(lat.ctx, p, p, p, p, 0, 0, 0, ctypes.byref(sp_shift), ctypes.byref(st)) == bq.BQ_ERR_ARG
    arr = (ctypes.c_void_p * 1)(p)
    out = (ctypes.c_double * 5)()
    assert lib.bq_trace_samples(lat.ctx, 0, arr, arr, 0, ctypes.byref(sp), out, None) == bq.BQ_ERR_ARG
    sh = (ctypes.c_double * 33)(*([0.1] * 33))
    xs = (ctypes.c_void_p * 33)(*([p] * 33))
    assert lib.bq_solve_multishift_cg_block(lat.ctx, 1, xs, arr, 0, 33, sh, ctypes.byref(sp), None,
                                            None) == bq.BQ_ERR_ARG
    sh[0] = -1.0
    assert lib.bq_solve_multishift_cg_block(lat.ctx, 1, xs, arr, 0, 2, sh, ctypes.byref(sp), None,
                                            None) == bq.BQ_ERR_ARG
    assert lib.bq_solve_multishift_cg_block(lat.ctx, 0, xs, arr, 0, 2, sh, ctypes.byref(sp), None,
                                            None) == bq.BQ_ERR_ARG
    assert b"bq_solve_multishift_cg_block" in lib.bq_last_error()
    lat.close()


def test_failure_detection_singular_clover_and_nan_source(bq):
    """Faults made on the host, reported as status codes, the context usable after:
    a clover block made singular on purpose (constant abelian field with
    kappa c_SW f_a = 1, so det A = prod (1 - (kappa c_SW f_a)^2)^2 = 0) and a NaN in
    the source of a solve."""
    from helpers import abelian_background

    dims = (4, 6, 4, 8)
    c = (1.0, 2.0, 0.0)
    U, phi = abelian_background(dims, 0, 1, 1, c, "mu")
    f = np.sin(phi * np.array(c))
    f -= f.mean()
    kappa = 0.13
    csw = 1.0 / (kappa * np.abs(f).max())
    lat = bq.Lattice(dims, kappa, csw, 0.0, -1.0)
    bq.bq_set_gauge(lat.ctx, U)
    psi = synth.gaussian_spinor(lat.Vh, 3)
    out = lat.spinor("double")
    with pytest.raises(bq.BqError) as e:
        bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi), 0, "double")
    assert e.value.status == bq.BQ_ERR_CLOVER_SINGULAR
    lat.close()
    # NaN source: the solve stops with BQ_ERR_NOT_CONVERGED; the next solve works
    lat, U, A, p = make(bq, (4, 4, 4, 6), kappa=0.12, csw=1.0)
    b = synth.gaussian_spinor(lat.Vh, 4)
    bad = b.copy()
    bad[3, 1, 2] = np.nan
    x = np.empty_like(b)
    with pytest.raises(bq.BqError) as e:
        bq.bq_solve_cg(lat.ctx, x, bad, tol=1e-10, precision="single")
    assert e.value.status == bq.BQ_ERR_NOT_CONVERGED
    st = bq.bq_solve_cg(lat.ctx, x, b, tol=1e-10, precision="single")
    op = oracle.Operator(p, U)
    assert st["converged"] and np.linalg.norm(op.mdagm(x) - b) / np.linalg.norm(b) <= 1e-10
    lat.close()


@pytest.mark.parametrize("prec", ["double", "single"])
def test_cg_initial_guess(bq, prec):
    """CG from a given x: from the solution itself it stops at once; from a
    perturbed solution it needs fewer iterations than from zero and reaches the
    same true residual (host and device buffers, single and batched)."""
    import torch

    dims = (6, 4, 6, 10)
    lat, U, A, p = make(bq, dims, kappa=0.13, csw=1.7, mu=0.1, recon=12 if prec == "single" else 18, precision=prec)
    op = oracle.Operator(p, U)
    b = synth.gaussian_spinor(lat.Vh, 91)
    x = np.empty_like(b)
    st0 = bq.bq_solve_cg(lat.ctx, x, b, tol=1e-10, precision=prec)
    st1 = bq.bq_solve_cg(lat.ctx, x, b, tol=1e-10, precision=prec, initial_guess=True)
    assert st1["converged"] and st1["iterations"] == 0
    xg = x + 1e-4 * synth.gaussian_spinor(lat.Vh, 92)
    st2 = bq.bq_solve_cg(lat.ctx, xg, b, tol=1e-10, precision=prec, initial_guess=True)
    res = np.linalg.norm(op.mdagm(xg) - b) / np.linalg.norm(b)
    assert st2["converged"] and res <= 1e-10 and st2["iterations"] < st0["iterations"]
    # batched, device buffers: one system from a guess, one from zero
    bs = [torch.from_numpy(b).cuda(), torch.from_numpy(synth.gaussian_spinor(lat.Vh, 93)).cuda()]
    xs = [torch.from_numpy(x + 1e-4 * synth.gaussian_spinor(lat.Vh, 94)).cuda(), torch.zeros_like(bs[1])]
    sts = bq.bq_solve_cg_batch([lat.ctx] * 2, xs, bs, tol=1e-10, precision=prec, initial_guess=True)
    for xd, bd, s_ in zip(xs, bs, sts):
        bh = bd.cpu().numpy()
        assert s_["converged"] and np.linalg.norm(op.mdagm(xd.cpu().numpy()) - bh) / np.linalg.norm(bh) <= 1e-10
    assert sts[0]["iterations"] < sts[1]["iterations"]
    lat.close()


def test_parameter_and_field_updates(bq):
    """The derived fields follow every change: kappa, c_SW, mu, the time boundary,
    the charge with a U(1) field, and a new gauge field, at FP64, FP32 and FP16,
    each apply checked against the oracle built from the new state."""
    dims = (6, 4, 6, 10)
    U1, U2 = synth.gauge_field(dims, 0.2, 1), synth.gauge_field(dims, 0.25, 2)
    A = synth.u1_field(dims, 0.1, 3)
    psi = synth.gaussian_spinor(dims[0] * dims[1] * dims[2] * dims[3] // 2, 5)
    lat = bq.Lattice(dims, 0.12, 1.0, 0.0, -1.0)
    bq.bq_set_gauge(lat.ctx, U1)
    states = [
        (dict(kappa=0.12, csw=1.0, mu=0.0, t_bc=-1.0, charge=0.0), U1, None),
        (dict(kappa=0.135, csw=1.9, mu=0.0, t_bc=-1.0, charge=0.0), U1, None),
        (dict(kappa=0.135, csw=1.9, mu=0.15, t_bc=+1.0, charge=0.0), U1, None),
        (dict(kappa=0.13, csw=1.7, mu=0.05, t_bc=-1.0, charge=2.0 / 3.0), U1, A),
        (dict(kappa=0.13, csw=1.7, mu=0.05, t_bc=-1.0, charge=-1.0 / 3.0), U2, A),
        (dict(kappa=0.13, csw=1.7, mu=0.05, t_bc=-1.0, charge=0.0), U2, None),
    ]
    for prm, U, A_ in states:
        bq.bq_set_params(lat.ctx, **prm)
        if U is U2:
            bq.bq_set_gauge(lat.ctx, U2)
        bq.bq_set_u1(lat.ctx, A_)
        p = oracle.params(dims, **prm)
        op = oracle.Operator(p, U, A_)
        ref = op.mhat(psi)
        for prec in ("double", "single", "half"):
            out = lat.spinor(prec)
            bq.bq_apply_mhat(lat.ctx, out, lat.pack(psi, prec), 0, prec)
            assert rel(lat.unpack(out, prec), ref) < TOL[prec], (prm, prec)
    lat.close()
