"""Batched Mhat^dag Mhat (bq_apply_mdagm_batch) against the FP64 oracle, per
system and per apply, for every mapping of right-hand sides onto threads.

Two lattices in one call (a ragged batch): 13 right-hand sides on a 6x4x6x10
lattice (V/2 = 720: 22.5 tiles of 32 sites, so the last tile is partly empty;
13 right-hand sides fill one shared-memory tile unit, or units of 8 + 5) and 3
on a 4^3x8 lattice, with chemical potential, and with U(1) phases on 18-real
links.
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


def lattice(bq, dims, prec, recon, mu, charge, seed):
    U = synth.gauge_field(dims, 0.2, seed)
    A = synth.u1_field(dims, 0.1, seed + 5) if charge else None
    lat = bq.Lattice(dims, 0.1350, 1.7, mu, -1.0, charge)
    bq.bq_set_gauge(lat.ctx, U)
    if A is not None:
        bq.bq_set_u1(lat.ctx, A)
    bq.bq_set_recon(lat.ctx, prec, recon)
    op = oracle.Operator(oracle.params(dims, kappa=0.1350, csw=1.7, mu=mu, t_bc=-1.0, charge=charge), U, A)
    return lat, op


@pytest.mark.parametrize("mapping", [0, -1, -2, -3, -4, -5, 1, 2, 4, 8])
@pytest.mark.parametrize("prec,recon,mu,charge", [("single", 12, 0.1, 0.0), ("half", 12, 0.0, 0.0),
                                                  ("single", 18, 0.0, 2.0 / 3.0), ("half", 18, 0.1, -1.0 / 3.0),
                                                  ("single", 8, 0.1, 0.0), ("half", 8, 0.0, 0.0),
                                                  ("double", 18, 0.1, 0.0)])
def test_batched_mdagm_parity(bq, mapping, prec, recon, mu, charge):
    if prec == "double" and mapping not in (0, -1, -3, -5):
        pytest.skip("FP64 systems take the block-interleaved mapping for tile requests; one warp mapping suffices")
    la, opa = lattice(bq, (6, 4, 6, 10), prec, recon, mu, charge, 1)
    lb, opb = lattice(bq, (4, 4, 4, 8), prec, recon, mu, charge, 2)
    bq.bq_set_recon(lb.ctx, prec, recon)
    bq.bq_set_batch_mapping(la.ctx, mapping)
    systems = [(la, opa)] * 13 + [(lb, opb)] * 3
    psis = [synth.gaussian_spinor(l.Vh, 40 + i) for i, (l, _) in enumerate(systems)]
    ins = [l.pack(p, prec) for (l, _), p in zip(systems, psis)]
    outs = [l.spinor(prec) for l, _ in systems]
    for rep in range(2):  # twice: the second call reuses the cached work vectors
        bq.bq_apply_mdagm_batch([l.ctx for l, _ in systems], outs, ins, prec)
        for i, ((l, op), p, o) in enumerate(zip(systems, psis, outs)):
            err = rel(l.unpack(o, prec), op.mdagm(p))
            assert err < TOL[prec], (rep, i, err)
    la.close()
    lb.close()


def test_batched_mdagm_matches_single_apply_and_rejects_aliasing(bq):
    """One system through the batched call equals bq_apply_mdagm; aliased buffers are refused."""
    lat, op = lattice(bq, (6, 4, 6, 10), "single", 12, 0.0, 0.0, 3)
    p = synth.gaussian_spinor(lat.Vh, 9)
    src = lat.pack(p, "single")
    o1, o2 = lat.spinor("single"), lat.spinor("single")
    bq.bq_apply_mdagm(lat.ctx, o1, src, "single")
    bq.bq_apply_mdagm_batch([lat.ctx], [o2], [src], "single")
    assert np.array_equal(lat.unpack(o1, "single"), lat.unpack(o2, "single"))
    with pytest.raises(bq.BqError) as e:
        bq.bq_apply_mdagm_batch([lat.ctx, lat.ctx], [o1, src], [src, o1], "single")
    assert e.value.status == bq.BQ_ERR_ARG
    lat.close()


@pytest.mark.parametrize("prec", ["single", "half"])
def test_tile_unit_split_at_sixteen(bq, prec):
    """17 right-hand sides of one lattice in the tile mapping: a unit of 16 and a
    unit of 1, every output against the oracle."""
    la, opa = lattice(bq, (4, 6, 4, 8), prec, 12, 0.0, 0.0, 4)
    bq.bq_set_batch_mapping(la.ctx, -3)
    psis = [synth.gaussian_spinor(la.Vh, 90 + i) for i in range(17)]
    ins = [la.pack(p, prec) for p in psis]
    outs = [la.spinor(prec) for _ in psis]
    bq.bq_apply_mdagm_batch([la.ctx] * 17, outs, ins, prec)
    assert bq.bq_get_batch_mapping(la.ctx) == -3
    for p, o in zip(psis, outs):
        assert rel(la.unpack(o, prec), opa.mdagm(p)) < TOL[prec]
    la.close()
