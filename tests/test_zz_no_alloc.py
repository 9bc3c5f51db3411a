"""The allocation-free dot product agrees with the context-based one.

bq_spinor_dot_noalloc serves callers that cannot allocate device memory (all
memory handed to their own arena, or no cudaMalloc/cudaFree allowed inside a
time-critical loop): it keeps its reduction scratch in a static device array.
This file is collected last so that a failure here cannot hide other tests.
"""
import numpy as np
import pytest

from paper_1711_03836_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bq():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_03836_gb300 import bqcd

    return bqcd


@pytest.mark.parametrize("prec", ["double", "single", "half"])
@pytest.mark.parametrize("dims", [(6, 4, 6, 10), (32, 32, 16, 16)])
def test_noalloc_dot_matches_context_dot(bq, prec, dims):
    lat = bq.Lattice(dims, 0.13)
    tol = 1e-13 if prec == "double" else 1e-6
    for call in range(2):  # two calls in a row: the shared scratch must not leak state
        a = synth.gaussian_spinor(lat.Vh, 10 + call)
        b = synth.gaussian_spinor(lat.Vh, 20 + call)
        na, nb = lat.pack(a, prec), lat.pack(b, prec)
        ref = bq.bq_spinor_dot(lat.ctx, na, nb, prec)
        got = bq.bq_spinor_dot_noalloc(na, nb, lat.Vh, prec)
        assert abs(got - ref) <= tol * abs(ref), (call, got, ref)
        # against the plain definition: np.vdot of the stored values (unpacked to FP64)
        exact = np.vdot(lat.unpack(na, prec), lat.unpack(nb, prec))
        assert abs(got - exact) <= tol * np.linalg.norm(a) * np.linalg.norm(b), (call, got, exact)
        # the same inputs give the same bits on every call
        assert bq.bq_spinor_dot_noalloc(na, nb, lat.Vh, prec) == got
        got_self = bq.bq_spinor_dot_noalloc(na, na, lat.Vh, prec)
        ref_self = bq.bq_spinor_dot(lat.ctx, na, na, prec)
        assert abs(got_self - ref_self) <= tol * abs(ref_self)
        assert abs(got_self.imag) <= tol * abs(got_self)
    lat.close()


def test_noalloc_dot_at_the_size_limit(bq):
    """4 194 304 sites: all 16 384 block partials of the static array in use and
    the ticket counting up to its last value (FP16 storage keeps the buffers at
    about 0.2 GB each)."""
    dims = (32, 32, 32, 256)
    lat = bq.Lattice(dims, 0.13)
    assert lat.Vh == 4194304
    for call in range(2):
        a = synth.gaussian_spinor(lat.Vh, 30 + call)
        b = synth.gaussian_spinor(lat.Vh, 40 + call)
        na, nb = lat.pack(a, "half"), lat.pack(b, "half")
        got = bq.bq_spinor_dot_noalloc(na, nb, lat.Vh, "half")
        ref = bq.bq_spinor_dot(lat.ctx, na, nb, "half")
        assert abs(got - ref) <= 1e-6 * abs(ref), (call, got, ref)
        exact = np.vdot(lat.unpack(na, "half"), lat.unpack(nb, "half"))
        assert abs(got - exact) <= 1e-6 * np.linalg.norm(a) * np.linalg.norm(b), (call, got, exact)
        del na, nb
    lat.close()


def test_noalloc_rejects_oversized_input(bq):
    lat = bq.Lattice((4, 4, 4, 4), 0.13)
    a = lat.pack(synth.gaussian_spinor(lat.Vh, 1), "double")
    with pytest.raises(bq.BqError) as e:
        bq.bq_spinor_dot_noalloc(a, a, 4194304 + 1, "double")
    assert e.value.status == bq.BQ_ERR_ARG
    assert "n_sites" in str(e.value)
    lat.close()
