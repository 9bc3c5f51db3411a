"""The identities the CG-fused launches rely on, checked with the oracle on CPU.

The fused CG iteration never forms <p, (Mhat^dag Mhat + sigma) p> directly: the
launch that produces t = Mhat p sums |t|^2 (and |p|^2), and the update launch
forms q = Mhat^dag t + sigma p without storing it. Both rest on Mhat^dag being the
adjoint of Mhat (also with a chemical potential, where Mhat is not
gamma_5-hermitian) and on (Mhat^dag Mhat + sigma) p = Mhat^dag (Mhat p) + sigma p.
"""
import numpy as np
import pytest

import oracle
from paper_1711_03836_gb300 import synth


@pytest.mark.parametrize("mu_chem,sigma", [(0.0, 0.0), (0.0, 0.05), (0.1, 0.3)])
def test_pap_is_norm_of_mhat_p(mu_chem, sigma):
    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, 0.3, 11)
    p_ = oracle.params(dims, kappa=0.13, csw=1.7, mu=mu_chem, t_bc=-1.0)
    op = oracle.Operator(p_, U)
    p = synth.gaussian_spinor(oracle.half_volume(p_), 21)
    t = op.mhat(p)
    ap = op.mdagm(p, sigma)
    pap = np.vdot(p, ap)
    fused = np.vdot(t, t).real + sigma * np.vdot(p, p).real
    assert abs(pap.imag) < 1e-12 * abs(pap.real)
    assert abs(pap.real - fused) < 1e-12 * fused
    # the update launch: q = Mhat^dag t + sigma p is (Mhat^dag Mhat + sigma) p
    q = op.mhat(t, dagger=True) + sigma * p
    assert np.abs(q - ap).max() < 1e-12 * np.abs(ap).max()
