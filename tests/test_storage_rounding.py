"""Storage rounding of the half-precision formats, on the CPU with the FP64 oracle.

The spinor (scaled per site by its largest component), the links and the
clover blocks are rounded to FP16 or BF16 and the FP64 oracle's Mhat is
applied to the rounded fields; the relative error against the unrounded
apply is what storage alone costs, before any arithmetic. FP16 (11-bit
significand) stays near 3e-4; BF16 (8-bit significand) is about eight times
larger and leaves only a factor of about two to the 5e-3 half-precision
tolerance, for the same bytes and the same number of conversions per value,
which is why the library stores half precision as FP16.
"""
import numpy as np
import torch

import oracle
from paper_1711_03836_gb300 import synth


def _round(z, dt):
    def r(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dt).to(torch.float64).numpy()
    return r(z.real) + 1j * r(z.imag)


def storage_error(dt, dims=(8, 8, 8, 8)):
    U = synth.gauge_field(dims, 0.2, 1)
    p = oracle.params(dims, kappa=0.1350, csw=1.7, mu=0.1, t_bc=-1.0)
    op = oracle.Operator(p, U)
    psi = synth.gaussian_spinor(op.Aee.shape[0], 9)
    ref = op.mhat(psi)
    m = np.max(np.abs(np.stack([psi.real, psi.imag])), axis=(0, 2, 3))[:, None, None]
    opq = oracle.Operator(p, _round(U, dt))
    opq.Aee, opq.Aoo_inv = _round(op.Aee, dt), _round(op.Aoo_inv, dt)
    got = opq.mhat(_round(psi / m, dt) * m)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_fp16_and_bf16_storage_rounding():
    e16 = storage_error(torch.float16)
    ebf = storage_error(torch.bfloat16)
    assert 1e-4 < e16 < 5e-4, e16
    assert 1.5e-3 < ebf < 3.5e-3, ebf
    assert ebf > 5 * e16
