"""Write tests/golden/oracle_regression.json from the FP64 oracle alone.

The paper prints no worked numerical example for the operator or the solvers,
so no value here is the paper's: these are regression values of the oracle
itself on a small lattice (components of Mhat psi, D_hop psi and A psi at a few
sites, the clover log det, one CG solution's norm and three trace samples),
written once by this script and compared by tests/test_oracle_golden.py, so
that an unintended change of the oracle's arithmetic shows up even where every
mathematical pin would still pass. Regenerate only together with a change of
the oracle that a passage of the paper justifies.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import oracle  # noqa: E402
from paper_1711_03836_gb300 import synth  # noqa: E402

DIMS = (4, 4, 4, 6)
SITES = [0, 7, 40, 95]


def compute():
    U = synth.gauge_field(DIMS, 0.3, 11)
    A = synth.u1_field(DIMS, 0.1, 12)
    p = oracle.params(DIMS, kappa=0.13, csw=1.7, mu=0.1, t_bc=-1.0, charge=2.0 / 3.0)
    op = oracle.Operator(p, U, A)
    Vh = oracle.half_volume(p)
    psi = synth.gaussian_spinor(Vh, 13)
    out = {"dims": list(DIMS), "sites": SITES}

    def pack(v):
        return [[float(z.real), float(z.imag)] for z in np.ravel(v)]

    out["mhat"] = pack(op.mhat(psi)[SITES])
    out["mhat_dag"] = pack(op.mhat(psi, dagger=True)[SITES])
    out["dhop_e"] = pack(oracle.dhop(p, U, A, psi, 0)[SITES])
    out["clover_odd"] = pack(oracle.clover_apply(op.Aoo, psi)[SITES])
    out["clover_logdet"] = [oracle.clover_logdet(p, U, par)[0] for par in (0, 1)]
    x, it = op.cg(psi, tol=1e-12)
    out["cg_solution_norm"] = float(np.linalg.norm(x))
    eta_e, eta_o = synth.z2_noise(Vh, 14), synth.z2_noise(Vh, 15)
    out["trace_samples"] = pack(op.trace_samples(eta_e, eta_o, tol=1e-13))
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(compute(), f, indent=1)
    print("written")
