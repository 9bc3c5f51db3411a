"""The oracle's pins have teeth: each plausible mistake planted in a copy of the
oracle's C source (a flipped projector, swapped e^{+-mu}, a lost boundary sign,
U instead of U^dagger, a mis-oriented or mis-normalised clover leaf, a dropped
trace subtraction, a wrong Schur-complement sign, a wrong U(1) phase sign) is
caught by at least one pin of tests/test_oracle_pins.py. Mistakes are planted
in the oracle on the CPU only."""
import os
import subprocess
import tempfile

import pytest

import oracle
import oracle.oracle as oimpl
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oimpl.__file__), "bqcd_oracle.c")

MUTATIONS = {
    "forward projector sign": ("            pf = -1.0;\n            pb = +1.0;", "            pf = +1.0;\n            pb = +1.0;"),
    "e^{+mu} and e^{-mu} swapped": ("        s *= exp(p->mu);\n        if (c[3] == p->L[3] - 1)", "        s *= exp(-p->mu);\n        if (c[3] == p->L[3] - 1)"),
    "boundary sign lost": ("        if (c[3] == 0) s *= p->t_bc;", "        if (c[3] == 0) s *= 1.0;"),
    "U instead of U^dagger backward": ("        dag3(link(U, xb, mu), Ud);", "        memcpy(Ud, link(U, xb, mu), sizeof Ud);"),
    "clover leaf orientation": ("    memcpy(d, link(U, xmm, mu), sizeof d);", "    dag3(link(U, xmm, mu), d);"),
    "clover normalisation": ("(Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0", "(Q[a * 3 + b] - conj(Q[b * 3 + a])) / 4.0"),
    "trace not removed": ("            F[0] -= tr; F[4] -= tr; F[8] -= tr;", "            (void)tr;"),
    "Schur complement sign": ("    for (long i = 0; i < 24 * Vh; i++) out[i] -= k2 * t1[i];", "    for (long i = 0; i < 24 * Vh; i++) out[i] += k2 * t1[i];"),
    "U(1) phase sign": ("    if (A) s *= cexp(-I * p->charge * A[x * 4 + mu]);", "    if (A) s *= cexp(I * p->charge * A[x * 4 + mu]);"),
}

# pins that do not need scipy/dense spectra, run against each mutant
PIN_CALLS = [
    lambda: pins.test_free_field_plane_wave((4, 6, 2, 8), -1.0, 0.1),
    lambda: pins.test_free_field_plane_wave((2, 4, 4, 6), +1.0, 0.25),
    lambda: pins.test_gamma5_hermiticity(2.0 / 3.0),
    lambda: pins.test_adjoint(0.1, 2.0 / 3.0),
    lambda: pins.test_gauge_covariance(0.1, -1.0 / 3.0),
    lambda: pins.test_clover_abelian_background(0, 1, "mu"),
    lambda: pins.test_clover_abelian_background(1, 2, "nu"),
    lambda: pins.test_schur_complement_dense(),
]


def _build_mutant(old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    path = os.path.join(tmp, "mutant.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", path, "-o", lib, "-lm"], check=True)
    return lib


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    old, new = MUTATIONS[name]
    with tempfile.TemporaryDirectory() as tmp:
        mutant = oracle.load_library(_build_mutant(old, new, tmp))
        monkeypatch.setattr(oimpl, "_lib", mutant)
        caught = []
        for call in PIN_CALLS:
            try:
                call()
            except AssertionError:
                caught.append(call)
        assert caught, f"no pin catches: {name}"
