"""The pins of the oracle's numpy parts (stout smearing, full operator and its
adjoint solve, trace samples, clover log det) have teeth: each plausible
mistake planted in a copy of the oracle's Python source (a mis-oriented
staple, Omega without U^dag, a lost trace term, the exponential's sign, the
sign of the hopping term in M, a non-adjoint hop in the adjoint solve, a wrong
gamma_5, |x|^2 instead of |y|^2, a halved log det, positive determinants
counted as negative) is caught by at least one
pin of tests/test_oracle_gauge_pins.py or tests/test_oracle_pins.py. Mistakes
are planted in the oracle on the CPU only."""
import types

import pytest

import oracle
import oracle.oracle as oimpl
import test_oracle_gauge_pins as gpins
import test_oracle_pins as pins

MUTATIONS = {
    "upper staple orientation": ("C += Unu @ at(Umu, nu, 1) @ dag(at(Unu, mu, 1))",
                                 "C += Unu @ at(Umu, nu, 1) @ at(Unu, mu, 1)"),
    "Omega without U^dag": ("Om = rho * C @ dag(Umu)", "Om = rho * C @ Umu"),
    "trace term lost": ("Q = 0.5j * D - (1j / 6.0) * np.trace(D, axis1=-2, axis2=-1)[..., None, None] * np.eye(3)",
                        "Q = 0.5j * D"),
    "exponential sign": ("expQ = (Wv * np.exp(1j * q)[..., None, :]) @ dag(Wv)",
                         "expQ = (Wv * np.exp(-1j * q)[..., None, :]) @ dag(Wv)"),
    "hopping sign in M": ("y_e = clover_apply(self.Aee, x_e) - k * dhop(self.p, self.U, self.A, x_o, 0)\n",
                          "y_e = clover_apply(self.Aee, x_e) + k * dhop(self.p, self.U, self.A, x_o, 0)\n"),
    "adjoint solve hops with D": ("clover_apply(self.Aoo_inv, b_o), 0, dagger=dagger)",
                                  "clover_apply(self.Aoo_inv, b_o), 0, dagger=False)"),
    "gamma_5 pattern": ("g5 = np.array([1, 1, -1, -1], float)", "g5 = np.array([1, -1, 1, -1], float)"),
    "|x|^2 for |y|^2": ("s3 = np.vdot(y_e, y_e).real + np.vdot(y_o, y_o).real",
                        "s3 = np.vdot(x_e, x_e).real + np.vdot(x_o, x_o).real"),
    "half the log det": ("return float(np.sum(ld)), int(np.sum(sign.real < 0))",
                         "return float(np.sum(ld)) / 2, int(np.sum(sign.real < 0))"),
    "positive determinants counted": ("int(np.sum(sign.real < 0))", "int(np.sum(sign.real > 0))"),
}

PIN_CALLS = [
    lambda: gpins.test_stout_abelian_closed_form(0.1),
    lambda: gpins.test_stout_gauge_covariance_and_group(),
    lambda: gpins.test_clover_logdet_closed_form(),
    lambda: gpins.test_clover_logdet_two_planes_negative(),
    lambda: gpins.test_trace_samples_sum_to_dense_traces(0.2, 2.0 / 3.0),
    lambda: pins.test_free_field_full_operator(0.15, 0.11),
]


def _mutant_module(old, new):
    src = open(oimpl.__file__).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = oimpl.__file__
    exec(compile(src.replace(old, new), oimpl.__file__, "exec"), mod.__dict__)
    # the C part is shared unmutated: the original bound library and its parameter type
    mod.Params = oimpl.Params
    mod._lib = oimpl._load()
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    mod = _mutant_module(*MUTATIONS[name])
    for attr in ("stout", "clover_logdet", "Operator"):
        monkeypatch.setattr(oracle, attr, getattr(mod, attr))
    caught = []
    for call in PIN_CALLS:
        try:
            call()
        except AssertionError:
            caught.append(call)
    assert caught, f"no pin catches: {name}"


def test_unmutated_copy_passes(monkeypatch):
    """The copy mechanism itself changes nothing: every pin passes on it."""
    mod = _mutant_module("def stout(", "def stout(")
    for attr in ("stout", "clover_logdet", "Operator"):
        monkeypatch.setattr(oracle, attr, getattr(mod, attr))
    for call in PIN_CALLS:
        call()
