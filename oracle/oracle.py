"""ctypes front end of the FP64 CPU oracle in ``bqcd_oracle.c``.

TEST INFRASTRUCTURE.  Each function names the part of arXiv:1711.03836 it
follows; the arithmetic lives in the C file and is written from the
definitions (Eq. 1 hopping term with chemical potential, Eq. 2 clover term,
Eq. 5 U(1) phases, the even-odd Schur complement of M = A - kappa D_hop,
textbook CG).  Stout smearing of the hopping links (Eq. 5's singly iterated
stout links, after Morningstar and Peardon 2004) and the clover log det are
written here in numpy: staples by array shifts, exp(iQ) by the eigen-
decomposition of the Hermitian Q, log det by numpy's slogdet of each site's
12x12 clover matrix.  Fields use the canonical host layouts:

  links   U[V][4][3][3] complex128, site lex = x + Lx*(y + Ly*(z + Lz*t))
  U(1)    A[V][4] float64 (or None)
  spinor  half lattice [V/2][4][3] complex128, indexed by lex/2

Nothing here imports the CUDA library, and the CUDA library imports nothing
from here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bqcd_oracle.c")
_LIB = os.path.join(_HERE, "libbqcd_oracle.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """Mirror of ``or_params`` in the C file."""

    _fields_ = [
        ("L", ctypes.c_int * 4),
        ("kappa", ctypes.c_double),
        ("csw", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("t_bc", ctypes.c_double),
        ("charge", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``libbqcd_oracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.POINTER(Params)
    dp = ctypes.c_void_p
    L = ctypes.c_long
    i = ctypes.c_int
    d = ctypes.c_double
    sig = {
        "or_gamma": (None, [i, dp]),
        "or_dhop": (None, [P, dp, dp, dp, i, i, dp]),
        "or_dhop_sites": (None, [P, dp, dp, dp, i, i, L, dp, dp]),
        "or_clover_field": (None, [P, dp, i, dp]),
        "or_clover_invert": (L, [L, dp, dp]),
        "or_clover_apply": (None, [L, dp, dp, i, dp]),
        "or_clover_sites": (i, [P, dp, i, i, L, dp, dp, dp]),
        "or_mhat": (None, [P, dp, dp, dp, dp, dp, i, dp]),
        "or_mdagm": (None, [P, dp, dp, dp, dp, dp, d, dp]),
        "or_mhat_sites": (i, [P, dp, dp, dp, i, L, dp, dp]),
        "or_cg": (i, [P, dp, dp, dp, dp, dp, d, d, i, dp]),
        "or_num_threads": (i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def load_library(path):
    """Load another build of the oracle's C source (used by the mutation tests)."""
    return _bind(ctypes.CDLL(path))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def params(dims, kappa=0.125, csw=0.0, mu=0.0, t_bc=-1.0, charge=0.0) -> Params:
    p = Params()
    for k in range(4):
        p.L[k] = int(dims[k])
    p.kappa, p.csw, p.mu, p.t_bc, p.charge = float(kappa), float(csw), float(mu), float(t_bc), float(charge)
    return p


def half_volume(p: Params) -> int:
    return p.L[0] * p.L[1] * p.L[2] * p.L[3] // 2


def num_threads() -> int:
    return _load().or_num_threads()


def gamma(k: int) -> np.ndarray:
    """The oracle's gamma_{k+1} (k=0..3) or gamma_5 (k=4), chiral basis."""
    out = np.zeros((4, 4), np.complex128)
    _load().or_gamma(k, _ptr(out))
    return out


def dhop(p, U, A, psi, out_parity, dagger=False):
    """D_hop (Eq. 1, Eq. 5) from the opposite parity onto ``out_parity``."""
    U, psi = _c128(U), _c128(psi)
    A = None if A is None else np.ascontiguousarray(A, np.float64)
    out = np.empty((half_volume(p), 4, 3), np.complex128)
    _load().or_dhop(ctypes.byref(p), _ptr(U), _ptr(A), _ptr(psi), out_parity, int(dagger), _ptr(out))
    return out


def dhop_sites(p, U, A, psi, out_parity, sites, dagger=False):
    U, psi = _c128(U), _c128(psi)
    A = None if A is None else np.ascontiguousarray(A, np.float64)
    sites = np.ascontiguousarray(sites, np.int64)
    out = np.empty((len(sites), 4, 3), np.complex128)
    _load().or_dhop_sites(ctypes.byref(p), _ptr(U), _ptr(A), _ptr(psi), out_parity, int(dagger),
                          len(sites), _ptr(sites), _ptr(out))
    return out


def clover_field(p, U, parity):
    """A(x) = 1 + i kappa c_SW sum_{mu<nu} sigma F (Eq. 2) as [V/2][12][12]."""
    U = _c128(U)
    out = np.empty((half_volume(p), 12, 12), np.complex128)
    _load().or_clover_field(ctypes.byref(p), _ptr(U), parity, _ptr(out))
    return out


def clover_invert(Am):
    Am = _c128(Am)
    out = np.empty_like(Am)
    bad = _load().or_clover_invert(Am.shape[0], _ptr(Am), _ptr(out))
    if bad:
        raise np.linalg.LinAlgError(f"{bad} singular clover sites")
    return out


def clover_apply(Am, psi, dagger=False):
    Am, psi = _c128(Am), _c128(psi)
    out = np.empty(psi.shape, np.complex128)
    _load().or_clover_apply(Am.shape[0], _ptr(Am), _ptr(psi), int(dagger), _ptr(out))
    return out


def clover_sites(p, U, parity, psi, sites, inverse=False):
    U, psi = _c128(U), _c128(psi)
    sites = np.ascontiguousarray(sites, np.int64)
    out = np.empty((len(sites), 4, 3), np.complex128)
    bad = _load().or_clover_sites(ctypes.byref(p), _ptr(U), parity, int(inverse), len(sites),
                                  _ptr(sites), _ptr(psi), _ptr(out))
    if bad:
        raise np.linalg.LinAlgError(f"{bad} singular clover sites")
    return out


def stout(dims, U, rho, n_iter=1):
    """n_iter stout steps of every link (Morningstar and Peardon 2004):
    C_mu(x) = rho sum_{nu != mu} [U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                  + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)],
    Omega = C_mu(x) U_mu(x)^dag, Q = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega),
    U'_mu(x) = exp(iQ) U_mu(x); links periodic in every direction."""
    Lx, Ly, Lz, Lt = dims
    W = _c128(U).reshape(Lt, Lz, Ly, Lx, 4, 3, 3)
    ax = {0: 3, 1: 2, 2: 1, 3: 0}

    def at(F, mu, d):
        """F(x + d mu-hat)."""
        return np.roll(F, -d, axis=ax[mu])

    def dag(F):
        return np.conj(np.swapaxes(F, -1, -2))

    for _ in range(n_iter):
        out = np.empty_like(W)
        for mu in range(4):
            Umu = W[..., mu, :, :]
            C = np.zeros_like(Umu)
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = W[..., nu, :, :]
                C += Unu @ at(Umu, nu, 1) @ dag(at(Unu, mu, 1))
                Unu_m = at(Unu, nu, -1)
                C += dag(Unu_m) @ at(Umu, nu, -1) @ at(Unu_m, mu, 1)
            Om = rho * C @ dag(Umu)
            D = dag(Om) - Om
            Q = 0.5j * D - (1j / 6.0) * np.trace(D, axis1=-2, axis2=-1)[..., None, None] * np.eye(3)
            Q = 0.5 * (Q + dag(Q))  # Hermitian up to rounding; eigh reads one triangle
            q, Wv = np.linalg.eigh(Q)
            expQ = (Wv * np.exp(1j * q)[..., None, :]) @ dag(Wv)
            out[..., mu, :, :] = expQ @ Umu
        W = out
    return W.reshape(np.shape(U))


def clover_logdet(p, U, parity):
    """(sum over the sites of `parity` of log|det A(x)|, number of sites with
    det A(x) < 0), A(x) the 12x12 clover matrix of Eq. 2."""
    sign, ld = np.linalg.slogdet(clover_field(p, U, parity))
    return float(np.sum(ld)), int(np.sum(sign.real < 0))


class Operator:
    """The even-odd operator of one gauge field: clover blocks built once.
    U_hop (optional) replaces U in the hopping term (stout-smeared links); the
    clover term is always built from U."""

    def __init__(self, p: Params, U, A=None, U_hop=None):
        self.p = p
        self.U_thin = _c128(U)
        self.U = self.U_thin if U_hop is None else _c128(U_hop)
        self.A = None if A is None else np.ascontiguousarray(A, np.float64)
        self.Aee = clover_field(p, self.U_thin, 0)
        self.Aoo = clover_field(p, self.U_thin, 1)
        self.Aoo_inv = clover_invert(self.Aoo)

    def mhat(self, psi, dagger=False):
        """Mhat psi = A_ee psi - kappa^2 D_eo A_oo^{-1} D_oe psi (or its adjoint)."""
        psi = _c128(psi)
        out = np.empty_like(psi)
        _load().or_mhat(ctypes.byref(self.p), _ptr(self.U), _ptr(self.A), _ptr(self.Aee),
                        _ptr(self.Aoo_inv), _ptr(psi), int(dagger), _ptr(out))
        return out

    def mdagm(self, psi, sigma=0.0):
        psi = _c128(psi)
        out = np.empty_like(psi)
        _load().or_mdagm(ctypes.byref(self.p), _ptr(self.U), _ptr(self.A), _ptr(self.Aee),
                         _ptr(self.Aoo_inv), _ptr(psi), float(sigma), _ptr(out))
        return out

    def cg(self, b, sigma=0.0, tol=1e-10, maxiter=10000):
        """Textbook CG on (Mhat^dagger Mhat + sigma) x = b from x = 0."""
        b = _c128(b)
        x = np.empty_like(b)
        it = _load().or_cg(ctypes.byref(self.p), _ptr(self.U), _ptr(self.A), _ptr(self.Aee),
                           _ptr(self.Aoo_inv), _ptr(b), float(sigma), float(tol), int(maxiter), _ptr(x))
        return x, it

    def multishift(self, b, shifts, tol=1e-10, maxiter=10000):
        """Multishift reference: one independent CG per shift."""
        return [self.cg(b, s, tol, maxiter)[0] for s in shifts]

    def full(self, x_e, x_o):
        """M x = (A - kappa D_hop) x on the whole lattice (Eq. 1, Eq. 2), as its
        even and odd halves: (M x)_p = A_pp x_p - kappa D_{p,1-p} x_{1-p}."""
        k = self.p.kappa
        y_e = clover_apply(self.Aee, x_e) - k * dhop(self.p, self.U, self.A, x_o, 0)
        y_o = clover_apply(self.Aoo, x_o) - k * dhop(self.p, self.U, self.A, x_e, 1)
        return y_e, y_o

    def full_dagger(self, x_e, x_o):
        """M^dag x = (A - kappa D_hop^dag) x (A Hermitian), as even and odd halves."""
        k = self.p.kappa
        y_e = clover_apply(self.Aee, x_e) - k * dhop(self.p, self.U, self.A, x_o, 0, dagger=True)
        y_o = clover_apply(self.Aoo, x_o) - k * dhop(self.p, self.U, self.A, x_e, 1, dagger=True)
        return y_e, y_o

    def solve_full(self, b_e, b_o, tol=1e-12, maxiter=20000, dagger=False):
        """x with M x = b by block elimination of the odd sites: CG on
        Mhat^dag Mhat x_e = Mhat^dag (b_e + kappa D_eo A_oo^{-1} b_o), then
        x_o = A_oo^{-1} (b_o + kappa D_oe x_e). For M^dag x = b the same with
        D^dag: Mhat^dag x_e = bhat by CG on Mhat^dag Mhat z = bhat, x_e = Mhat z."""
        k = self.p.kappa
        bhat = _c128(b_e) + k * dhop(self.p, self.U, self.A, clover_apply(self.Aoo_inv, b_o), 0, dagger=dagger)
        if dagger:
            z, _ = self.cg(bhat, tol=tol, maxiter=maxiter)
            x_e = self.mhat(z)
        else:
            x_e, _ = self.cg(self.mhat(bhat, dagger=True), tol=tol, maxiter=maxiter)
        x_o = clover_apply(self.Aoo_inv, _c128(b_o) + k * dhop(self.p, self.U, self.A, x_e, 1, dagger=dagger))
        return x_e, x_o

    def trace_samples(self, eta_e, eta_o, tol=1e-12):
        """(eta^dag M^{-1} eta, eta^dag gamma_5 M^{-1} eta, |M^{-dag} eta|^2) of one
        noise vector: the summands of the stochastic estimates of Tr M^{-1},
        Tr gamma_5 M^{-1} and Tr (M^dag M)^{-1}."""
        x_e, x_o = self.solve_full(eta_e, eta_o, tol=tol)
        y_e, y_o = self.solve_full(eta_e, eta_o, tol=tol, dagger=True)
        g5 = np.array([1, 1, -1, -1], float)[None, :, None]
        s1 = np.vdot(eta_e, x_e) + np.vdot(eta_o, x_o)
        s2 = np.vdot(eta_e, g5 * x_e) + np.vdot(eta_o, g5 * x_o)
        s3 = np.vdot(y_e, y_e).real + np.vdot(y_o, y_o).real
        return np.array([s1, s2, s3])


def mhat_sites(p, U, A, psi, sites, dagger=False):
    """Mhat psi (or Mhat^dagger psi) at listed even half sites, built on the fly."""
    U, psi = _c128(U), _c128(psi)
    A = None if A is None else np.ascontiguousarray(A, np.float64)
    sites = np.ascontiguousarray(sites, np.int64)
    out = np.empty((len(sites), 4, 3), np.complex128)
    bad = _load().or_mhat_sites(ctypes.byref(p), _ptr(U), _ptr(A), _ptr(psi), int(dagger), len(sites),
                                _ptr(sites), _ptr(out))
    if bad:
        raise np.linalg.LinAlgError(f"{bad} singular clover sites")
    return out
