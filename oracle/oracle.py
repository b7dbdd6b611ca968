"""Python front end of the plain CPU FP64 oracle (``qcs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the product library never
imports it.  It compiles ``qcs_oracle.c`` with the host C compiler on first
use (or when the source is newer than the built library) and exposes each
exported C function with numpy arguments.

The oracle follows arXiv 2506.22408: Eq. (b_mat) and SI "Matrix Definitions"
for the matrices, Eq. (a_mat) and the node/interpolation paragraph of Sec.
"Classical shadows and the evaluation of overlaps" for the Pfaffian
polynomial, the estimator equation of the same section for o_p, Eqs.
(force_bias) and (force_bias_diff) for the force bias.  The header of
``qcs_oracle.c`` maps each step to its passage.

``variant(k)`` returns the same interface bound to a build with planted
mistake k (``-DORC_MUTATION=k``); the test-suite uses it to show that its
pins catch each planted mistake.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()

INTERP_ROOTS = 0
INTERP_CHEBYSHEV = 1

#: planted mistakes available through variant(k)
MUTATIONS = {
    1: "kappa = 1 (factor 2 of the (|0>+|Psi_T>)/sqrt2 preparation dropped)",
    2: "selected row (1, +i)/sqrt2 instead of (1, -i)/sqrt2 for occupied modes",
    3: "covariance sign flipped",
    4: "|det R| dropped (phase of det R kept)",
    5: "G = Q C_b Q^T instead of Q^T C_b Q",
    6: "phase i^{eta/2} dropped",
    7: "channel eigenvalues used as weights instead of their inverses",
    8: "Pfaffian pivot swap without the sign flip",
    9: "V = U^T instead of U^dagger",
    10: "1-RDM off-diagonal: signs of the mixed Majorana terms swapped",
    11: "gradient: column j not cleared before the unit entry is substituted",
    12: "force bias: tr(L G^T) instead of tr(L G)",
    13: "VCE factor: det R_c instead of its conjugate",
    14: "local energy: factor 2 of the symmetric second-derivative pairs dropped",
}


def _lib_path(mutation: int) -> str:
    return os.path.join(_BUILD, "liboracle.so" if mutation == 0 else f"liboracle_mut{mutation}.so")


def build(force: bool = False, mutation: int = 0) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _lib_path(mutation)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", f"-DORC_MUTATION={int(mutation)}",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Oracle:
    """The oracle's exported C functions with numpy arguments."""

    def __init__(self, mutation: int = 0):
        lib = ctypes.CDLL(build(mutation=mutation))
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.orc_covariance.argtypes = [i32, P, P]
        lib.orc_snapshot_G.argtypes = [i32, P, P, P]
        lib.orc_walker_qr.argtypes = [i32, i32, P, P, P]
        lib.orc_selection.argtypes = [i32, i32, P]
        lib.orc_selection.restype = i32
        lib.orc_pfaffian.argtypes = [i32, P, P]
        lib.orc_pair.argtypes = [i32, i32, P, P, P, i32, i32, P, P, P]
        lib.orc_pair_matrices.argtypes = [i32, i32, P, P, P, P, P, P]
        lib.orc_overlap.argtypes = [i32, i32, i64, i64, P, P, P, i32, i32, i32, P, P, P]
        lib.orc_overlap.restype = i32
        lib.orc_overlap_grad.argtypes = [i32, i32, i64, i64, P, P, P, i32, i32, i32, P, P]
        lib.orc_overlap_grad.restype = i32
        lib.orc_force_bias.argtypes = [i32, i32, i64, i32, P, P, P, P, f64, P]
        lib.orc_max_threads.restype = i32
        lib.orc_shadow_rdm.argtypes = [i32, i64, P, P, P, P, P, P, P, P]
        lib.orc_shadow_rdm.restype = i32
        lib.orc_vce_transform.argtypes = [i32, i32, i32, i32, P, P, P]
        lib.orc_vce_transform.restype = i32
        lib.orc_local_energy.argtypes = [i32, i32, i64, i64, P, P, P, P, P, i32, P, i32, P, P, P]
        lib.orc_local_energy.restype = i32
        self.lib = lib
        self.mutation = mutation

    def covariance(self, n, b):
        """C_b (2n x 2n), SI "Matrix Definitions" item 2."""
        b = _c(b, np.uint8)
        C = np.empty((2 * n, 2 * n))
        self.lib.orc_covariance(n, _p(b), _p(C))
        return C

    def snapshot_G(self, Q, b):
        """G = Q^T C_b Q, Eq. (b_mat)."""
        Q = _c(Q, np.float64)
        n = Q.shape[0] // 2
        b = _c(b, np.uint8)
        G = np.empty_like(Q)
        self.lib.orc_snapshot_G(n, _p(Q), _p(b), _p(G))
        return G

    def walker_qr(self, Phi):
        """Complete Householder QR: Phi = U[:, :ne] R."""
        Phi = _c(Phi, np.complex128)
        n, ne = Phi.shape
        U = np.empty((n, n), np.complex128)
        R = np.empty((ne, ne), np.complex128)
        self.lib.orc_walker_qr(n, ne, _p(Phi), _p(U), _p(R))
        return U, R

    def selection(self, n, ne):
        idx = np.empty(2 * n, np.int32)
        m = self.lib.orc_selection(n, ne, _p(idx))
        return idx[:m].copy()

    def pfaffian(self, A):
        """Pfaffian of a complex skew-symmetric matrix (Parlett-Reid, partial pivoting)."""
        A = _c(A, np.complex128)
        out = np.zeros(1, np.complex128)
        self.lib.orc_pfaffian(A.shape[0], _p(A), _p(out))
        return complex(out[0])

    def pair(self, Q, b, Phi, mode=INTERP_ROOTS, nodes=0):
        """One (walker, snapshot) pair: returns (o_p, coefficients c_0..c_ell, scale)."""
        Q = _c(Q, np.float64)
        b = _c(b, np.uint8)
        Phi = _c(Phi, np.complex128)
        n, ne = Phi.shape
        ell = n - ne // 2
        coef = np.zeros(ell + 1, np.complex128)
        out = np.zeros(1, np.complex128)
        sc = np.zeros(1)
        self.lib.orc_pair(n, ne, _p(Q), _p(b), _p(Phi), mode, nodes, _p(coef), _p(out), _p(sc))
        return complex(out[0]), coef, float(sc[0])

    def pair_matrices(self, Q, b, Phi):
        """(B^(s), C_0^(s), det R) of one pair."""
        Q = _c(Q, np.float64)
        b = _c(b, np.uint8)
        Phi = _c(Phi, np.complex128)
        n, ne = Phi.shape
        m = 2 * n - ne
        Bs = np.zeros((m, m), np.complex128)
        C0s = np.zeros((m, m))
        detR = np.zeros(1, np.complex128)
        self.lib.orc_pair_matrices(n, ne, _p(Q), _p(b), _p(Phi), _p(Bs), _p(C0s), _p(detR))
        return Bs, C0s, complex(detR[0])

    def overlap(self, Phi, Q, b, mode=INTERP_ROOTS, nodes=0, threads=0, per_pair=False):
        """Shadow overlaps <Psi_T|phi_w> for every walker (mean over snapshots).

        Phi: (W, n, ne) complex; Q: (P, 2n, 2n); b: (P, n) 0/1 bytes.
        Returns (overlap[W], per_pair[W, P] or None, scale[W, P] or None, threads_used).
        """
        Phi = _c(Phi, np.complex128)
        Q = _c(Q, np.float64)
        b = _c(b, np.uint8)
        W, n, ne = Phi.shape
        P = Q.shape[0]
        ov = np.zeros(W, np.complex128)
        pp = np.zeros((W, P), np.complex128) if per_pair else None
        sc = np.zeros((W, P)) if per_pair else None
        used = self.lib.orc_overlap(n, ne, W, P, _p(Phi), _p(Q), _p(b), mode, nodes, threads, _p(ov), _p(pp),
                                    _p(sc))
        return ov, pp, sc, used

    def overlap_grad(self, Phi, Q, b, mode=INTERP_ROOTS, nodes=0, threads=0):
        """(overlap[W], grad[W, n, ne], threads_used); grad = dO/dPhi (holomorphic)."""
        Phi = _c(Phi, np.complex128)
        Q = _c(Q, np.float64)
        b = _c(b, np.uint8)
        W, n, ne = Phi.shape
        P = Q.shape[0]
        ov = np.zeros(W, np.complex128)
        g = np.zeros((W, n, ne), np.complex128)
        used = self.lib.orc_overlap_grad(n, ne, W, P, _p(Phi), _p(Q), _p(b), mode, nodes, threads, _p(ov), _p(g))
        return ov, g, used

    def force_bias(self, L, Phi, ov, grad, sqrt_dt=0.0):
        """xbar[W, nchol] = -sqrt_dt * i tr(L_gamma Phi g^T / O); sqrt_dt = 0 returns <v_gamma>."""
        L = _c(L, np.complex128)
        Phi = _c(Phi, np.complex128)
        ov = _c(ov, np.complex128)
        grad = _c(grad, np.complex128)
        W, n, ne = Phi.shape
        nchol = L.shape[0]
        xb = np.zeros((W, nchol), np.complex128)
        self.lib.orc_force_bias(n, ne, W, nchol, _p(L), _p(Phi), _p(ov), _p(grad), float(sqrt_dt), _p(xb))
        return xb

    def shadow_rdm(self, Q, b, w=None, R=None, deg4=False):
        """Shadow estimates (SI "Reduced Density Matrices"): dict(gam2 (2n x 2n real,
        <g~_mu g~_nu> = i gam2), gam4 (C(2n,4) real, mu<nu<rho<sigma lexicographic) when
        deg4, rdm1 (n x n complex), npart).  w: optional per-snapshot weights; R: rotation."""
        Q = _c(Q, np.float64)
        b = _c(b, np.uint8)
        P, N2, _ = Q.shape
        n = N2 // 2
        w = _c(w, np.float64) if w is not None else None
        R = _c(R, np.float64) if R is not None else None
        gam2 = np.zeros((N2, N2))
        from math import comb
        gam4 = np.zeros(comb(N2, 4)) if deg4 else None
        rdm1 = np.zeros((n, n), np.complex128)
        npart = ctypes.c_double(0.0)
        rc = self.lib.orc_shadow_rdm(n, P, _p(Q), _p(b), _p(w), _p(R), _p(gam2), _p(gam4), _p(rdm1),
                                     ctypes.byref(npart))
        if rc != 0:
            raise ValueError("orc_shadow_rdm: bad sizes")
        return dict(gam2=gam2, gam4=gam4, rdm1=rdm1, npart=npart.value)

    def vce_transform(self, Phi, nc, na, nea):
        """(act[na, nea], factor) of the virtual-correlation-energy transform of one
        spin sector of a full-space walker Phi (NB x (nc + nea))."""
        Phi = _c(Phi, np.complex128)
        NB = Phi.shape[0]
        act = np.zeros((na, nea), np.complex128)
        f = np.zeros(1, np.complex128)
        if self.lib.orc_vce_transform(NB, nc, na, nea, _p(Phi), _p(act), _p(f)) != 0:
            raise ValueError("orc_vce_transform: bad sizes")
        return act, f[0]

    def local_energy(self, Phi, Q, b, L, h=None, threads=0, w=None):
        """(overlap[W], e1[W], e2[W]): e1 = <Psi_T|hhat|phi>/O (zeros without h),
        e2 = sum_gamma <Psi_T|Lhat_gamma^2|phi>/O, by walker-side column substitution."""
        Phi = _c(Phi, np.complex128)
        Q = _c(Q, np.float64)
        b = _c(b, np.uint8)
        L = _c(L, np.complex128)
        hh = _c(h, np.complex128) if h is not None else None
        w = _c(w, np.float64) if w is not None else None
        W, n, ne = Phi.shape
        P = Q.shape[0]
        ov = np.zeros(W, np.complex128)
        e1 = np.zeros(W, np.complex128)
        e2 = np.zeros(W, np.complex128)
        self.lib.orc_local_energy(n, ne, W, P, _p(Phi), _p(Q), _p(b), _p(w), _p(hh), L.shape[0], _p(L), threads,
                                  _p(ov), _p(e1), _p(e2))
        return ov, e1, e2

    def max_threads(self) -> int:
        return int(self.lib.orc_max_threads())


_instances: dict[int, Oracle] = {}


def variant(mutation: int = 0) -> Oracle:
    with _lock:
        if mutation not in _instances:
            _instances[mutation] = Oracle(mutation)
        return _instances[mutation]


def _default() -> Oracle:
    return variant(0)


def covariance(n, b):
    return _default().covariance(n, b)


def snapshot_G(Q, b):
    return _default().snapshot_G(Q, b)


def walker_qr(Phi):
    return _default().walker_qr(Phi)


def selection(n, ne):
    return _default().selection(n, ne)


def pfaffian(A):
    return _default().pfaffian(A)


def pair(Q, b, Phi, mode=INTERP_ROOTS, nodes=0):
    return _default().pair(Q, b, Phi, mode, nodes)


def pair_matrices(Q, b, Phi):
    return _default().pair_matrices(Q, b, Phi)


def overlap(Phi, Q, b, mode=INTERP_ROOTS, nodes=0, threads=0, per_pair=False):
    return _default().overlap(Phi, Q, b, mode, nodes, threads, per_pair)


def overlap_grad(Phi, Q, b, mode=INTERP_ROOTS, nodes=0, threads=0):
    return _default().overlap_grad(Phi, Q, b, mode, nodes, threads)


def force_bias(L, Phi, ov, grad, sqrt_dt=0.0):
    return _default().force_bias(L, Phi, ov, grad, sqrt_dt)


def shadow_rdm(Q, b, w=None, R=None, deg4=False):
    return _default().shadow_rdm(Q, b, w, R, deg4)


def vce_transform(Phi, nc, na, nea):
    return _default().vce_transform(Phi, nc, na, nea)


def local_energy(Phi, Q, b, L, h=None, threads=0, w=None):
    return _default().local_energy(Phi, Q, b, L, h, threads, w)


def max_threads() -> int:
    return _default().max_threads()
