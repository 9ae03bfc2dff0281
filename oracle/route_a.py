"""Route A of the oracle: determinant space, literal Jordan-Wigner application.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (this implementation's readings where the paper is silent or ambiguous):

* qubit j = spin-orbital j = 2p + sigma (sigma = 0 alpha, 1 beta); bit j of a
  basis index is its occupation (introduction; Methodology, Strategy 2, the
  Jordan-Wigner mapping of a+_{p sigma} a_{q sigma}).
* an excitation row is ``(kind, i, j, a, b)``: kind 1 is T = a+_a a_i (j, b
  unused), kind 2 is T = a+_a a+_b a_j a_i with i<j and a<b; kinds 3 and 4 are
  the qubit excitations of the QEB pool ("Computational Details"): the same
  products of qubit raising / lowering operators, without the Jordan-Wigner sign.  The ansatz is
  U_L ... U_1 |ref> with U_k = exp(theta_k (T_k - T_k^dagger)), op 1 acting
  first (ADAPT-VQE pool of fermionic excitations, Methodology, "Computational
  Details").
* H = E_nuc + sum h_pq a+_{p s} a_{q s} + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
  (FCIDUMP chemist notation, "Computational Details").
* E = <psi|H|psi> / <psi|psi>; gradient dE/dtheta_k in Ha per radian of theta_k.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        lib.orc_sector_dim.restype = i64
        lib.orc_sector_dim.argtypes = [i32, i32, i32]
        lib.orc_sector_list.restype = i64
        lib.orc_sector_list.argtypes = [i32, i32, i32, vp]
        lib.orc_det_index.restype = i64
        lib.orc_det_index.argtypes = [vp, i64, ctypes.c_uint64]
        lib.orc_exc_apply.restype = i32
        lib.orc_exc_apply.argtypes = [vp, ctypes.c_uint64, vp]
        lib.orc_generator_apply.restype = None
        lib.orc_generator_apply.argtypes = [vp, i64, vp, vp, vp]
        lib.orc_rotate.restype = None
        lib.orc_rotate.argtypes = [vp, i64, vp, dbl, vp, vp]
        lib.orc_hamiltonian_apply.restype = None
        lib.orc_hamiltonian_apply.argtypes = [i32, vp, i64, vp, vp, dbl, vp, vp, vp, i64]
        lib.orc_rdm1.restype = None
        lib.orc_rdm1.argtypes = [i32, vp, i64, vp, vp]
        lib.orc_num_threads.restype = i32
        lib.orc_num_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the C core uses."""
    return int(_load().orc_num_threads())


class Sector:
    """All determinants with ``na`` alpha and ``nb`` beta electrons, sorted ascending."""

    def __init__(self, n: int, na: int, nb: int):
        lib = _load()
        self.n, self.na, self.nb = int(n), int(na), int(nb)
        D = lib.orc_sector_dim(self.n, self.na, self.nb)
        if D < 0:
            raise ValueError("bad sector (n=%d, na=%d, nb=%d)" % (n, na, nb))
        self.dets = np.empty(D, dtype=np.uint64)
        got = lib.orc_sector_list(self.n, self.na, self.nb, _ptr(self.dets))
        if got != D:
            raise RuntimeError("sector enumeration failed")
        self.D = int(D)

    def index(self, x: int) -> int:
        """Position of determinant ``x`` in the list (-1 if it is not in the sector)."""
        return int(_load().orc_det_index(_ptr(self.dets), self.D, ctypes.c_uint64(int(x))))


def _op_row(op) -> np.ndarray:
    r = np.asarray(op, dtype=np.int32).reshape(-1)
    if r.size != 5:
        raise ValueError("an excitation row is (kind, i, j, a, b)")
    return np.ascontiguousarray(r)


def exc_apply(op, x: int):
    """T|x> for one determinant: returns (sign, y); sign 0 when T annihilates |x>."""
    y = np.zeros(1, dtype=np.uint64)
    s = _load().orc_exc_apply(_ptr(_op_row(op)), ctypes.c_uint64(int(x)), _ptr(y))
    return int(s), int(y[0])


def hf_state(sec: Sector, occ) -> np.ndarray:
    """|x_HF> with the listed spin-orbitals occupied (complex128 over the sector)."""
    x = 0
    for j in occ:
        x |= 1 << int(j)
    I = sec.index(x)
    if I < 0:
        raise ValueError("reference determinant is not in the sector")
    psi = np.zeros(sec.D, dtype=np.complex128)
    psi[I] = 1.0
    return psi


def generator_apply(sec: Sector, op, psi: np.ndarray) -> np.ndarray:
    """(T - T^dagger) psi."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().orc_generator_apply(_ptr(sec.dets), sec.D, _ptr(_op_row(op)), _ptr(psi), _ptr(out))
    return out


def rotate(sec: Sector, op, theta: float, psi: np.ndarray) -> np.ndarray:
    """exp(theta (T - T^dagger)) psi."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    _load().orc_rotate(_ptr(sec.dets), sec.D, _ptr(_op_row(op)), float(theta), _ptr(psi), _ptr(out))
    return out


def apply_ansatz(sec: Sector, ops, theta, psi0: np.ndarray) -> np.ndarray:
    """U_L ... U_1 psi0, op 0 of ``ops`` acting first."""
    ops = np.asarray(ops, dtype=np.int32).reshape(-1, 5)
    theta = np.asarray(theta, dtype=np.float64).reshape(-1)
    if len(theta) != len(ops):
        raise ValueError("one angle per excitation")
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    for k in range(len(ops)):
        psi = rotate(sec, ops[k], theta[k], psi)
    return psi


def hamiltonian_apply(sec: Sector, h, eri, e_nuc: float, psi: np.ndarray, rows=None) -> np.ndarray:
    """H psi (every determinant, or only the determinant positions in ``rows``)."""
    N = sec.n // 2
    h = np.ascontiguousarray(h, dtype=np.float64).reshape(N, N)
    eri = np.ascontiguousarray(eri, dtype=np.float64).reshape(N, N, N, N)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    if rows is None:
        out = np.empty(sec.D, dtype=np.complex128)
        rp, nr = None, 0
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(len(rows), dtype=np.complex128)
        rp, nr = _ptr(rows), len(rows)
    _load().orc_hamiltonian_apply(sec.n, _ptr(sec.dets), sec.D, _ptr(h), _ptr(eri), float(e_nuc),
                                  _ptr(psi), _ptr(out), rp, nr)
    return out


def energy(sec: Sector, h, eri, e_nuc: float, psi: np.ndarray) -> float:
    """E = <psi|H|psi> / <psi|psi>."""
    sigma = hamiltonian_apply(sec, h, eri, e_nuc, psi)
    return float(np.vdot(psi, sigma).real / np.vdot(psi, psi).real)


def energy_grad(sec: Sector, h, eri, e_nuc: float, ops, theta, psi0: np.ndarray):
    """Energy and exact gradient of E(theta) = <psi(theta)|H|psi(theta)>, psi = U_L..U_1 psi0.

    Textbook adjoint recursion: with psi_k = U_k..U_1 psi0 and lambda_k =
    U_{k+1}^dagger .. U_L^dagger H psi_L, dE/dtheta_k = 2 Re <lambda_k| G_k psi_k>
    (dU_k/dtheta_k = G_k U_k).  Walking k = L..1 turns psi_k into psi_{k-1} and
    lambda_k into lambda_{k-1} by applying U_k^dagger = exp(-theta_k G_k).
    Returns (E, g) with g[k] = dE/dtheta_k.
    """
    ops = np.asarray(ops, dtype=np.int32).reshape(-1, 5)
    theta = np.asarray(theta, dtype=np.float64).reshape(-1)
    psi = apply_ansatz(sec, ops, theta, psi0)
    lam = hamiltonian_apply(sec, h, eri, e_nuc, psi)
    norm = np.vdot(psi, psi).real
    E = float(np.vdot(psi, lam).real / norm)
    g = np.zeros(len(ops))
    for k in range(len(ops) - 1, -1, -1):
        g[k] = 2.0 * np.vdot(lam, generator_apply(sec, ops[k], psi)).real / norm
        psi = rotate(sec, ops[k], -theta[k], psi)
        lam = rotate(sec, ops[k], -theta[k], lam)
    return E, g


def rdm1(sec: Sector, psi: np.ndarray) -> np.ndarray:
    """n[sigma, p, q] = <psi|a+_{p sigma} a_{q sigma}|psi> / <psi|psi>, complex [2, N, N]."""
    N = sec.n // 2
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty((2, N, N), dtype=np.complex128)
    _load().orc_rdm1(sec.n, _ptr(sec.dets), sec.D, _ptr(psi), _ptr(out))
    return out / np.vdot(psi, psi).real


def cnot_counts(ops):
    """CNOT cost of an ansatz in the two pools of Table IV: (QEB pool, qubit pool).

    Table IV's caption prints the formulas garbled; the reading that fits every
    row of the table is N_CNOT = 3 N_single + 13 N_double (QEB pool) and
    2 N_single + 6 N_double (qubit pool).
    """
    ops = np.asarray(ops, dtype=np.int32).reshape(-1, 5)
    ns = int(np.sum((ops[:, 0] == 1) | (ops[:, 0] == 3)))
    nd = int(np.sum((ops[:, 0] == 2) | (ops[:, 0] == 4)))
    return 3 * ns + 13 * nd, 2 * ns + 6 * nd
