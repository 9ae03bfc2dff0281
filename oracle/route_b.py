"""Route B of the oracle: dense 2^n matrices (n <= 12).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Everything here is built from explicit 2x2 matrices and library linear algebra,
independently of route A's bit arithmetic:

* a_j = I (x) ... (x) I (x) s (x) Z (x) ... (x) Z  with s = |0><1| on qubit j and
  the Jordan-Wigner string Z on every qubit k < j (Methodology, Strategy 2: the
  Jordan-Wigner mapping).  The left-most factor acts on the highest qubit, so
  bit j of the dense index is qubit j.
* H, T, G = T - T^dagger are matrix products of these a_j and their adjoints.
* U = scipy's matrix exponential of theta G.
* the ground state of a sector is the lowest eigenvalue of H restricted to the
  basis states with the right alpha / beta electron counts.
"""
import itertools

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg

_I2 = sp.identity(2, dtype=np.complex128, format="csr")
_Z = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]], dtype=np.complex128))
_S = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]], dtype=np.complex128))  # |0><1|


def annihilators(n: int):
    """[a_0, ..., a_{n-1}] as sparse 2^n x 2^n matrices."""
    if n > 14:
        raise ValueError("route B is for n <= 14")
    out = []
    for j in range(n):
        m = sp.identity(1, dtype=np.complex128, format="csr")
        for q in range(n - 1, -1, -1):          # left-most factor = highest qubit
            f = _I2 if q > j else (_S if q == j else _Z)
            m = sp.kron(m, f, format="csr")
        out.append(m.tocsr())
    return out


def qubit_lowering(n: int):
    """[s_0, ..., s_{n-1}]: |0><1| on one qubit, identity elsewhere (no Jordan-Wigner string)."""
    out = []
    for j in range(n):
        m = sp.identity(1, dtype=np.complex128, format="csr")
        for q in range(n - 1, -1, -1):
            m = sp.kron(m, _S if q == j else _I2, format="csr")
        out.append(m.tocsr())
    return out


def hamiltonian(n: int, h, eri, e_nuc: float, a=None):
    """Dense-index sparse H = E_nuc + sum h[PQ] a+_P a_Q + 1/2 sum [PQ|RS] a+_P a+_R a_S a_Q."""
    N = n // 2
    h = np.asarray(h, dtype=np.float64).reshape(N, N)
    eri = np.asarray(eri, dtype=np.float64).reshape(N, N, N, N)
    a = annihilators(n) if a is None else a
    ad = [m.conj().T.tocsr() for m in a]
    H = e_nuc * sp.identity(2 ** n, dtype=np.complex128, format="csr")
    for P in range(n):
        for Q in range(n):
            if P % 2 != Q % 2:
                continue
            H = H + h[P // 2, Q // 2] * (ad[P] @ a[Q])
    for P, Q, R, S in itertools.product(range(n), repeat=4):
        if P % 2 != Q % 2 or R % 2 != S % 2:
            continue
        v = eri[P // 2, Q // 2, R // 2, S // 2]
        if v == 0.0:
            continue
        H = H + (0.5 * v) * (ad[P] @ ad[R] @ a[S] @ a[Q])
    return H.tocsr()


def excitation_T(op, a, s=None):
    """T for a row (kind, i, j, a, b): a+_a a_i (kind 1), a+_a a+_b a_j a_i (kind 2); kinds 3, 4 are the
    same products of qubit operators s_j = |0><1| (list `s`, from qubit_lowering) with no string."""
    kind, i, j, va, vb = [int(v) for v in op]
    ops = a if kind <= 2 else s
    if ops is None:
        raise ValueError("qubit excitations need the qubit operators")
    ad = lambda k: ops[k].conj().T  # noqa: E731
    if kind in (1, 3):
        return (ad(va) @ ops[i]).tocsr()
    return (ad(va) @ ad(vb) @ ops[j] @ ops[i]).tocsr()


def generator(op, a, s=None):
    T = excitation_T(op, a, s)
    return (T - T.conj().T).tocsr()


def basis_state(n: int, occ) -> np.ndarray:
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[sum(1 << int(j) for j in occ)] = 1.0
    return psi


def unitary(op, theta: float, a, s=None) -> np.ndarray:
    """exp(theta G) as a dense matrix (scipy.linalg.expm)."""
    return scipy.linalg.expm(theta * generator(op, a, s).toarray())


def apply_ansatz(ops, theta, psi0, a, s=None):
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    for op, t in zip(np.asarray(ops).reshape(-1, 5), np.asarray(theta).reshape(-1)):
        psi = unitary(op, t, a, s) @ psi
    return psi


def energy(H, psi) -> float:
    return float(np.vdot(psi, H @ psi).real / np.vdot(psi, psi).real)


def gradient(H, ops, theta, psi0, a, s=None) -> np.ndarray:
    """dE/dtheta_k = 2 Re <psi_L| H U_L..U_{k+1} G_k U_k..U_1 |psi0>, one k at a time."""
    ops = np.asarray(ops).reshape(-1, 5)
    theta = np.asarray(theta).reshape(-1)
    L = len(ops)
    Us = [unitary(ops[k], theta[k], a, s) for k in range(L)]
    psi_L = np.array(psi0, dtype=np.complex128)
    for U in Us:
        psi_L = U @ psi_L
    Hpsi = H @ psi_L
    g = np.zeros(L)
    for k in range(L):
        v = np.array(psi0, dtype=np.complex128)
        for m in range(k + 1):
            v = Us[m] @ v
        v = generator(ops[k], a, s) @ v
        for m in range(k + 1, L):
            v = Us[m] @ v
        g[k] = 2.0 * np.vdot(Hpsi, v).real
    return g


def sector_indices(n: int, na: int, nb: int) -> np.ndarray:
    """Dense indices with na alpha (even-bit) and nb beta (odd-bit) electrons."""
    idx = np.arange(2 ** n, dtype=np.int64)
    ca = np.zeros_like(idx)
    cb = np.zeros_like(idx)
    for j in range(n):
        bit = (idx >> j) & 1
        if j % 2 == 0:
            ca += bit
        else:
            cb += bit
    return idx[(ca == na) & (cb == nb)]


def sector_spectrum(H, n: int, na: int, nb: int) -> np.ndarray:
    """All eigenvalues of H restricted to the (na, nb) sector, ascending."""
    s = sector_indices(n, na, nb)
    Hs = H[s][:, s].toarray()
    return np.linalg.eigvalsh(Hs)


def rdm1(psi, a, n: int) -> np.ndarray:
    """n[sigma, p, q] = <psi|a+_{p sigma} a_{q sigma}|psi> / <psi|psi>."""
    N = n // 2
    out = np.zeros((2, N, N), dtype=np.complex128)
    nrm = np.vdot(psi, psi).real
    for s in range(2):
        for p in range(N):
            for q in range(N):
                P, Q = 2 * p + s, 2 * q + s
                out[s, p, q] = np.vdot(psi, a[P].conj().T @ (a[Q] @ psi)) / nrm
    return out
