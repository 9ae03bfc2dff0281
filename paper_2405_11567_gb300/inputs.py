"""Seeded synthetic inputs shaped like the paper's molecular workloads.

This module only draws numbers and enumerates operator lists.  It holds none of
the method's arithmetic (no state, no Hamiltonian action, no signs), so both the
CUDA path's tests and the CPU oracle's tests take their inputs from here.

The paper's workloads are real molecules (H2O, N2, LiH, H2, H8 in STO-3G, 6-31G
and system-adapted basis sets, 4-32 qubits: Table II) whose integrals are not
available here.  These generators stand in for them with the same shapes:
N spatial orbitals, closed-shell Hartree-Fock reference, real 8-fold symmetric
positive-semidefinite two-electron integrals with a positive diagonal, and
ADAPT-style ansatz lengths comparable to Table IV (7 to 999 operators).

Recipe (fixed draw order from ``numpy.random.default_rng(seed)``):
  1. h off-diagonal: N(0, 0.05) (standard deviation), upper triangle, mirrored;
     h diagonal: ``linspace(-2, 1, N)`` (ascending, so the HF reference is aufbau).
  2. 2N symmetric Cholesky-like vectors L^k with N(0, 1) entries (upper triangle
     incl. diagonal, mirrored).
  3. t_p ~ U[0.3, 0.8]; L^k_pq <- d_p d_q L^k_pq with d_p = (t_p / sum_k (L^k_pp)^2)^(1/4),
     so that (pp|pp) = t_p exactly; (pq|rs) = sum_k L^k_pq L^k_rs.
  4. theta ~ N(0, 0.05) (standard deviation), one per operator.
  5. ADAPT-style list: operators drawn uniformly from the UCCSD pool, without
     replacement when the pool is at least as long as the list, else with.
E_nuc = 0.7.  Config seeds: 1000 + config id; batched instance i: 2000 + i.
"""
import numpy as np

E_NUC = 0.7


def synthetic_integrals(n_orb: int, rng):
    """(h [N,N], eri [N,N,N,N] chemist (pq|rs), e_nuc) drawn from ``rng`` (steps 1-3)."""
    N = int(n_orb)
    iu = np.triu_indices(N, 1)
    h = np.zeros((N, N))
    h[iu] = rng.normal(0.0, 0.05, size=len(iu[0]))
    h = h + h.T
    h[np.diag_indices(N)] = np.linspace(-2.0, 1.0, N)
    iu0 = np.triu_indices(N, 0)
    L = np.zeros((2 * N, N, N))
    raw = rng.normal(0.0, 1.0, size=(2 * N, len(iu0[0])))
    for k in range(2 * N):
        L[k][iu0] = raw[k]
        L[k] = L[k] + np.triu(L[k], 1).T
    t = rng.uniform(0.3, 0.8, size=N)
    diag = np.einsum("kpp->p", L * L)
    d = (t / diag) ** 0.25
    L = L * d[None, :, None] * d[None, None, :]
    eri = np.einsum("kpq,krs->pqrs", L, L)
    return h, eri, E_NUC


def hf_occupation(n_elec: int):
    """Spin-orbitals of the HF reference: the lowest ``n_elec`` (interleaved alpha/beta)."""
    return list(range(int(n_elec)))


def qeb_pool(n_qubits: int, n_elec: int) -> np.ndarray:
    """The same excitations as uccsd_pool as qubit excitations (kinds 3 and 4: no Jordan-Wigner sign)."""
    pool = uccsd_pool(n_qubits, n_elec).copy()
    pool[:, 0] += 2
    return pool


def uccsd_pool(n_qubits: int, n_elec: int) -> np.ndarray:
    """All spin-conserving singles then doubles from the HF reference, rows (kind, i, j, a, b).

    Singles: i occupied, a virtual, same spin, ordered by (i, a).  Doubles:
    i<j occupied, a<b virtual, same number of alpha spin-orbitals in {i,j} and
    {a,b}, ordered lexicographically by (i, j, a, b).  Unused slots are -1.
    """
    occ = list(range(n_elec))
    vir = list(range(n_elec, n_qubits))
    rows = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                rows.append((1, i, -1, a, -1))
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for ia, a in enumerate(vir):
                for b in vir[ia + 1:]:
                    if sorted((i % 2, j % 2)) == sorted((a % 2, b % 2)):
                        rows.append((2, i, j, a, b))
    return np.array(rows, dtype=np.int32).reshape(-1, 5)


def adapt_list(pool: np.ndarray, length: int, rng) -> np.ndarray:
    """``length`` operators drawn from ``pool`` (step 5)."""
    replace = len(pool) < length
    idx = rng.choice(len(pool), size=int(length), replace=replace)
    return np.ascontiguousarray(pool[idx])


def batch_electrons(n_qubits: int) -> int:
    """Electrons for a batched instance: qubits/4 rounded to an even number, ties up."""
    return 2 * int(np.floor(n_qubits / 8.0 + 0.5))


# The five workloads.  "ansatz": "uccsd" uses the whole pool in pool order,
# an integer means an ADAPT-style list of that length.
CONFIGS = {
    1: dict(n_qubits=8, n_elec=2, ansatz="uccsd", dtype="c128", what="energy"),
    2: dict(n_qubits=16, n_elec=4, ansatz="uccsd", dtype="c128", what="energy+grad"),
    3: dict(n_qubits=24, n_elec=8, ansatz=120, dtype="c64", what="energy+grad+rdm1"),
    4: dict(batch=512, qubit_choices=(10, 12, 14, 16, 18, 20), ansatz=40, dtype="c64",
            what="energy+grad"),
    5: dict(n_qubits=30, n_elec=10, ansatz=200, dtype="c64", what="energy+grad+rdm1"),
}


def make_problem(n_qubits: int, n_elec: int, ansatz, seed: int) -> dict:
    """One seeded problem: integrals, HF occupation, operator list and angles."""
    rng = np.random.default_rng(seed)
    N = n_qubits // 2
    h, eri, e_nuc = synthetic_integrals(N, rng)
    pool = uccsd_pool(n_qubits, n_elec)
    L = len(pool) if ansatz == "uccsd" else int(ansatz)
    theta = rng.normal(0.0, 0.05, size=L)
    ops = pool.copy() if ansatz == "uccsd" else adapt_list(pool, L, rng)
    return dict(n_qubits=int(n_qubits), n_elec=int(n_elec), n_orb=N,
                na=n_elec // 2, nb=n_elec // 2,
                h=h, eri=eri, e_nuc=float(e_nuc), occ=hf_occupation(n_elec),
                ops=np.ascontiguousarray(ops, dtype=np.int32), theta=theta, seed=int(seed))


def config_problem(cid: int) -> dict:
    """The problem of single-instance config ``cid`` (1, 2, 3 or 5)."""
    c = CONFIGS[cid]
    if "batch" in c:
        raise ValueError("config %d is batched: use batch_problems()" % cid)
    p = make_problem(c["n_qubits"], c["n_elec"], c["ansatz"], 1000 + cid)
    p["dtype"] = c["dtype"]
    return p


def batch_problems(count: int = 512, first: int = 0):
    """Instances ``first .. first+count-1`` of the batched config (config 4)."""
    c = CONFIGS[4]
    rng = np.random.default_rng(1004)
    qubits = rng.choice(np.array(c["qubit_choices"]), size=c["batch"])
    out = []
    for i in range(first, first + count):
        q = int(qubits[i % c["batch"]])
        out.append(make_problem(q, batch_electrons(q), c["ansatz"], 2000 + i))
    return out


def random_sector_state(n_qubits: int, na: int, nb: int, rng) -> np.ndarray:
    """A normalised complex dense 2^n vector supported on the (na, nb) sector."""
    dim = 1 << n_qubits
    idx = np.arange(dim, dtype=np.int64)
    ca = np.zeros(dim, dtype=np.int64)
    cb = np.zeros(dim, dtype=np.int64)
    for j in range(n_qubits):
        if j % 2 == 0:
            ca += (idx >> j) & 1
        else:
            cb += (idx >> j) & 1
    mask = (ca == na) & (cb == nb)
    v = np.zeros(dim, dtype=np.complex128)
    m = int(mask.sum())
    v[mask] = rng.normal(size=m) + 1j * rng.normal(size=m)
    return v / np.linalg.norm(v)
