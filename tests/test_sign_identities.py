"""Jordan-Wigner sign identities the string-row kernels rely on (pure arithmetic, CPU).

With interleaved spin-orbitals j = 2p + s, the sign of a same-spin single p -> q on a
determinant x is (-1)^popc(x & between(2p, 2q)), and of a same-spin double
p1 < p2 -> q1 < q2 taken as -(a+_q1 a_p2)(a+_q2 a_p1) it is the product of the two
single signs in that order.  k_sigma_same evaluates both from the prefix-parity words
pp(s) (bit u = parity of the bits of s below u) of the alpha and beta strings:
    single  popc(PP & {p, q}) + [p < q]
    double  popc(PP & {p1, p2, q1, q2}) + [p1<q2] + [q2<p2] + [p1<q1] + [p2<q1]
with PP = pp(a) ^ pp(b) (the orbital-order terms are folded into its integral table).
"""
import itertools

import numpy as np
import pytest


def _par(v):
    return bin(v).count("1") & 1


def _between(a, b):
    lo, hi = min(a, b), max(a, b)
    return ((1 << hi) - 1) & ~((2 << lo) - 1)


def _spread(s, off, N):
    return sum(1 << (2 * p + off) for p in range(N) if (s >> p) & 1)


def _pp(s):
    return sum((_par(s & ((1 << u) - 1)) << u) for u in range(17))


def _pp_scan(s):
    """The kernel's prefix-xor scan of s << 1 (5 shift-xor steps)."""
    y = (s << 1) & 0xFFFFFFFF
    for k in (1, 2, 4, 8, 16):
        y ^= (y << k) & 0xFFFFFFFF
    return y


def test_prefix_parity_scan():
    for s in list(range(1 << 10)) + [0xFFFF, 0xA5A5, 0x8001]:
        assert _pp_scan(s) & 0x1FFFF == _pp(s)


def test_same_spin_signs_from_prefix_parity():
    N = 7
    rng = np.random.default_rng(5)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, 1 << N, size=(400, 2))]
    bad = 0
    for a, b in pairs:
        for spin in (0, 1):
            own, other = (a, b) if spin == 0 else (b, a)
            x = _spread(a, 0, N) | _spread(b, 1, N)
            # for a beta excitation the roles of the strings swap and the other string's
            # orbitals at the excitation's own indices count as "below": pp(other) ^ other
            PP = _pp(own) ^ (_pp(other) if spin == 0 else (_pp(other) ^ other))
            occ = [p for p in range(N) if (own >> p) & 1]
            emp = [p for p in range(N) if not (own >> p) & 1]
            for p in occ:
                for q in emp:
                    ref = _par(x & _between(2 * p + spin, 2 * q + spin))
                    bad += ref != (_par(PP & ((1 << p) | (1 << q))) ^ (p < q))
            for p1, p2 in itertools.combinations(occ, 2):
                for q1, q2 in itertools.combinations(emp, 2):
                    i, j, aa, bb = (2 * t + spin for t in (p1, p2, q1, q2))
                    x1 = x ^ (1 << i) ^ (1 << bb)
                    ref = 1 ^ _par(x & _between(i, bb)) ^ _par(x1 & _between(j, aa))
                    s0 = (p1 < q2) ^ (q2 < p2) ^ (p1 < q1) ^ (p2 < q1)
                    bad += ref != (_par(PP & ((1 << p1) | (1 << p2) | (1 << q1) | (1 << q2))) ^ s0)
    assert bad == 0


def test_blocked_basis_same_spin_signs():
    """The same-spin products (expectation variant 4) work in the string-blocked basis:
    with phi(a, b) = (-1)^popc(a & pp(b)) and C~ = phi C, the sign of a same-spin
    excitation between x = (a, b) and x' is phi(x) phi(x') times its interleaved
    Jordan-Wigner sign, and must depend on that spin's string alone:
        single  popc(pp(own) & {p, q}) + [p < q]
        double  popc(pp(own) & {p1, p2, q1, q2}) + the orbital-order terms.
    Checked against the between-mask definition for every excitation of random strings."""
    N = 7
    rng = np.random.default_rng(9)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, 1 << N, size=(300, 2))]

    def phi(a, b):
        return _par(a & _pp(b))

    for a, b in pairs:
        for spin in (0, 1):
            own = a if spin == 0 else b
            x = _spread(a, 0, N) | _spread(b, 1, N)
            occ = [p for p in range(N) if (own >> p) & 1]
            emp = [p for p in range(N) if not (own >> p) & 1]
            for p in occ:
                for q in emp:
                    m = (1 << p) | (1 << q)
                    jw = _par(x & _between(2 * p + spin, 2 * q + spin))
                    a2, b2 = (a ^ m, b) if spin == 0 else (a, b ^ m)
                    blocked = jw ^ phi(a, b) ^ phi(a2, b2)
                    assert blocked == _par(_pp(own) & m) ^ int(p < q)
            for p1, p2 in itertools.combinations(occ, 2):
                for q1, q2 in itertools.combinations(emp, 2):
                    m = (1 << p1) | (1 << p2) | (1 << q1) | (1 << q2)
                    i, j, aa, bb = (2 * o + spin for o in (p1, p2, q1, q2))
                    xm = x ^ (1 << i) ^ (1 << bb)  # after a+_q2 a_p1
                    jw = 1 ^ _par(x & _between(i, bb)) ^ _par(xm & _between(j, aa))
                    a2, b2 = (a ^ m, b) if spin == 0 else (a, b ^ m)
                    blocked = jw ^ phi(a, b) ^ phi(a2, b2)
                    order = int(p1 < q2) ^ int(q2 < p2) ^ int(p1 < q1) ^ int(p2 < q1)
                    assert blocked == _par(_pp(own) & m) ^ order


def _jw_ops(n):
    """Annihilation operators a_j (j = 0..n-1, qubit j = bit j of the basis index) by the
    Jordan-Wigner construction: Z on every qubit below j, sigma^- on qubit j."""
    import scipy.sparse as sp
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    I2 = sp.identity(2, format="csr")
    lower = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |0><1|: removes an occupation
    ops = []
    for j in range(n):
        m = sp.identity(1, format="csr")
        for k in range(n - 1, -1, -1):  # kron order: qubit n-1 first, so qubit k is bit k
            m = sp.kron(m, lower if k == j else (Z if k < j else I2), format="csr")
        ops.append(m)
    return ops


def _sym_eri(N, rng):
    g = rng.normal(size=(N, N, N, N))
    e = np.zeros_like(g)
    for perm in ((0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
                 (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)):
        e += g.transpose(perm)
    return e / 8.0


@pytest.mark.parametrize("N,na,nb,seed", [(5, 2, 3, 21), (4, 4, 1, 22), (5, 3, 2, 23)])
def test_blocked_basis_alpha_beta_products(N, na, nb, seed):
    """Expectation variant 5 takes the alpha-beta part of H = sum (pq|rs) E^a_pq E^b_rs as
    products in the string-blocked basis: with X = phi C,
        H[b'][j][a] = sum_kappa A_b'[a][kappa] B[j][kappa]
    over kappa = the orbitals p (A = X(a, b') if p in a) and the unordered pairs p < q
    (A = s_a X(a ^ {p, q}, b') if exactly one of p, q is in a, s_a the parity of a's bits
    between them), columns j = b''s excitations (s in b' -> r not in b', B = (qp|sr)) and an
    own column (B = sum_{l in b'} (qp|ll), 0 on the diagonal); then
        sigma~_ab(a, b) = sum_{r in b, s not in b} (-1)^popc(b & between(r, s)) H[b ^ {r, s}][col][a]
                          + H[b][own][a],
    sigma_ab = phi sigma~_ab + sum_{p in a, l in b} (pp|ll) C.  Checked against the operator
    built from Jordan-Wigner fermion operators (interleaved spin-orbitals 2p + spin)."""
    pytest.importorskip("scipy")
    import math
    rng = np.random.default_rng(seed)
    n = 2 * N
    eri = _sym_eri(N, rng)
    strs_a = [s for s in range(1 << N) if bin(s).count("1") == na]
    strs_b = [s for s in range(1 << N) if bin(s).count("1") == nb]
    ra = {s: i for i, s in enumerate(strs_a)}
    rb = {s: i for i, s in enumerate(strs_b)}
    Da, Db = len(strs_a), len(strs_b)
    assert (Da, Db) == (math.comb(N, na), math.comb(N, nb))
    C = rng.normal(size=(Db, Da)) + 1j * rng.normal(size=(Db, Da))
    # reference: the operator on the full 2^n space
    psi = np.zeros(1 << n, dtype=complex)
    for ib, b in enumerate(strs_b):
        for ia, a in enumerate(strs_a):
            psi[_spread(a, 0, N) | _spread(b, 1, N)] = C[ib, ia]
    ann = _jw_ops(n)
    cre = [m.T.tocsr() for m in ann]
    ref = np.zeros_like(psi)
    for r in range(N):
        for s in range(N):
            eb = cre[2 * r + 1] @ (ann[2 * s + 1] @ psi)  # E^b_rs psi
            if not np.any(eb):
                continue
            for p in range(N):
                for q in range(N):
                    ref += eri[p, q, r, s] * (cre[2 * p] @ (ann[2 * q] @ eb))
    # the decomposition
    phi = np.array([[_par(a & _pp(b)) for a in strs_a] for b in strs_b])
    X = np.where(phi == 1, -C, C)
    kap = [(p, p) for p in range(N)] + [(p, q) for p in range(N) for q in range(p + 1, N)]
    assert len(kap) == N * (N + 1) // 2
    ncols = nb * (N - nb) + 1
    H = np.zeros((Db, ncols, Da), dtype=complex)
    for jb, bp in enumerate(strs_b):
        occ = [o for o in range(N) if (bp >> o) & 1]
        emp = [o for o in range(N) if not (bp >> o) & 1]
        B = np.zeros((ncols, len(kap)))
        for k, (p, q) in enumerate(kap):
            for i, s in enumerate(occ):
                for jj, r in enumerate(emp):
                    B[i * len(emp) + jj, k] = eri[q, p, s, r]
            if p != q:
                B[ncols - 1, k] = sum(eri[q, p, l, l] for l in occ)
        A = np.zeros((Da, len(kap)), dtype=complex)
        for ia, a in enumerate(strs_a):
            for k, (p, q) in enumerate(kap):
                if p == q:
                    if (a >> p) & 1:
                        A[ia, k] = X[jb, ia]
                elif ((a >> p) ^ (a >> q)) & 1:
                    sgn = -1.0 if _par(a & _between(p, q)) else 1.0
                    A[ia, k] = sgn * X[jb, ra[a ^ (1 << p) ^ (1 << q)]]
        H[jb] = (A @ B.T).T
    out = np.zeros_like(psi)
    for ib, b in enumerate(strs_b):
        occ = [o for o in range(N) if (b >> o) & 1]
        emp = [o for o in range(N) if not (b >> o) & 1]
        st = H[ib, ncols - 1].copy()
        for r in occ:
            for s in emp:
                bp = b ^ (1 << r) ^ (1 << s)
                col = bin(bp & ((1 << s) - 1)).count("1") * (N - nb) + \
                    bin(~bp & ((1 << N) - 1) & ((1 << r) - 1)).count("1")
                st += (-1.0 if _par(b & _between(r, s)) else 1.0) * H[rb[bp], col]
        for ia, a in enumerate(strs_a):
            d = sum(eri[p, p, l, l] for p in range(N) if (a >> p) & 1 for l in occ)
            val = (-st[ia] if phi[ib, ia] else st[ia]) + d * C[ib, ia]
            out[_spread(a, 0, N) | _spread(b, 1, N)] = val
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("N,na,nb,seed", [(5, 2, 3, 31), (4, 1, 3, 32), (5, 3, 3, 33)])
def test_blocked_basis_same_spin_products(N, na, nb, seed):
    """Expectation variants 4 and 5 take the same-spin part of H as Ma (x) 1 + 1 (x) Mb in the
    string-blocked basis (X = phi C; sigma~ = Ma X + X Mb^T), with
        Ma[a][a - p + q] = s (h_qp + sum_{o in a} ((qp|oo) - (qo|op)))        singles p -> q,
        Ma[a][a - p1 - p2 + q1 + q2] = s ((q1p1|q2p2) - (q1p2|q2p1))          doubles,
        dA[a] = sum_{k in a} h_kk + sum_{k < l in a} ((kk|ll) - (kl|lk))      on the diagonal,
    s = (-1)^(popc(pp(a) & m) + the orbital-order terms) from the string alone; Mb, dB
    likewise.  Checked against the same-spin part of H built from Jordan-Wigner fermion
    matrices: sum h_pq a+_p a_q + 1/2 sum (pq|rs) a+_p a+_r a_s a_q over spin-orbitals of
    one spin, both spins."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(seed)
    n = 2 * N
    eri = _sym_eri(N, rng)
    h = rng.normal(size=(N, N))
    h = 0.5 * (h + h.T)
    strs_a = [s for s in range(1 << N) if bin(s).count("1") == na]
    strs_b = [s for s in range(1 << N) if bin(s).count("1") == nb]
    Da, Db = len(strs_a), len(strs_b)
    C = rng.normal(size=(Db, Da)) + 1j * rng.normal(size=(Db, Da))
    psi = np.zeros(1 << n, dtype=complex)
    for ib, b in enumerate(strs_b):
        for ia, a in enumerate(strs_a):
            psi[_spread(a, 0, N) | _spread(b, 1, N)] = C[ib, ia]
    ann = _jw_ops(n)
    cre = [m.T.tocsr() for m in ann]
    ref = np.zeros_like(psi)
    for spin in (0, 1):
        for p in range(N):
            for q in range(N):
                ref += h[p, q] * (cre[2 * p + spin] @ (ann[2 * q + spin] @ psi))
        for q in range(N):
            for s in range(N):
                t = ann[2 * s + spin] @ (ann[2 * q + spin] @ psi)
                if not np.any(t):
                    continue
                for p in range(N):
                    for r in range(N):
                        ref += 0.5 * eri[p, q, r, s] * (cre[2 * p + spin] @ (cre[2 * r + spin] @ t))

    def order(p1, p2, q1, q2):
        return int(p1 < q2) ^ int(q2 < p2) ^ int(p1 < q1) ^ int(p2 < q1)

    def one_spin(strs):
        rank = {s: i for i, s in enumerate(strs)}
        M = np.zeros((len(strs), len(strs)))
        for i, a in enumerate(strs):
            occ = [o for o in range(N) if (a >> o) & 1]
            emp = [o for o in range(N) if not (a >> o) & 1]
            M[i, i] = sum(h[k, k] for k in occ) + sum(eri[k, k, l, l] - eri[k, l, l, k]
                                                    for k, l in itertools.combinations(occ, 2))
            for p in occ:
                for q in emp:
                    m = (1 << p) | (1 << q)
                    v = h[q, p] + sum(eri[q, p, o, o] - eri[q, o, o, p] for o in occ)
                    sg = _par(_pp(a) & m) ^ int(p < q)
                    M[i, rank[a ^ m]] = -v if sg else v
            for p1, p2 in itertools.combinations(occ, 2):
                for q1, q2 in itertools.combinations(emp, 2):
                    m = (1 << p1) | (1 << p2) | (1 << q1) | (1 << q2)
                    v = eri[q1, p1, q2, p2] - eri[q1, p2, q2, p1]
                    sg = _par(_pp(a) & m) ^ order(p1, p2, q1, q2)
                    M[i, rank[a ^ m]] = -v if sg else v
        return M

    Ma, Mb = one_spin(strs_a), one_spin(strs_b)
    phi = np.array([[_par(a & _pp(b)) for a in strs_a] for b in strs_b])
    X = np.where(phi == 1, -C, C)
    G = X @ Ma.T + Mb @ X  # rows b, columns a: sum_a' Ma[a][a'] X[b][a'] + sum_b' Mb[b][b'] X[b'][a]
    out = np.zeros_like(psi)
    for ib, b in enumerate(strs_b):
        for ia, a in enumerate(strs_a):
            out[_spread(a, 0, N) | _spread(b, 1, N)] = -G[ib, ia] if phi[ib, ia] else G[ib, ia]
    assert np.max(np.abs(out - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
