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
