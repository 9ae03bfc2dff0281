"""Pins for the CPU oracle: facts fixed by the mathematics or printed in the paper.

Each test ties the oracle to something other than itself: route B (dense
Kronecker-product matrices + scipy), textbook closed forms (Slater-Condon
diagonal and one-gate curves, non-interacting fermions, first-quantised
two-electron problems), invariants (orbital-rotation invariance, norm, traces)
and Table IV.  A plausible slip anywhere in the oracle -- a dropped exchange
term, a wrong Jordan-Wigner sign, a transposed integral index -- fails at least
one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import route_a as A
from oracle import route_b as B
from paper_2405_11567_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(n, ne, seed, ansatz="uccsd"):
    return inputs.make_problem(n, ne, ansatz, seed)


def _sector_matrix(sec, h, eri, e_nuc):
    """Route A's Hamiltonian restricted to the sector, column by column."""
    D = sec.D
    M = np.zeros((D, D), dtype=np.complex128)
    for c in range(D):
        e = np.zeros(D, dtype=np.complex128)
        e[c] = 1.0
        M[:, c] = A.hamiltonian_apply(sec, h, eri, e_nuc, e)
    return M


def _spin(j):
    return j % 2


# ---------------------------------------------------------------- route A vs B

@pytest.mark.parametrize("n,ne,seed", [(8, 2, 1001), (8, 4, 11), (10, 4, 12)])
def test_route_a_matches_route_b(n, ne, seed):
    p = _problem(n, ne, seed)
    a = B.annihilators(n)
    H = B.hamiltonian(n, p["h"], p["eri"], p["e_nuc"], a)
    sec = oracle.Sector(n, ne // 2, ne // 2)
    ops, theta = p["ops"], p["theta"] * 6.0          # larger angles: more mixing
    psiA = A.apply_ansatz(sec, ops, theta, A.hf_state(sec, p["occ"]))
    psiB = B.apply_ansatz(ops, theta, B.basis_state(n, p["occ"]), a)
    np.testing.assert_allclose(psiA, psiB[sec.dets.astype(np.int64)], atol=1e-13)
    # nothing outside the sector
    outside = np.ones(2 ** n, bool)
    outside[sec.dets.astype(np.int64)] = False
    assert np.max(np.abs(psiB[outside])) < 1e-14
    EA, gA = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], ops, theta, A.hf_state(sec, p["occ"]))
    EB = B.energy(H, psiB)
    gB = B.gradient(H, ops, theta, B.basis_state(n, p["occ"]), a)
    assert abs(EA - EB) < 1e-12
    np.testing.assert_allclose(gA, gB, atol=1e-11)
    np.testing.assert_allclose(A.rdm1(sec, psiA), B.rdm1(psiB, a, n), atol=1e-13)


def test_route_a_matches_route_b_complex_start_open_shell():
    """Complex amplitudes and N_alpha != N_beta exercise every conj() and both spins."""
    n, na, nb = 10, 3, 1
    p = _problem(n, 4, 21)
    rng = np.random.default_rng(5)
    dense0 = inputs.random_sector_state(n, na, nb, rng)
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    # operators valid in this sector: take spin-conserving ones from a pool on (na+nb) electrons,
    # keeping only those that connect some determinants here
    pool = inputs.uccsd_pool(n, 4)
    ops = pool[rng.choice(len(pool), size=12, replace=False)]
    theta = rng.normal(0, 0.4, size=len(ops))
    a = B.annihilators(n)
    H = B.hamiltonian(n, p["h"], p["eri"], p["e_nuc"], a)
    psiB = B.apply_ansatz(ops, theta, dense0, a)
    psiA = A.apply_ansatz(sec, ops, theta, psi0)
    np.testing.assert_allclose(psiA, psiB[sec.dets.astype(np.int64)], atol=1e-13)
    EA, gA = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], ops, theta, psi0)
    assert abs(EA - B.energy(H, psiB)) < 1e-12
    np.testing.assert_allclose(gA, B.gradient(H, ops, theta, dense0, a), atol=1e-11)
    rA = A.rdm1(sec, psiA)
    np.testing.assert_allclose(rA, B.rdm1(psiB, a, n), atol=1e-13)
    assert np.max(np.abs(rA.imag)) > 1e-3          # the complex part is really exercised


@pytest.mark.parametrize("n", [8, 10])
def test_jw_signs_literal_vs_matrix(n):
    """Route A's sequential sign rule equals the Kronecker-product matrix element, for every x."""
    a = B.annihilators(n)
    ne = 2 if n == 8 else 4
    pool = inputs.uccsd_pool(n, ne)
    # also operators whose occupied / virtual indices interleave in position
    extra = np.array([(2, 1, 6, 2, 5), (2, 0, 5, 2, 3), (1, 5, -1, 1, -1), (2, 2, 3, 0, 7)], np.int32)
    for op in np.vstack([pool, extra]):
        T = B.excitation_T(op, a).tocsc()
        for x in range(2 ** n):
            s, y = A.exc_apply(op, x)
            col = T[:, x].toarray().ravel()
            nz = np.nonzero(np.abs(col) > 0.5)[0]
            if s == 0:
                assert len(nz) == 0
            else:
                assert list(nz) == [y] and col[y].real == s


# ---------------------------------------------------------------- closed forms

def _hf_energy_closed_form(h, eri, e_nuc, occ):
    """E_HF = E_nuc + sum_i h_ii + 1/2 sum_{i != j} [(ii|jj) - delta_spin (ij|ji)] (Slater-Condon)."""
    E = e_nuc
    for i in occ:
        E += h[i // 2, i // 2]
    for i in occ:
        for j in occ:
            if i == j:
                continue
            E += 0.5 * eri[i // 2, i // 2, j // 2, j // 2]
            if _spin(i) == _spin(j):
                E -= 0.5 * eri[i // 2, j // 2, j // 2, i // 2]
    return E


@pytest.mark.parametrize("n,na,nb,seed", [(8, 1, 1, 1), (10, 2, 2, 2), (12, 3, 1, 3), (12, 2, 2, 4)])
def test_reference_energy_closed_form(n, na, nb, seed):
    p = _problem(n, 2, seed)
    sec = oracle.Sector(n, na, nb)
    rng = np.random.default_rng(seed)
    for _ in range(4):   # several determinants of the sector, not only aufbau
        x = int(sec.dets[rng.integers(sec.D)])
        occ = [j for j in range(n) if (x >> j) & 1]
        psi = np.zeros(sec.D, complex)
        psi[sec.index(x)] = 1.0
        E = A.energy(sec, p["h"], p["eri"], p["e_nuc"], psi)
        assert abs(E - _hf_energy_closed_form(p["h"], p["eri"], p["e_nuc"], occ)) < 1e-12


def _coupling_from_reference(h, eri, occ, op):
    """<x'|H|x> / <x'|T|x> for x = reference, x' = T x: the sign-free Slater-Condon coefficient."""
    kind, i, j, a, b = [int(v) for v in op]
    g = lambda P, Q, R, S: (eri[P // 2, Q // 2, R // 2, S // 2]  # noqa: E731
                            if _spin(P) == _spin(Q) and _spin(R) == _spin(S) else 0.0)
    if kind == 1:
        v = h[a // 2, i // 2] if _spin(a) == _spin(i) else 0.0
        for k in occ:
            if k != i:
                v += g(a, i, k, k) - g(a, k, k, i)
        return v
    return g(a, i, b, j) - g(a, j, b, i)


@pytest.mark.parametrize("seed", [31, 32])
def test_one_gate_curve(seed):
    """One excitation from the reference: E(t) = c^2 E_ref + s^2 E_exc + 2 s c V (sign-free)."""
    n, ne = 10, 4
    p = _problem(n, ne, seed)
    sec = oracle.Sector(n, 2, 2)
    psi0 = A.hf_state(sec, p["occ"])
    for op in p["ops"][::7]:
        s, y = A.exc_apply(op, sum(1 << j for j in p["occ"]))
        assert s != 0
        occ_exc = [j for j in range(n) if (y >> j) & 1]
        E_ref = _hf_energy_closed_form(p["h"], p["eri"], p["e_nuc"], p["occ"])
        E_exc = _hf_energy_closed_form(p["h"], p["eri"], p["e_nuc"], occ_exc)
        V = _coupling_from_reference(p["h"], p["eri"], p["occ"], op)
        for t in (0.3, -0.7, 1.1):
            E = A.energy(sec, p["h"], p["eri"], p["e_nuc"], A.rotate(sec, op, t, psi0))
            ref = np.cos(t) ** 2 * E_ref + np.sin(t) ** 2 * E_exc + 2 * np.sin(t) * np.cos(t) * V
            assert abs(E - ref) < 1e-12
        # gradient at theta = 0 is 2 V for the one-operator ansatz
        _, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], op[None, :], [0.0], psi0)
        assert abs(g[0] - 2 * V) < 1e-12


def test_gradient_at_zero_is_twice_the_coupling():
    p = _problem(10, 4, 41)
    sec = oracle.Sector(10, 2, 2)
    psi0 = A.hf_state(sec, p["occ"])
    _, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], np.zeros(len(p["ops"])), psi0)
    ref = [2 * _coupling_from_reference(p["h"], p["eri"], p["occ"], op) for op in p["ops"]]
    np.testing.assert_allclose(g, ref, atol=1e-12)


def test_one_body_ground_state_is_aufbau_of_h():
    """eri = 0: non-interacting fermions, E_0 = E_nuc + lowest na + lowest nb eigenvalues of h."""
    n, na, nb = 10, 3, 2
    p = _problem(n, 2, 51)
    eri0 = np.zeros_like(p["eri"])
    sec = oracle.Sector(n, na, nb)
    M = _sector_matrix(sec, p["h"], eri0, p["e_nuc"])
    e = np.linalg.eigvalsh(p["h"])
    assert abs(np.linalg.eigvalsh(M)[0] - (p["e_nuc"] + e[:na].sum() + e[:nb].sum())) < 1e-12


def test_two_electron_singlet_sector_first_quantised():
    """One alpha + one beta electron: H_(pq),(rs) = h_pr d_qs + d_pr h_qs + (pr|qs) on |p_alpha q_beta>."""
    n = 10
    N = n // 2
    p = _problem(n, 2, 61)
    sec = oracle.Sector(n, 1, 1)
    M = _sector_matrix(sec, p["h"], p["eri"], p["e_nuc"])
    h, eri = p["h"], p["eri"]
    F = np.zeros((N * N, N * N))
    I = np.eye(N)
    for (pp, q), (r, s) in itertools.product(itertools.product(range(N), repeat=2), repeat=2):
        F[pp * N + q, r * N + s] = h[pp, r] * I[q, s] + I[pp, r] * h[q, s] + eri[pp, r, q, s]
    F += p["e_nuc"] * np.eye(N * N)
    np.testing.assert_allclose(np.linalg.eigvalsh(M), np.linalg.eigvalsh(F), atol=1e-11)


def test_two_same_spin_electrons_first_quantised():
    """Two alpha electrons: antisymmetrised pairs p<q, <pq|H|rs> with direct minus exchange."""
    n = 12
    N = n // 2
    p = _problem(n, 2, 71)
    sec = oracle.Sector(n, 2, 0)
    M = _sector_matrix(sec, p["h"], p["eri"], p["e_nuc"])
    h, eri = p["h"], p["eri"]
    pairs = [(a, b) for a in range(N) for b in range(a + 1, N)]
    F = np.zeros((len(pairs), len(pairs)))
    d = np.eye(N)
    for u, (pp, q) in enumerate(pairs):
        for v, (r, s) in enumerate(pairs):
            F[u, v] = (h[pp, r] * d[q, s] + h[q, s] * d[pp, r] - h[pp, s] * d[q, r] - h[q, r] * d[pp, s]
                       + eri[pp, r, q, s] - eri[pp, s, q, r])
    F += p["e_nuc"] * np.eye(len(pairs))
    np.testing.assert_allclose(np.linalg.eigvalsh(M), np.linalg.eigvalsh(F), atol=1e-11)


def test_orbital_rotation_invariance_of_spectrum():
    """A real orthogonal change of orbitals leaves the sector spectrum unchanged."""
    n, na, nb = 10, 2, 2
    N = n // 2
    p = _problem(n, 4, 81)
    rng = np.random.default_rng(3)
    C, _ = np.linalg.qr(rng.normal(size=(N, N)))
    h2 = C.T @ p["h"] @ C
    eri2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", p["eri"], C, C, C, C)
    sec = oracle.Sector(n, na, nb)
    e1 = np.linalg.eigvalsh(_sector_matrix(sec, p["h"], p["eri"], p["e_nuc"]))
    e2 = np.linalg.eigvalsh(_sector_matrix(sec, h2, eri2, p["e_nuc"]))
    np.testing.assert_allclose(e1, e2, atol=1e-11)


def test_hamiltonian_real_symmetric_and_matches_route_b_block():
    n = 8
    p = _problem(n, 4, 91)
    sec = oracle.Sector(n, 2, 2)
    M = _sector_matrix(sec, p["h"], p["eri"], p["e_nuc"])
    assert np.max(np.abs(M - M.T)) < 1e-13 and np.max(np.abs(M.imag)) == 0.0
    H = B.hamiltonian(n, p["h"], p["eri"], p["e_nuc"])
    s = sec.dets.astype(np.int64)
    np.testing.assert_allclose(M, H[s][:, s].toarray(), atol=1e-13)


# ---------------------------------------------------------------- gradient / variational

def test_gradient_central_differences():
    p = _problem(10, 4, 101, ansatz=20)
    sec = oracle.Sector(10, 2, 2)
    psi0 = A.hf_state(sec, p["occ"])
    theta = p["theta"] * 5
    _, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    hstep = 1e-5
    for k in range(0, len(theta), 3):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += hstep
        tm[k] -= hstep
        Ep = A.energy(sec, p["h"], p["eri"], p["e_nuc"], A.apply_ansatz(sec, p["ops"], tp, psi0))
        Em = A.energy(sec, p["h"], p["eri"], p["e_nuc"], A.apply_ansatz(sec, p["ops"], tm, psi0))
        assert abs((Ep - Em) / (2 * hstep) - g[k]) < 1e-8


def test_variational_bound():
    n = 10
    p = _problem(n, 4, 111)
    E0 = B.sector_spectrum(B.hamiltonian(n, p["h"], p["eri"], p["e_nuc"]), n, 2, 2)[0]
    sec = oracle.Sector(n, 2, 2)
    rng = np.random.default_rng(0)
    for _ in range(5):
        th = rng.normal(0, 0.5, size=len(p["ops"]))
        E = A.energy(sec, p["h"], p["eri"], p["e_nuc"], A.apply_ansatz(sec, p["ops"], th, A.hf_state(sec, p["occ"])))
        assert E >= E0 - 1e-12


# ---------------------------------------------------------------- state and RDM invariants

def test_norm_preserved_and_real():
    p = _problem(12, 4, 121)
    sec = oracle.Sector(12, 2, 2)
    psi = A.apply_ansatz(sec, p["ops"], p["theta"] * 10, A.hf_state(sec, p["occ"]))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13
    assert np.max(np.abs(psi.imag)) == 0.0


def test_rdm1_invariants():
    n, na, nb = 12, 3, 2
    p = _problem(n, 4, 131)
    sec = oracle.Sector(n, na, nb)
    rng = np.random.default_rng(9)
    psi0 = inputs.random_sector_state(n, na, nb, rng)[sec.dets.astype(np.int64)]
    psi = A.apply_ansatz(sec, p["ops"], p["theta"] * 8, psi0)
    g = A.rdm1(sec, psi)
    assert abs(np.trace(g[0]).real - na) < 1e-12 and abs(np.trace(g[1]).real - nb) < 1e-12
    for s in range(2):
        assert np.max(np.abs(g[s] - g[s].conj().T)) < 1e-13
        ev = np.linalg.eigvalsh(g[s])
        assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12
    # a single determinant: diagonal occupation numbers
    x = int(sec.dets[17])
    e = np.zeros(sec.D, complex)
    e[17] = 1.0
    gd = A.rdm1(sec, e)
    for s in range(2):
        np.testing.assert_allclose(gd[s], np.diag([(x >> (2 * q + s)) & 1 for q in range(n // 2)]), atol=0)


def test_one_body_energy_equals_contraction_with_rdm1():
    """eri = 0: E = E_nuc + sum_sigma sum_pq h_pq n_pq,sigma (cross-pins H with the RDM)."""
    n = 12
    p = _problem(n, 4, 141)
    sec = oracle.Sector(n, 2, 2)
    psi = A.apply_ansatz(sec, p["ops"], p["theta"] * 8, A.hf_state(sec, p["occ"]))
    eri0 = np.zeros_like(p["eri"])
    E = A.energy(sec, p["h"], eri0, p["e_nuc"], psi)
    g = A.rdm1(sec, psi)
    assert abs(E - (p["e_nuc"] + np.einsum("pq,spq->", p["h"], g).real)) < 1e-12


# ---------------------------------------------------------------- Table IV

def test_table_iv_cnot_formula_reading():
    """CNOT counts of Table IV fit 3 N_s + 13 N_d (QEB) and 2 N_s + 6 N_d (qubit pool).

    Every row admits one integer split N_s + N_d = N_op that reproduces both counts,
    except Be/cc-pVDZ, whose two counts imply different splits (a misprint).
    """
    bad = []
    for line in open(os.path.join(GOLDEN, "table4_cnot.txt")):
        if line.startswith("#") or not line.strip():
            continue
        sysname, basis, nq, qeb, qub, nop, nit = line.split()
        qeb, qub, nop = int(qeb), int(qub), int(nop)
        fits = [(ns, nop - ns) for ns in range(nop + 1)
                if 3 * ns + 13 * (nop - ns) == qeb and 2 * ns + 6 * (nop - ns) == qub]
        if fits:
            ns, nd = fits[0]
            ops = np.array([(1, 0, -1, 2, -1)] * ns + [(2, 0, 1, 2, 3)] * nd, np.int32).reshape(-1, 5)
            assert A.cnot_counts(ops) == (qeb, qub)
        else:
            bad.append((sysname, basis))
    assert bad == [("Be", "cc-pVDZ")]


# ---------------------------------------------------------------- qubit excitations (QEB pool)

def test_qubit_excitations_route_a_matches_route_b():
    n = 10
    p = _problem(n, 4, 151)
    pool = inputs.qeb_pool(n, 4)
    rng = np.random.default_rng(8)
    ops = pool[rng.choice(len(pool), size=16, replace=False)]
    theta = rng.normal(0, 0.4, size=len(ops))
    a = B.annihilators(n)
    sq = B.qubit_lowering(n)
    H = B.hamiltonian(n, p["h"], p["eri"], p["e_nuc"], a)
    sec = oracle.Sector(n, 2, 2)
    psiA = A.apply_ansatz(sec, ops, theta, A.hf_state(sec, p["occ"]))
    psiB = B.apply_ansatz(ops, theta, B.basis_state(n, p["occ"]), a, sq)
    np.testing.assert_allclose(psiA, psiB[sec.dets.astype(np.int64)], atol=1e-13)
    EA, gA = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], ops, theta, A.hf_state(sec, p["occ"]))
    assert abs(EA - B.energy(H, psiB)) < 1e-12
    np.testing.assert_allclose(gA, B.gradient(H, ops, theta, B.basis_state(n, p["occ"]), a, sq), atol=1e-11)


def test_qubit_excitation_is_the_fermionic_one_up_to_the_string_sign():
    """Same partner determinant; the fermionic sign is the JW parity, the qubit one is +1."""
    n = 10
    for op in inputs.uccsd_pool(n, 4):
        q = op.copy()
        q[0] += 2
        for x in range(1 << n):
            sf, yf = A.exc_apply(op, x)
            sq, yq = A.exc_apply(q, x)
            assert (sf == 0) == (sq == 0)
            if sf:
                assert yf == yq and sq == 1
