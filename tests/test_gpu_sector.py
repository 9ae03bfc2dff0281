"""GPU parity for sector storage (sv_create_sector): the state held as only its
(N_alpha, N_beta) sector, C[rank(beta string)][rank(alpha string)], against the
CPU oracle, with the tolerances of the dense path.  Integer work (signs, partner
ranks, which amplitudes are exactly zero) is compared bit for bit."""
import math

import numpy as np
import pytest

import oracle
from oracle import route_a as A
from oracle import route_b as B
from paper_2405_11567_gb300 import inputs, sv
from paper_2405_11567_gb300.adapt import adapt_vqe

pytestmark = pytest.mark.gpu

TOL = {"c128": dict(E=1e-10, g=1e-9, amp=1e-12, rdm=1e-12), "c64": dict(E=1e-5, g=1e-5, amp=2e-6, rdm=2e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


def _state(n, na, nb, dtype):
    return sv.StateVector(n, dtype, sector=(na, nb))


def _outside(n, na, nb):
    x = np.arange(1 << n, dtype=np.int64)
    ca = sum(((x >> j) & 1) for j in range(0, n, 2))
    cb = sum(((x >> j) & 1) for j in range(1, n, 2))
    return (ca != na) | (cb != nb)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,ne,seed", [(8, 2, 1001), (10, 4, 7), (12, 4, 8), (14, 6, 9)])
def test_ansatz_state_matches_oracle(n, ne, seed, dtype):
    p = inputs.make_problem(n, ne, "uccsd", seed)
    theta = p["theta"] * 8
    sec = oracle.Sector(n, p["na"], p["nb"])
    ref = A.apply_ansatz(sec, p["ops"], theta, A.hf_state(sec, p["occ"]))
    st = _state(n, p["na"], p["nb"], dtype)
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], theta)
    got = st.state()
    assert np.max(np.abs(got[sec.dets.astype(np.int64)] - ref)) <= TOL[dtype]["amp"]
    assert np.count_nonzero(got[_outside(n, p["na"], p["nb"])]) == 0
    assert np.count_nonzero(got.imag) == 0


def test_jordan_wigner_signs_bit_exact():
    """A rotation by pi/2 sends a basis state to T|x> with amplitude exactly +-1: sign and partner
    (through the string ranks) must equal the oracle's literal operator application."""
    n = 10
    ops = np.vstack([inputs.uccsd_pool(n, 4), inputs.qeb_pool(n, 4)[::3],
                     np.array([(2, 1, 6, 2, 5), (2, 0, 5, 2, 3), (1, 5, -1, 1, -1), (2, 2, 3, 0, 7),
                               (1, 8, -1, 2, -1)], np.int32)])
    st = _state(n, 2, 2, "c128")
    sec = oracle.Sector(n, 2, 2)
    rng = np.random.default_rng(0)
    for op in ops:
        froms = [int(x) for x in sec.dets if A.exc_apply(op, int(x))[0] != 0]
        for x in rng.choice(froms, size=min(6, len(froms)), replace=False):
            s, y = A.exc_apply(op, int(x))
            v = np.zeros(1 << n, np.complex128)
            v[int(x)] = 1.0
            st.prepare_state(v, 2, 2)
            st.apply_ansatz(op[None, :], [np.pi / 2])
            got = st.state()
            assert got[y].real == float(s) and got[y].imag == 0.0
            assert abs(got[int(x)]) < 1e-15
            assert np.count_nonzero(np.abs(got) > 1e-15) == 1


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("cid", [1, 2])
def test_config_energy_grad(cid, dtype):
    p = inputs.config_problem(cid)
    sec = oracle.Sector(p["n_qubits"], p["na"], p["nb"])
    psi0 = A.hf_state(sec, p["occ"])
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(p["n_qubits"], p["na"], p["nb"], dtype)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], p["theta"])
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    assert abs(st.energy(ham) - Eref) <= TOL[dtype]["E"]          # the handle holds psi(theta)
    psi = A.apply_ansatz(sec, p["ops"], p["theta"], psi0)
    assert np.max(np.abs(st.amplitudes(sec.dets.astype(np.uint64)) - psi)) <= TOL[dtype]["amp"] * 10


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_config3_energy_grad_rdm(dtype, config3_oracle):
    p, Eref, gref, rdm_ref = config3_oracle
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(p["n_qubits"], p["na"], p["nb"], dtype)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], p["theta"])
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    assert np.max(np.abs(st.rdm1() - rdm_ref)) <= TOL[dtype]["rdm"]


@pytest.fixture(scope="module")
def config3_oracle():
    p = inputs.config_problem(3)
    sec = oracle.Sector(p["n_qubits"], p["na"], p["nb"])
    psi0 = A.hf_state(sec, p["occ"])
    E, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], psi0)
    rdm = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], p["theta"], psi0))
    return p, E, g, rdm


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_complex_start_open_shell(dtype):
    """Complex multi-determinant start, N_alpha != N_beta: every conj() of the path."""
    n, na, nb = 12, 3, 2
    p = inputs.make_problem(n, 4, 40, seed=55)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(3))
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 6
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(n, na, nb, dtype)
    st.prepare_state(dense0.astype(np.complex64 if dtype == "c64" else np.complex128), na, nb)
    E, g = st.energy_grad(ham, p["ops"], theta)
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    rdm_ref = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], theta, psi0))
    assert np.max(np.abs(st.rdm1() - rdm_ref)) <= TOL[dtype]["rdm"]


@pytest.mark.parametrize("variant", [0, 2, 3])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_rdm1_matches_oracle(dtype, variant):
    p = inputs.make_problem(14, 6, 60, seed=66)
    sec = oracle.Sector(14, 3, 3)
    psi = A.apply_ansatz(sec, p["ops"], p["theta"] * 5, A.hf_state(sec, p["occ"]))
    st = _state(14, 3, 3, dtype)
    st.set_option(sv.SV_OPT_RDM_VARIANT, variant)
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"] * 5)
    assert np.max(np.abs(st.rdm1() - A.rdm1(sec, psi))) <= TOL[dtype]["rdm"]


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-9), ("c64", 1e-5)])
def test_pool_gradients_match_oracle(dtype, tol, variant):
    n = 14
    p = inputs.make_problem(n, 6, 30, seed=202)
    pool = np.vstack([inputs.uccsd_pool(n, 6), inputs.qeb_pool(n, 6)[::5]])
    sec = oracle.Sector(n, 3, 3)
    theta = p["theta"] * 6
    psi = A.apply_ansatz(sec, p["ops"], theta, A.hf_state(sec, p["occ"]))
    sig = A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi)
    nrm = np.vdot(psi, psi).real
    gref = np.array([2 * np.vdot(sig, A.generator_apply(sec, op, psi)).real / nrm for op in pool])
    st = _state(n, 3, 3, dtype)
    st.set_option(sv.SV_OPT_POOL_VARIANT, variant)
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], theta)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    E, g = st.pool_gradients(ham, pool)
    assert abs(E - np.vdot(psi, sig).real / nrm) <= (1e-10 if dtype == "c128" else 1e-5)
    assert np.max(np.abs(g - gref)) <= tol
    # the pool's pair lists are kept beside the ansatz's: alternating calls, and a
    # changed pool, give the same answers
    E2, g2 = st.energy_grad(ham, p["ops"], theta)
    Eg, gg = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, A.hf_state(sec, p["occ"]))
    assert abs(E2 - Eg) <= (1e-10 if dtype == "c128" else 1e-5) and np.max(np.abs(g2 - gg)) <= tol
    _, g3 = st.pool_gradients(ham, pool[::-3])
    assert np.max(np.abs(g3 - gref[::-3])) <= tol
    _, g4 = st.pool_gradients(ham, pool)
    assert np.array_equal(g4, g)


@pytest.mark.parametrize("variant", [4, 5])
@pytest.mark.parametrize("storage", ["sector", "dense"])
def test_same_spin_products_match_oracle(storage, variant):
    """Expectation variant 4 (same-spin part as two dense products in the string-blocked
    basis, on the tensor cores with bf16x3 operands; variant 5 also the alpha-beta part
    as tensor-core products) on an open-shell complex
    start: energy, gradient and pool gradients within the complex64 tolerance, and reruns
    bit-identical."""
    n, na, nb = 16, 3, 4
    p = inputs.make_problem(n, 7, 40, seed=303)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(31))
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 5
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = sv.StateVector(n, "c64", sector=(na, nb) if storage == "sector" else None)
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    runs = []
    for _ in range(2):
        st.prepare_state(dense0.astype(np.complex64), na, nb)
        runs.append(st.energy_grad(ham, p["ops"], theta))
    E, g = runs[0]
    assert abs(E - Eref) <= TOL["c64"]["E"] and np.max(np.abs(g - gref)) <= TOL["c64"]["g"]
    assert runs[1][0] == E and np.array_equal(runs[1][1], g)
    pool = inputs.uccsd_pool(n, 7)[::5]
    psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
    sig = A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi)
    gp_ref = np.array([2 * np.vdot(sig, A.generator_apply(sec, op, psi)).real for op in pool])
    _, gp = st.pool_gradients(ham, pool)
    assert np.max(np.abs(gp - gp_ref)) <= TOL["c64"]["g"]


@pytest.mark.parametrize("variant", [4, 5])
def test_same_spin_products_several_tiles(variant):
    """The tensor-core same-spin products over several output tiles with ragged edges in
    both directions (D_alpha = 330: three 128-row tiles, the last 74 rows; D_beta = 462:
    two 256-column tiles, the last 206) and K blocks of 32 with a ragged last block, on
    an open-shell complex start: energy and gradient match the oracle within the
    complex64 tolerance, and agree to rounding with the split gather form (variant 3,
    no products on the tensor cores).  Variant
    5 adds the alpha-beta products over the same three alpha tiles (units of one tile and
    one partner row: 3 x 462, spread over the SMs with a ragged last round)."""
    n, na, nb = 22, 4, 5
    p = inputs.make_problem(n, 9, 6, seed=404)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(5))
    sec = oracle.Sector(n, na, nb)
    assert (math.comb(n // 2, na), math.comb(n // 2, nb)) == (330, 462)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 5
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    out = {}
    for v in (3, variant):
        st = _state(n, na, nb, "c64")
        st.set_option(sv.SV_OPT_EXPECT_VARIANT, v)
        st.prepare_state(dense0.astype(np.complex64), na, nb)
        E, g = st.energy_grad(ham, p["ops"], theta)
        assert abs(E - Eref) <= TOL["c64"]["E"] and np.max(np.abs(g - gref)) <= TOL["c64"]["g"], v
        out[v] = (E, g)
    assert abs(out[3][0] - out[variant][0]) <= TOL["c64"]["E"]
    assert np.max(np.abs(out[3][1] - out[variant][1])) <= TOL["c64"]["g"]


def _applies_in(sec, op):
    """Whether op has a pair in the sector: it annihilates at most N_alpha alpha and
    N_beta beta spin-orbitals (uccsd_pool rows: kind, i, j, a, b with i, j annihilated)."""
    ann = [int(op[1])] + ([int(op[2])] if op[0] == 2 else [])
    return sum(j % 2 == 0 for j in ann) <= sec.na and sum(j % 2 == 1 for j in ann) <= sec.nb


@pytest.mark.parametrize("storage", ["dense", "sector"])
@pytest.mark.parametrize("variant", [1, 2])
def test_pool_gradients_ops_outside_the_sector(storage, variant):
    """One alpha electron: every alpha-alpha double has no pair in the sector (empty
    alpha list), so its gradient is exactly zero; the other operators still match."""
    n = 12
    p = inputs.make_problem(n, 4, 20, seed=515)
    occ = [0, 1, 3, 5]                                       # alpha orbital 0; beta 0, 1, 2
    sec = oracle.Sector(n, 1, 3)
    psi0 = A.hf_state(sec, occ)
    pool = inputs.uccsd_pool(n, 4)
    rng = np.random.default_rng(5)
    # an ansatz of beta singles / alpha-beta doubles that stays in the (1, 3) sector
    keep = [op for op in pool if _applies_in(sec, op)]
    ans = np.array(keep[:12])
    theta = rng.uniform(-0.4, 0.4, len(ans))
    psi = A.apply_ansatz(sec, ans, theta, psi0)
    sig = A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi)
    gref = np.array([2 * np.vdot(sig, A.generator_apply(sec, op, psi)).real for op in pool])
    st = sv.StateVector(n, "c128", sector=(1, 3) if storage == "sector" else None)
    st.set_option(sv.SV_OPT_POOL_VARIANT, variant)
    st.prepare_hf(occ)
    st.apply_ansatz(ans, theta)
    _, g = st.pool_gradients(sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"]), pool)
    assert np.max(np.abs(g - gref)) <= 1e-9
    dead = [k for k, op in enumerate(pool) if not _applies_in(sec, op)]
    assert dead and all(g[k] == 0.0 for k in dead)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_checkpoints_and_byte_cap(dtype):
    p = inputs.make_problem(14, 4, 50, seed=77)
    sec = oracle.Sector(14, 2, 2)
    theta = p["theta"] * 4
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    amp = 8 if dtype == "c64" else 16
    for interval, cap in [(7, 0), (1, 0), (5, 6 * sec.D * amp)]:
        st = _state(14, 2, 2, dtype)
        st.set_option(sv.SV_OPT_CHECKPOINT_INTERVAL, interval)
        if cap:
            st.set_option(sv.SV_OPT_MAX_BYTES, cap + (1 << 22))
        st.prepare_hf(p["occ"])
        E, g = st.energy_grad(ham, p["ops"], theta)
        assert abs(E - Eref) <= TOL[dtype]["E"]
        assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]


@pytest.mark.parametrize("na,nb,ops", [
    (2, 0, [(1, 0, -1, 4, -1), (1, 2, -1, 6, -1), (2, 0, 2, 4, 6), (1, 0, -1, 6, -1)]),   # one beta row
    (4, 1, [(1, 1, -1, 3, -1), (1, 1, -1, 7, -1), (1, 3, -1, 5, -1)]),                     # one alpha column
    (1, 1, [(1, 0, -1, 2, -1), (2, 0, 1, 4, 5), (1, 1, -1, 7, -1), (4, 0, 1, 2, 7)]),
])
def test_degenerate_sectors(na, nb, ops):
    """Sectors with a single string on one spin (D_alpha or D_beta = 1), and an empty ansatz."""
    n = 8
    rng = np.random.default_rng(na * 10 + nb)
    ops = np.array(ops, np.int32)
    theta = rng.normal(0, 0.7, len(ops))
    h, eri, e_nuc = inputs.synthetic_integrals(n // 2, rng)
    dense0 = inputs.random_sector_state(n, na, nb, rng)
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    Eref, gref = A.energy_grad(sec, h, eri, e_nuc, ops, theta, psi0)
    ham = sv.Hamiltonian(h, eri, e_nuc)
    st = _state(n, na, nb, "c128")
    st.prepare_state(dense0, na, nb)
    E, g = st.energy_grad(ham, ops, theta)
    assert abs(E - Eref) <= 1e-10 and np.max(np.abs(g - gref)) <= 1e-9
    assert np.max(np.abs(st.rdm1() - A.rdm1(sec, A.apply_ansatz(sec, ops, theta, psi0)))) <= 1e-12
    E0, g0 = st.energy_grad(ham, np.zeros((0, 5), np.int32), np.zeros(0))
    assert abs(E0 - A.energy(sec, h, eri, e_nuc, psi0)) <= 1e-10 and len(g0) == 0


def test_host_views_and_errors():
    n = 10
    p = inputs.make_problem(n, 4, 20, seed=12)
    st = _state(n, 2, 2, "c128")
    with pytest.raises(sv.SvError) as e:
        st.prepare_hf([0, 1, 2])                                 # 2 alpha + 1 beta: another sector
    assert e.value.status == 1
    with pytest.raises(sv.SvError):
        st.prepare_state(inputs.random_sector_state(n, 3, 1, np.random.default_rng(1)), 3, 1)
    with pytest.raises(sv.SvError):
        st.set_layout(np.arange(n)[::-1].copy())
    st.set_layout(np.arange(n))                                  # identity is accepted
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"] * 3)
    dense = st.state()
    xs = np.arange(1 << n, dtype=np.uint64)
    assert np.array_equal(st.amplitudes(xs), dense)             # gather == host scatter, bit for bit
    assert np.count_nonzero(dense[_outside(n, 2, 2)]) == 0
    assert sv.sv_state_device_ptr(st.handle) != 0


def test_deterministic_and_equal_to_dense():
    """Reruns are bit-identical; the sector handle agrees with the dense handle (same arithmetic per pair,
    different summation order) within the float64 tolerance."""
    p = inputs.config_problem(2)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(p["n_qubits"], p["na"], p["nb"], "c128")
    st.prepare_hf(p["occ"])
    E1, g1 = st.energy_grad(ham, p["ops"], p["theta"])
    E2, g2 = st.energy_grad(ham, p["ops"], p["theta"])
    assert E1 == E2 and np.array_equal(g1, g2)
    dn = sv.StateVector(p["n_qubits"], "c128")
    dn.prepare_hf(p["occ"])
    E3, g3 = dn.energy_grad(ham, p["ops"], p["theta"])
    assert abs(E1 - E3) <= 1e-11 and np.max(np.abs(g1 - g3)) <= 1e-10


def test_adapt_vqe_on_sector_storage_reaches_fci():
    n, ne, seed = 8, 4, 305
    p = inputs.make_problem(n, ne, "uccsd", seed=seed)
    E0 = B.sector_spectrum(B.hamiltonian(n, p["h"], p["eri"], p["e_nuc"]), n, ne // 2, ne // 2)[0]
    st = _state(n, ne // 2, ne // 2, "c128")
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    out = adapt_vqe(st, ham, p["occ"], inputs.uccsd_pool(n, ne), max_ops=60, grad_tol=1e-6, energy_tol=1e-12,
                    vqe_gtol=1e-9)
    assert out["energy"] >= E0 - 1e-10 and out["energy"] - E0 < 1e-8


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("chunk", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("variant", [2, 3, 4, 5])
def test_expectation_forms_and_chunks(variant, chunk, dtype):
    """Single-kernel (2), split (3) and split with same-spin products (4; complex64 only,
    complex128 keeps 3) string-row expectation, every partner-row chunk size, on an
    open-shell complex start: the same energy, gradient and pool gradients to the precision's
    rounding."""
    n, na, nb = 14, 4, 2
    p = inputs.make_problem(n, 6, 30, seed=91)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(21))
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 5
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(n, na, nb, dtype)
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    st.set_option(sv.SV_OPT_AB_CHUNK, chunk)
    st.prepare_state(dense0.astype(np.complex64 if dtype == "c64" else np.complex128), na, nb)
    E, g = st.energy_grad(ham, p["ops"], theta)
    assert abs(E - Eref) <= TOL[dtype]["E"] and np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    pool = inputs.uccsd_pool(n, 6)[::4]
    psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
    sig = A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi)
    gp_ref = np.array([2 * np.vdot(sig, A.generator_apply(sec, op, psi)).real for op in pool])
    _, gp = st.pool_gradients(ham, pool)
    assert np.max(np.abs(gp - gp_ref)) <= TOL[dtype]["g"]


@pytest.mark.parametrize("na,nb", [(0, 3), (4, 0), (5, 2), (1, 5)])
@pytest.mark.parametrize("variant", [3, 4, 5])
def test_expectation_degenerate_string_spaces(na, nb, variant):
    """Sectors where one spin has a single string (no electrons, or every orbital filled):
    1 x 1 same-spin matrices, no excitations of that spin, empty pair lists; energy,
    gradient and 1-RDM match the oracle in both split forms (complex64)."""
    n = 10
    p = inputs.make_problem(n, 4, 24, seed=919)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(na * 7 + nb))
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 6
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
    for storage in ("sector", "dense"):
        st = sv.StateVector(n, "c64", sector=(na, nb) if storage == "sector" else None)
        st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
        st.prepare_state(dense0.astype(np.complex64), na, nb)
        E, g = st.energy_grad(sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"]), p["ops"], theta)
        assert abs(E - Eref) <= TOL["c64"]["E"] and np.max(np.abs(g - gref)) <= TOL["c64"]["g"], storage
        assert np.max(np.abs(st.rdm1() - A.rdm1(sec, psi))) <= TOL["c64"]["rdm"], storage


@pytest.mark.parametrize("variant", [3, 5])
def test_sixteen_orbitals(variant):
    """N = 16 spatial orbitals (32 qubits), the most the string tables and the tensor-core
    alpha-beta form take (K = 16 orbitals + 120 pairs = 136: nine K blocks of 16, the last
    partly padding), in sector storage from the Hartree-Fock state with a 24-operator
    ansatz (2 + 2 electrons: 120 x 120 strings): energy and gradient match the oracle
    within the complex64 tolerance, in the tensor-core form and in the split form."""
    n, ne = 32, 4
    p = inputs.make_problem(n, ne, 24, seed=3232)
    sec = oracle.Sector(n, ne // 2, ne // 2)
    psi0 = A.hf_state(sec, p["occ"])
    theta = p["theta"] * 8
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    st = _state(n, ne // 2, ne // 2, "c64")
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"]), p["ops"], theta)
    assert abs(E - Eref) <= TOL["c64"]["E"] and np.max(np.abs(g - gref)) <= TOL["c64"]["g"]


def test_automatic_form_and_the_byte_cap():
    """The automatic expectation form on a sector of 1.66 M determinants (26 qubits, 5 + 5
    electrons, 1,287 strings per spin): the tensor-core alpha-beta form (variant 5,
    bit-identical to choosing it) where its planes (2 x 1287 x 41 x 1287 floats, 543 MB)
    fit, and variant 4 (bit-identical to choosing it) under a byte cap they do not fit."""
    n, na, nb = 26, 5, 5
    p = inputs.make_problem(n, 10, 12, seed=2626)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])

    def energy(variant, cap=0):
        st = _state(n, na, nb, "c64")
        st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
        if cap:
            st.set_option(sv.SV_OPT_MAX_BYTES, cap)
        st.prepare_hf(p["occ"])
        st.apply_ansatz(p["ops"], p["theta"] * 5)
        return st.energy(ham)

    E4, E5 = energy(4), energy(5)
    assert energy(0) == E5
    assert energy(0, cap=400 << 20) == E4
    assert abs(E4 - E5) <= TOL["c64"]["E"]


@pytest.mark.parametrize("dtype", ["c128", "c64", "r64", "r32"])
def test_whole_sweep_launches_match_per_op_and_oracle(dtype):
    """Sector storage: the forward and reverse sweeps as one cooperative launch each
    (SV_OPT_SECTOR_SWEEP = 1, grid barriers between operators) and as one launch per
    operator (0): energy, gradient and psi(theta) match the oracle in both modes and
    agree with each other to rounding.  The operator list mixes singles, doubles and
    operators with no pair in the sector (they annihilate more beta electrons than the
    sector holds: skipped with no barrier, gradient exactly 0); the sector of 20 qubits
    with 3 + 1 electrons has 120 x 10 strings."""
    n, na, nb = 20, 3, 1
    p = inputs.make_problem(n, 4, 80, seed=919)
    extra = np.array([(2, 1, 3, 11, 13), (2, 1, 3, 15, 17), (2, 3, 5, 7, 9)], np.int32)   # two beta holes each
    ops = np.vstack([p["ops"][:30], extra[:2], p["ops"][30:], extra[2:]])
    theta = np.concatenate([p["theta"][:30], [0.3, -0.2], p["theta"][30:], [0.1]]) * 4
    sec = oracle.Sector(n, na, nb)
    if dtype.startswith("c"):
        dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(91))
    else:
        dense0 = np.zeros(1 << n)
        dense0[(1 << 0) | (1 << 2) | (1 << 4) | (1 << 1)] = 1.0
    psi0 = dense0[sec.dets.astype(np.int64)]
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], ops, theta, psi0)
    psi_ref = A.apply_ansatz(sec, ops, theta, psi0)
    tol = TOL["c128" if dtype in ("c128", "r64") else "c64"]
    npdt = {"c128": np.complex128, "c64": np.complex64, "r64": np.float64, "r32": np.float32}[dtype]
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    out = {}
    for mode in (1, 0):
        st = _state(n, na, nb, dtype)
        st.set_option(sv.SV_OPT_SECTOR_SWEEP, mode)
        assert st.option(sv.SV_OPT_SECTOR_SWEEP) == mode
        st.prepare_state(dense0.astype(npdt), na, nb)
        E, g = st.energy_grad(ham, ops, theta)
        assert abs(E - Eref) <= tol["E"], (mode, E, Eref)
        assert np.max(np.abs(g - gref)) <= tol["g"], mode
        assert g[30] == 0.0 and g[31] == 0.0 and g[-1] == 0.0
        got = st.state()
        assert np.max(np.abs(got[sec.dets.astype(np.int64)] - psi_ref)) <= tol["amp"]
        st.prepare_state(dense0.astype(npdt), na, nb)          # the forward sweep alone (sv_apply_ansatz)
        st.apply_ansatz(ops, theta)
        assert np.max(np.abs(st.state()[sec.dets.astype(np.int64)] - psi_ref)) <= tol["amp"]
        out[mode] = (E, g)
        st.close()
    assert abs(out[0][0] - out[1][0]) <= tol["E"]
    assert np.max(np.abs(out[0][1] - out[1][1])) <= tol["g"]


def test_whole_sweep_barrier_wait_runs_out_reports_and_recovers():
    """With one poll per barrier wait the whole-sweep launch's grid barriers run out (no
    block waits more than a poll; every block then stops): the call reports SV_ERR_CUDA
    and the handle refuses work until a state is prepared again; with the default limit
    the same handle matches the oracle."""
    n, na, nb = 16, 2, 2
    p = inputs.config_problem(2)
    sec = oracle.Sector(n, na, nb)
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(n, na, nb, "c128")
    st.set_option(sv.SV_OPT_WAIT_POLLS, 1)
    st.prepare_hf(p["occ"])
    with pytest.raises(sv.SvError) as e:
        st.energy_grad(ham, p["ops"], p["theta"])
    assert e.value.status == 3 and "bounded wait" in str(e.value)
    with pytest.raises(sv.SvError) as e2:
        st.energy(ham)
    assert e2.value.status == 5
    st.set_option(sv.SV_OPT_WAIT_POLLS, 1 << 22)
    for _ in range(2):
        st.prepare_hf(p["occ"])
        E, g = st.energy_grad(ham, p["ops"], p["theta"])
        assert abs(E - Eref) <= 1e-10 and np.max(np.abs(g - gref)) <= 1e-9
