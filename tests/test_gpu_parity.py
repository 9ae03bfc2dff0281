"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Tolerances (the workload specification): float64 state |dE| <= 1e-10 Ha,
|dg| <= 1e-9 Ha/rad; complex64 state with float64 reductions |dE| <= 1e-5 Ha,
|dg| <= 1e-5.  Integer work (Jordan-Wigner signs, pair indices, which amplitudes
stay exactly zero) is compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs
from paper_2405_11567_gb300 import sv

pytestmark = pytest.mark.gpu

TOL = {"c128": dict(E=1e-10, g=1e-9, amp=1e-12, rdm=1e-12), "c64": dict(E=1e-5, g=1e-5, amp=2e-6, rdm=2e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


def _gpu_state(n, dtype):
    return sv.StateVector(n, dtype)


def _oracle_problem(p, na=None, nb=None):
    na = p["na"] if na is None else na
    nb = p["nb"] if nb is None else nb
    return oracle.Sector(p["n_qubits"], na, nb)


def _sector_mask(n, na, nb):
    x = np.arange(1 << n, dtype=np.int64)
    ca = sum(((x >> j) & 1) for j in range(0, n, 2))
    cb = sum(((x >> j) & 1) for j in range(1, n, 2))
    return (ca == na) & (cb == nb)


# ---------------------------------------------------------------- rotations / signs

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,ne,seed", [(8, 2, 1001), (10, 4, 7), (12, 4, 8)])
def test_ansatz_state_matches_oracle(n, ne, seed, dtype):
    p = inputs.make_problem(n, ne, "uccsd", seed)
    theta = p["theta"] * 8
    sec = _oracle_problem(p)
    ref = A.apply_ansatz(sec, p["ops"], theta, A.hf_state(sec, p["occ"]))
    st = _gpu_state(n, dtype)
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], theta)
    got = st.state()
    idx = sec.dets.astype(np.int64)
    assert np.max(np.abs(got[idx] - ref)) <= TOL[dtype]["amp"]
    outside = ~_sector_mask(n, p["na"], p["nb"])
    assert np.count_nonzero(got[outside]) == 0            # exact zeros outside the sector
    assert np.count_nonzero(got.imag) == 0                # real angles, real start: exactly real


def test_jordan_wigner_signs_bit_exact():
    """Rotation by pi/2 moves a basis state onto T|x> with amplitude exactly +-1: the sign and the
    partner index must equal the oracle's literal operator application, bit for bit."""
    n = 10
    pool = inputs.uccsd_pool(n, 4)
    extra = np.array([(2, 1, 6, 2, 5), (2, 0, 5, 2, 3), (1, 5, -1, 1, -1), (2, 2, 3, 0, 7), (1, 8, -1, 2, -1)],
                     np.int32)
    ops = np.vstack([pool, extra])
    st = _gpu_state(n, "c128")
    rng = np.random.default_rng(0)
    for op in ops:
        na = 2 if op[0] == 2 else 2
        sec = oracle.Sector(n, 2, 2)
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


# ---------------------------------------------------------------- energy / gradient

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config1_energy(dtype):
    p = inputs.config_problem(1)
    sec = _oracle_problem(p)
    Eref = A.energy(sec, p["h"], p["eri"], p["e_nuc"],
                    A.apply_ansatz(sec, p["ops"], p["theta"], A.hf_state(sec, p["occ"])))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], dtype)
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"])
    assert abs(st.energy(ham) - Eref) <= TOL[dtype]["E"]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config2_energy_grad(dtype):
    p = inputs.config_problem(2)
    sec = _oracle_problem(p)
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], dtype)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], p["theta"])
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    # the handle holds psi(theta) afterwards
    psi = A.apply_ansatz(sec, p["ops"], p["theta"], A.hf_state(sec, p["occ"]))
    assert np.max(np.abs(st.state()[sec.dets.astype(np.int64)] - psi)) <= TOL[dtype]["amp"] * 10


@pytest.mark.parametrize("dtype", ["c128", "r64", "c64"])
def test_large_angles_both_rotation_forms(dtype):
    """Angles over the whole circle: float64 amplitudes rotate by three shears when
    cos(theta) > 0 and by the direct form otherwise; both match the oracle, including
    exact quarter and half turns."""
    n = 10
    p = inputs.make_problem(n, 4, 40, seed=616)
    rng = np.random.default_rng(17)
    theta = rng.uniform(-np.pi, np.pi, len(p["ops"]))
    theta[:4] = [np.pi / 2, -np.pi / 2, np.pi, -np.pi]
    sec = _oracle_problem(p)
    psi0 = A.hf_state(sec, p["occ"])
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(n, dtype)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], theta)
    tol = TOL["c64" if dtype == "c64" else "c128"]
    assert abs(E - Eref) <= tol["E"] and np.max(np.abs(g - gref)) <= tol["g"]
    psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
    assert np.max(np.abs(st.state()[sec.dets.astype(np.int64)] - psi)) <= tol["amp"] * 10


def test_config2_gradient_central_differences():
    p = inputs.config_problem(2)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], "c128")
    st.prepare_hf(p["occ"])
    _, g = st.energy_grad(ham, p["ops"], p["theta"])
    hstep = 1e-5
    for k in range(0, len(p["ops"]), 23):
        tp, tm = p["theta"].copy(), p["theta"].copy()
        tp[k] += hstep
        tm[k] -= hstep
        st.prepare_hf(p["occ"])
        st.apply_ansatz(p["ops"], tp)
        Ep = st.energy(ham)
        st.prepare_hf(p["occ"])
        st.apply_ansatz(p["ops"], tm)
        Em = st.energy(ham)
        assert abs((Ep - Em) / (2 * hstep) - g[k]) < 1e-8


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_2405_11567_gb300.autograd import energy
    p = inputs.config_problem(2)
    sec = _oracle_problem(p)
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], "c128")
    st.prepare_hf(p["occ"])
    th = torch.tensor(p["theta"], dtype=torch.float64, requires_grad=True)
    E = energy(th, st, ham, p["ops"])
    (3.0 * E).backward()
    assert abs(E.item() - Eref) <= 1e-10
    assert np.max(np.abs(th.grad.numpy() - 3.0 * gref)) <= 3e-9


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_complex_start_open_shell(dtype):
    """A complex multi-determinant start with N_alpha != N_beta exercises every conj() of the path."""
    n, na, nb = 12, 3, 2
    p = inputs.make_problem(n, 4, 40, seed=55)
    rng = np.random.default_rng(3)
    dense0 = inputs.random_sector_state(n, na, nb, rng)
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 6
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(n, dtype)
    st.prepare_state(dense0.astype(np.complex64 if dtype == "c64" else np.complex128), na, nb)
    E, g = st.energy_grad(ham, p["ops"], theta)
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    rdm_ref = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], theta, psi0))
    assert np.max(np.abs(st.rdm1() - rdm_ref)) <= TOL[dtype]["rdm"]


# ---------------------------------------------------------------- 1-RDM

@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_rdm1_matches_oracle(dtype, variant):
    """Sector gather (1), string rows in the state's arithmetic (2) and in float-float
    arithmetic (3: float64 states; complex64 takes 2) against the oracle."""
    p = inputs.make_problem(14, 6, 60, seed=66)
    sec = _oracle_problem(p)
    psi = A.apply_ansatz(sec, p["ops"], p["theta"] * 5, A.hf_state(sec, p["occ"]))
    ref = A.rdm1(sec, psi)
    st = _gpu_state(14, dtype)
    st.set_option(sv.SV_OPT_RDM_VARIANT, variant)
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"] * 5)
    got = st.rdm1()
    assert np.max(np.abs(got - ref)) <= TOL[dtype]["rdm"]


# ---------------------------------------------------------------- config 3 (24 qubits)

@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_config3_energy_grad_rdm(dtype, config3_oracle):
    p, Eref, gref, rdm_ref = config3_oracle
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], dtype)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], p["theta"])
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    assert np.max(np.abs(st.rdm1() - rdm_ref)) <= TOL[dtype]["rdm"]


@pytest.fixture(scope="module")
def config3_oracle():
    p = inputs.config_problem(3)
    sec = _oracle_problem(p)
    psi0 = A.hf_state(sec, p["occ"])
    E, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], p["theta"], psi0)
    rdm = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], p["theta"], psi0))
    return p, E, g, rdm


# ---------------------------------------------------------------- options, edges, errors

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_checkpoints_and_byte_cap(dtype):
    p = inputs.make_problem(14, 4, 50, seed=77)
    sec = _oracle_problem(p)
    theta = p["theta"] * 4
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    for interval, cap in [(7, 0), (1, 0), (5, 6 * (1 << 14) * (8 if dtype == "c64" else 16))]:
        st = _gpu_state(14, dtype)
        st.set_option(sv.SV_OPT_CHECKPOINT_INTERVAL, interval)
        if cap:
            st.set_option(sv.SV_OPT_MAX_BYTES, cap + (1 << 22))
        st.prepare_hf(p["occ"])
        E, g = st.energy_grad(ham, p["ops"], theta)
        assert abs(E - Eref) <= TOL[dtype]["E"]
        assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]


def test_edge_cases():
    # no operators: E is the reference energy, empty gradient
    p = inputs.make_problem(8, 2, "uccsd", 3)
    sec = _oracle_problem(p)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(8, "c128")
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"][:0], [])
    assert abs(E - A.energy(sec, p["h"], p["eri"], p["e_nuc"], A.hf_state(sec, p["occ"]))) <= 1e-12 and len(g) == 0
    # vacuum and fully occupied registers; the smallest register (one orbital)
    for n, occ in [(8, []), (8, list(range(8))), (2, [0, 1]), (2, [1])]:
        q = inputs.make_problem(n, 2, "uccsd", 4)
        na = sum(1 for j in occ if j % 2 == 0)
        nb = len(occ) - na
        s2 = oracle.Sector(n, na, nb)
        e_ref = A.energy(s2, q["h"], q["eri"], q["e_nuc"], A.hf_state(s2, occ))
        hq = sv.Hamiltonian(q["h"], q["eri"], q["e_nuc"])
        st2 = _gpu_state(n, "c128")
        st2.prepare_hf(occ)
        assert abs(st2.energy(hq) - e_ref) <= 1e-12
        r = st2.rdm1()
        assert abs(np.trace(r[0]).real - na) < 1e-12 and abs(np.trace(r[1]).real - nb) < 1e-12


def test_deterministic_reruns():
    p = inputs.config_problem(2)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], "c64")
    st.prepare_hf(p["occ"])
    E1, g1 = st.energy_grad(ham, p["ops"], p["theta"])
    E2, g2 = st.energy_grad(ham, p["ops"], p["theta"])
    assert E1 == E2 and np.array_equal(g1, g2)


def test_errors_are_reported_not_raised_on_device():
    p = inputs.config_problem(1)
    st = _gpu_state(8, "c64")
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    with pytest.raises(sv.SvError) as e:
        st.energy(ham)                       # no prepared state
    assert e.value.status == 5
    st.prepare_hf(p["occ"])
    for bad in [(2, 1, 0, 2, 3), (2, 0, 1, 2, 2), (1, 0, -1, 1, -1), (2, 0, 1, 2, 9), (5, 0, 1, 2, 3),
                (3, 0, -1, 1, -1), (4, 0, 1, 2, 4)]:
        with pytest.raises(sv.SvError) as e:
            st.apply_ansatz(np.array([bad], np.int32), [0.1])
        assert e.value.status == 1
    with pytest.raises(sv.SvError):
        st.apply_ansatz(p["ops"][:1], [float("nan")])
    with pytest.raises(sv.SvError):
        st.prepare_hf([0, 0])
    v = np.zeros(256, np.complex64)
    v[3] = 1.0
    with pytest.raises(sv.SvError):
        st.prepare_state(v, 2, 0)            # x = 3 has one alpha and one beta electron
    big = sv.Hamiltonian(*inputs.synthetic_integrals(5, np.random.default_rng(0)))
    with pytest.raises(sv.SvError):
        st.energy(big)                       # n_orb mismatch
    # the handle still works after argument errors
    st.apply_ansatz(p["ops"], p["theta"])
    assert np.isfinite(st.energy(ham))


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation_variants_match_oracle(variant, dtype):
    """Record scan (1), string rows in one kernel (2), split (3), split with same-spin
    products (4) and with the alpha-beta part as tensor-core products too (5; complex128
    keeps 3), split in float-float arithmetic (6; complex64 keeps 3) on an open-shell
    complex state and on config 2."""
    n, na, nb = 12, 3, 2
    p = inputs.make_problem(n, 4, 30, seed=88)
    rng = np.random.default_rng(11)
    dense0 = inputs.random_sector_state(n, na, nb, rng)
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 7
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(n, dtype)
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    st.prepare_state(dense0.astype(np.complex64 if dtype == "c64" else np.complex128), na, nb)
    E, g = st.energy_grad(ham, p["ops"], theta)
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    q = inputs.config_problem(2)
    s2 = _oracle_problem(q)
    Eq, gq = A.energy_grad(s2, q["h"], q["eri"], q["e_nuc"], q["ops"], q["theta"], A.hf_state(s2, q["occ"]))
    hq = sv.Hamiltonian(q["h"], q["eri"], q["e_nuc"])
    st2 = _gpu_state(q["n_qubits"], dtype)
    st2.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    st2.prepare_hf(q["occ"])
    E2, g2 = st2.energy_grad(hq, q["ops"], q["theta"])
    assert abs(E2 - Eq) <= TOL[dtype]["E"]
    assert np.max(np.abs(g2 - gq)) <= TOL[dtype]["g"]


def test_sigma_vector_matches_oracle():
    """At theta = 0 every gradient entry is 2 Re <(H - c) psi0| G_k psi0>, a projection of sigma
    onto G_k psi0: a random complex start and many directions G_k probe sigma from the
    record scan, the string rows, their split form in float64 and in float-float
    arithmetic (variants 1, 2, 3, 6) in complex128 to 1e-11."""
    n = 12
    p = inputs.make_problem(n, 4, "uccsd", seed=91)
    sec = _oracle_problem(p)
    rng = np.random.default_rng(2)
    dense0 = inputs.random_sector_state(n, 2, 2, rng)
    psi0 = dense0[sec.dets.astype(np.int64)]
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    ops = p["ops"][::9]
    zeros = np.zeros(len(ops))
    _, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], ops, zeros, psi0)
    for variant in (1, 2, 3, 6):
        st = _gpu_state(n, "c128")
        st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
        st.prepare_state(dense0, 2, 2)
        _, g = st.energy_grad(ham, ops, zeros)
        assert np.max(np.abs(g - gref)) <= 1e-11, variant


# ---------------------------------------------------------------- storage layout

def test_layout_roundtrip_bit_exact():
    n = 12
    rng = np.random.default_rng(21)
    v = inputs.random_sector_state(n, 3, 2, rng)
    for dtype, cast in (("c128", np.complex128), ("c64", np.complex64)):
        st = _gpu_state(n, dtype)
        st.prepare_state(v.astype(cast), 3, 2)
        perm = rng.permutation(n)
        st.set_layout(perm)
        assert np.array_equal(st.layout(), perm)
        assert np.array_equal(st.state(), v.astype(cast))          # moved on the device, read back in qubit order
        st.set_layout(np.arange(n)[::-1].copy())
        assert np.array_equal(st.state(), v.astype(cast))


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_permuted_layout_parity(variant, dtype):
    """A random storage permutation changes nothing observable: state, energy, gradient, 1-RDM."""
    n, na, nb = 12, 3, 2
    p = inputs.make_problem(n, 4, 30, seed=99)
    rng = np.random.default_rng(5)
    dense0 = inputs.random_sector_state(n, na, nb, rng)
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 7
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    psi_ref = A.apply_ansatz(sec, p["ops"], theta, psi0)
    rdm_ref = A.rdm1(sec, psi_ref)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(n, dtype)
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    st.set_layout(rng.permutation(n))                              # also turns the automatic layout off
    st.prepare_state(dense0.astype(np.complex64 if dtype == "c64" else np.complex128), na, nb)
    st.apply_ansatz(p["ops"], theta)
    got = st.state()
    assert np.max(np.abs(got[sec.dets.astype(np.int64)] - psi_ref)) <= TOL[dtype]["amp"] * 10
    assert np.count_nonzero(got[~_sector_mask(n, na, nb)]) == 0
    assert abs(st.energy(ham) - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(st.rdm1() - rdm_ref)) <= TOL[dtype]["rdm"]
    E, g = st.energy_grad(ham, p["ops"], theta)
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]


def test_automatic_layout_moves_frequent_qubits_high():
    p = inputs.config_problem(2)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(p["n_qubits"], "c64")
    st.prepare_hf(p["occ"])
    st.energy_grad(ham, p["ops"], p["theta"])
    lay = st.layout()
    assert sorted(lay) == list(range(p["n_qubits"]))
    cnt = np.zeros(p["n_qubits"])
    for k, i, j, a, b in p["ops"]:
        for q in ((i, a) if k == 1 else (i, j, a, b)):
            cnt[q] += 1
    # address bit order follows usage: counts are non-decreasing along the address bits
    by_bit = cnt[np.argsort(lay)]
    assert np.all(np.diff(by_bit) >= 0)


def test_apply_ansatz_takes_the_automatic_layout_on_a_fresh_reference():
    """sv_apply_ansatz on the determinant sv_prepare_hf wrote takes the layout its operator
    list prefers (the one sv_energy_grad chooses) and gives the oracle's state; applied to any
    other state, or with SV_OPT_LAYOUT_AUTO off, it keeps the layout."""
    p = inputs.config_problem(2)
    n = p["n_qubits"]
    sec = _oracle_problem(p)
    psi_ref = A.apply_ansatz(sec, p["ops"], p["theta"], A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(n, "c128")
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"])
    lay = st.layout()
    assert not np.array_equal(lay, np.arange(n))
    got = st.state()
    assert np.max(np.abs(got[sec.dets.astype(np.int64)] - psi_ref)) <= TOL["c128"]["amp"]
    assert np.count_nonzero(np.delete(got, sec.dets.astype(np.int64))) == 0
    st2 = _gpu_state(n, "c128")
    st2.prepare_hf(p["occ"])
    st2.energy_grad(ham, p["ops"], p["theta"])
    assert np.array_equal(st2.layout(), lay)
    st.apply_ansatz(p["ops"][:5], p["theta"][:5])        # not the reference any more: layout kept
    assert np.array_equal(st.layout(), lay)
    st3 = _gpu_state(n, "c128")
    st3.set_option(sv.SV_OPT_LAYOUT_AUTO, 0)
    st3.prepare_hf(p["occ"])
    st3.apply_ansatz(p["ops"], p["theta"])
    assert np.array_equal(st3.layout(), np.arange(n))
    assert np.max(np.abs(st3.state() - got)) <= TOL["c128"]["amp"]


# ---------------------------------------------------------------- qubit excitations (QEB pool)

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_qubit_excitation_ansatz_matches_oracle(dtype):
    n = 14
    p = inputs.make_problem(n, 4, 50, seed=123)
    pool = inputs.qeb_pool(n, 4)
    rng = np.random.default_rng(6)
    ops = np.vstack([pool[rng.choice(len(pool), size=30, replace=False)], p["ops"][:10]])  # QEB and fermionic mixed
    theta = rng.normal(0, 0.3, size=len(ops))
    sec = _oracle_problem(p)
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], ops, theta, A.hf_state(sec, p["occ"]))
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _gpu_state(n, dtype)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, ops, theta)
    assert abs(E - Eref) <= TOL[dtype]["E"]
    assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]
    psi = A.apply_ansatz(sec, ops, theta, A.hf_state(sec, p["occ"]))
    assert np.max(np.abs(st.state()[sec.dets.astype(np.int64)] - psi)) <= TOL[dtype]["amp"] * 10
    b = sv.Batch([dict(p, ops=ops, theta=theta)], dtype)
    Eb, gb = b.energy_grad(theta)
    assert abs(Eb[0] - Eref) <= TOL[dtype]["E"] and np.max(np.abs(gb[0] - gref)) <= TOL[dtype]["g"]


@pytest.mark.parametrize("layout", ["identity", "auto"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "r64", "r32"])
def test_reverse_sweep_interleaved_and_separate(dtype, layout):
    """The dense reverse sweep on psi(theta) and lambda interleaved in one buffer
    (SV_OPT_REVERSE_INTERLEAVED = 1, the default) and on two separate vectors (0): both
    match the oracle's energy and gradient, agree with each other to rounding, and leave
    psi(theta) in the handle.  With the identity layout the ansatz's excitations sit on
    address bits 0, 1, 2 and above, so every vector width of the interleaved kernel runs
    (one, two and, for real float32, four pairs per access); a complex open-shell start
    for the complex types, the closed-shell HF start (real) for the real ones."""
    n, ne = 12, 5
    p = inputs.make_problem(n, ne, 60, seed=515)
    theta = p["theta"] * 6
    na, nb = 3, 2
    sec = oracle.Sector(n, na, nb)
    if dtype.startswith("c"):
        dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(12))
    else:
        dense0 = np.zeros(1 << n)
        dense0[sum(1 << j for j in (0, 1, 2, 3, 4))] = 1.0
    psi0 = dense0[sec.dets.astype(np.int64)]
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    psi_ref = A.apply_ansatz(sec, p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    tol = TOL["c128" if dtype in ("c128", "r64") else "c64"]
    npdt = {"c128": np.complex128, "c64": np.complex64, "r64": np.float64, "r32": np.float32}[dtype]
    out = {}
    for inter in (1, 0):
        st = sv.StateVector(n, dtype)
        if layout == "identity":
            st.set_option(sv.SV_OPT_LAYOUT_AUTO, 0)
        st.set_option(sv.SV_OPT_REVERSE_INTERLEAVED, inter)
        assert st.option(sv.SV_OPT_REVERSE_INTERLEAVED) == inter
        st.prepare_state(dense0.astype(npdt), na, nb)
        E, g = st.energy_grad(ham, p["ops"], theta)
        assert abs(E - Eref) <= tol["E"], (inter, E, Eref)
        assert np.max(np.abs(g - gref)) <= tol["g"], inter
        got = st.state()
        assert np.max(np.abs(got[sec.dets.astype(np.int64)] - psi_ref)) <= tol["amp"], inter
        assert np.count_nonzero(got[~_sector_mask(n, na, nb)]) == 0
        out[inter] = (E, g)
        st.close()
    assert abs(out[0][0] - out[1][0]) <= tol["E"]
    assert np.max(np.abs(out[0][1] - out[1][1])) <= tol["g"]


def test_float_float_sigma_matches_float64_and_oracle():
    """Expectation variant 6 (float64 states: the split form's sums in float-float
    arithmetic on the FP32 pipe) against variant 3 (the same form in float64) and the
    oracle: energy and gradient on an open-shell complex start, in both storages, with
    the two forms within 1e-11 / 1e-10 of each other."""
    n, na, nb = 14, 4, 3
    p = inputs.make_problem(n, 7, 40, seed=616)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(61))
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)]
    theta = p["theta"] * 6
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    for sector in (None, (na, nb)):
        res = {}
        for v in (3, 6):
            st = sv.StateVector(n, "c128", sector=sector)
            st.set_option(sv.SV_OPT_EXPECT_VARIANT, v)
            st.prepare_state(dense0, na, nb)
            res[v] = st.energy_grad(ham, p["ops"], theta)
            assert abs(res[v][0] - Eref) <= 1e-10, (sector, v)
            assert np.max(np.abs(res[v][1] - gref)) <= 1e-9, (sector, v)
            st.close()
        assert abs(res[3][0] - res[6][0]) <= 1e-11
        assert np.max(np.abs(res[3][1] - res[6][1])) <= 1e-10
