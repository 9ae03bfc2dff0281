"""Real-amplitude states (SV_R32 / SV_R64) against the oracle: the real-angle ansatz on
a real reference keeps every amplitude real, so these handles store one real per
amplitude.  Same tolerances as the complex path of the same precision."""
import numpy as np
import pytest

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs, sv

pytestmark = pytest.mark.gpu

TOL = {"r64": dict(E=1e-10, g=1e-9, amp=1e-12, rdm=1e-12), "r32": dict(E=1e-5, g=1e-5, amp=2e-6, rdm=2e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


def _state(n, na, nb, dtype, storage):
    return sv.StateVector(n, dtype, sector=None if storage == "dense" else (na, nb))


@pytest.mark.parametrize("variant", [0, 4, 5, 6])
@pytest.mark.parametrize("storage", ["dense", "sector"])
@pytest.mark.parametrize("dtype", ["r64", "r32"])
def test_energy_grad_rdm_state(dtype, storage, variant):
    p = inputs.make_problem(14, 6, 80, seed=515)
    sec = oracle.Sector(14, 3, 3)
    psi0 = A.hf_state(sec, p["occ"])
    theta = p["theta"] * 6
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = _state(14, 3, 3, dtype, storage)
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)  # 4, 5: tensor-core products (float32; float64 keeps 3)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], theta)
    t = TOL[dtype]
    assert abs(E - Eref) <= t["E"] and np.max(np.abs(g - gref)) <= t["g"]
    got = st.state()
    assert got.dtype == (np.float64 if dtype == "r64" else np.float32)
    assert np.max(np.abs(got[sec.dets.astype(np.int64)] - psi.real)) <= t["amp"] * 10
    assert np.max(np.abs(psi.imag)) == 0.0
    rdm = st.rdm1()
    assert np.max(np.abs(rdm - A.rdm1(sec, psi))) <= t["rdm"]
    assert np.count_nonzero(rdm.imag) == 0
    assert abs(st.energy(ham) - Eref) <= t["E"]


@pytest.mark.parametrize("storage", ["dense", "sector"])
def test_real_matches_complex_and_open_shell_start(storage):
    """A real open-shell multi-determinant start: r64 and c128 handles agree to rounding."""
    n, na, nb = 12, 3, 2
    p = inputs.make_problem(n, 4, 40, seed=616)
    rng = np.random.default_rng(9)
    dense0 = inputs.random_sector_state(n, na, nb, rng).real.copy()
    dense0 /= np.linalg.norm(dense0)
    sec = oracle.Sector(n, na, nb)
    psi0 = dense0[sec.dets.astype(np.int64)].astype(np.complex128)
    theta = p["theta"] * 5
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    out = {}
    for dtype in ("r64", "c128", "r32"):
        st = _state(n, na, nb, dtype, storage)
        st.prepare_state(dense0, na, nb)
        out[dtype] = st.energy_grad(ham, p["ops"], theta)
    assert abs(out["r64"][0] - Eref) <= 1e-10 and np.max(np.abs(out["r64"][1] - gref)) <= 1e-9
    assert abs(out["r64"][0] - out["c128"][0]) <= 1e-11
    assert abs(out["r32"][0] - Eref) <= 1e-5 and np.max(np.abs(out["r32"][1] - gref)) <= 1e-5


@pytest.mark.parametrize("storage", ["dense", "sector"])
def test_jordan_wigner_signs_bit_exact_real(storage):
    n = 10
    ops = np.vstack([inputs.uccsd_pool(n, 4)[::3], inputs.qeb_pool(n, 4)[::7]])
    st = _state(n, 2, 2, "r64", storage)
    sec = oracle.Sector(n, 2, 2)
    rng = np.random.default_rng(1)
    for op in ops:
        froms = [int(x) for x in sec.dets if A.exc_apply(op, int(x))[0] != 0]
        for x in rng.choice(froms, size=min(3, len(froms)), replace=False):
            s, y = A.exc_apply(op, int(x))
            v = np.zeros(1 << n)
            v[int(x)] = 1.0
            st.prepare_state(v, 2, 2)
            st.apply_ansatz(op[None, :], [np.pi / 2])
            got = st.state()
            assert got[y] == float(s) and abs(got[int(x)]) < 1e-15
            assert np.count_nonzero(np.abs(got) > 1e-15) == 1


@pytest.mark.parametrize("dtype", ["r64", "r32"])
def test_pool_gradients_and_autotune_real(dtype):
    n = 14
    p = inputs.make_problem(n, 6, 30, seed=202)
    pool = np.vstack([inputs.uccsd_pool(n, 6)[::3], inputs.qeb_pool(n, 6)[::9]])
    sec = oracle.Sector(n, 3, 3)
    theta = p["theta"] * 6
    psi = A.apply_ansatz(sec, p["ops"], theta, A.hf_state(sec, p["occ"]))
    sig = A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi)
    gref = np.array([2 * np.vdot(sig, A.generator_apply(sec, op, psi)).real for op in pool])
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    for storage in ("dense", "sector"):
        st = _state(n, 3, 3, dtype, storage)
        st.prepare_hf(p["occ"])
        st.apply_ansatz(p["ops"], theta)
        before = st.state()
        st.autotune(ham, p["ops"], theta)
        assert np.array_equal(st.state(), before)
        for variant in (1, 2):
            st.set_option(sv.SV_OPT_POOL_VARIANT, variant)
            _, g = st.pool_gradients(ham, pool)
            assert np.max(np.abs(g - gref)) <= TOL[dtype]["g"]


def test_real_handles_reject_complex_only_calls():
    with pytest.raises(ValueError):
        st = sv.StateVector(8, "r64")
        st.prepare_state(np.full(256, 1j / 16), 1, 1)
    with pytest.raises(sv.SvError):
        sv.Batch(inputs.batch_problems(2), sv.SV_R32)
