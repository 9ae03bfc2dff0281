"""The largest register the library accepts, 32 qubits (16 spatial orbitals), against the
oracle: dense storage (2^32 amplitudes, 32 GiB per complex64 and 64 GiB per complex128
vector, the latter under a 200 GiB byte cap: every address and count passes 2^31) and
sector storage, on sectors small enough for the oracle."""
import numpy as np
import pytest

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs, sv

pytestmark = pytest.mark.gpu

TOL = {"c128": (1e-10, 1e-9, 1e-12), "c64": (1e-5, 1e-5, 2e-6)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


@pytest.fixture(scope="module")
def problems():
    out = {}
    for ne, L, seed in ((2, 40, 3232), (6, 30, 3233)):
        p = inputs.make_problem(32, ne, L, seed)
        sec = oracle.Sector(32, ne // 2, ne // 2)
        psi0 = A.hf_state(sec, p["occ"])
        theta = p["theta"] * 5
        E, g = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
        psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
        out[ne] = (p, sec, theta, E, g, psi, A.rdm1(sec, psi))
    return out


@pytest.mark.parametrize("ne,storage,dtype", [(2, "dense", "c64"), (2, "sector", "c128"), (6, "dense", "c64"),
                                              (6, "dense", "c128"), (6, "sector", "c64"), (6, "sector", "c128")])
def test_32_qubits(problems, ne, storage, dtype):
    p, sec, theta, Eref, gref, psi, rdm_ref = problems[ne]
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = sv.StateVector(32, dtype, sector=None if storage == "dense" else (ne // 2, ne // 2))
    try:
        if storage == "dense" and dtype == "c128":
            st.set_option(sv.SV_OPT_MAX_BYTES, 200 << 30)  # 64 GiB vectors: psi and the (psi, lambda) pair
        st.prepare_hf(p["occ"])
        E, g = st.energy_grad(ham, p["ops"], theta)
        tE, tg, tr = TOL[dtype]
        assert abs(E - Eref) <= tE and np.max(np.abs(g - gref)) <= tg
        assert np.max(np.abs(st.rdm1() - rdm_ref)) <= tr
        # sampled amplitudes: every sector determinant plus a seeded sample outside the sector
        xs = sec.dets.astype(np.uint64)
        assert np.max(np.abs(st.amplitudes(xs) - psi)) <= tr * 10
        rng = np.random.default_rng(32)
        far = rng.integers(0, 1 << 32, size=4096, dtype=np.uint64)
        far = far[~np.isin(far, xs)]
        assert np.count_nonzero(st.amplitudes(far)) == 0
    finally:
        st.close()
        ham.close()


def test_32_qubits_half_filling_properties():
    """8 + 8 electrons in 16 orbitals: C(16,8)^2 = 165,636,900 determinants (string ranks at the
    15-bit limit of the pair lists, rows too long for the split expectation, so its one-kernel form
    runs).  Too large for the oracle, so properties that hold at any size: the energy of the
    reference is the Slater-Condon closed form, the 1-RDM traces to the electron counts, and the
    adjoint gradient matches central differences; complex64 agrees with complex128."""
    p = inputs.make_problem(32, 16, 12, seed=3216)
    h, eri, e_nuc = p["h"], p["eri"], p["e_nuc"]
    occ = [2 * i for i in range(8)] + [2 * i + 1 for i in range(8)]
    # closed form: E = E_nuc + sum_i h_ii + 1/2 sum_ij ([ii|jj] - [ij|ji] delta(s_i, s_j)) over spin-orbitals
    E_hf = e_nuc + sum(h[j // 2, j // 2] for j in occ)
    for i in occ:
        for j in occ:
            if i != j:
                E_hf += 0.5 * eri[i // 2, i // 2, j // 2, j // 2]
                if i % 2 == j % 2:
                    E_hf -= 0.5 * eri[i // 2, j // 2, j // 2, i // 2]
    ham = sv.Hamiltonian(h, eri, e_nuc)
    theta = p["theta"] * 4
    res = {}
    for dtype in ("c128", "c64"):
        st = sv.StateVector(32, dtype, sector=(8, 8))
        try:
            st.prepare_hf(occ)
            assert abs(st.energy(ham) - E_hf) <= (1e-9 if dtype == "c128" else 1e-5)
            E, g = st.energy_grad(ham, p["ops"], theta)
            rdm = st.rdm1()
            tt = 1e-9 if dtype == "c128" else 1e-6  # complex64 amplitudes, 165 M terms per trace
            assert abs(np.trace(rdm[0].real) - 8) < tt and abs(np.trace(rdm[1].real) - 8) < tt
            if dtype == "c128":
                for k in (0, len(theta) - 1):
                    tp, tm = theta.copy(), theta.copy()
                    tp[k] += 1e-5
                    tm[k] -= 1e-5
                    st.prepare_hf(occ)
                    st.apply_ansatz(p["ops"], tp)
                    Ep = st.energy(ham)
                    st.prepare_hf(occ)
                    st.apply_ansatz(p["ops"], tm)
                    Em = st.energy(ham)
                    assert abs((Ep - Em) / 2e-5 - g[k]) < 1e-7
            res[dtype] = (E, g)
        finally:
            st.close()
    assert abs(res["c64"][0] - res["c128"][0]) < 1e-4 and np.max(np.abs(res["c64"][1] - res["c128"][1])) < 1e-4
    ham.close()
