"""The autotuners (sv_autotune, sv_batch_autotune): they choose among launch forms and
geometries only (which can change the order of sums), so after tuning every result still
matches the oracle or the untuned run to the precision's rounding, the state the tuner ran
beside is unchanged bit for bit, and the chosen values come from the candidate sets."""
import numpy as np
import pytest

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs, sv

pytestmark = pytest.mark.gpu

TOL = {"c128": (1e-10, 1e-9), "c64": (1e-5, 1e-5)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


@pytest.mark.parametrize("storage", ["dense", "sector"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_autotune_keeps_results(storage, dtype):
    p = inputs.make_problem(16, 6, 60, seed=404)
    sec = oracle.Sector(16, 3, 3)
    psi0 = A.hf_state(sec, p["occ"])
    theta = p["theta"] * 4
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = sv.StateVector(16, dtype, sector=None if storage == "dense" else (3, 3))
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], theta)
    before = st.state()
    choice = st.autotune(ham, p["ops"], theta)
    assert np.array_equal(st.state(), before)                 # the tuner leaves psi alone
    assert choice["expect_variant"] in ((2, 3, 4, 5) if dtype == "c64" else (2, 3, 6))
    if choice["expect_variant"] in (3, 4, 6):
        assert choice["ab_chunk"] in ((2, 4, 6, 8) if dtype == "c64" else (1, 2, 3, 4))
    assert choice["rot_blocks_per_sm"] in (4, 8, 16, 32) and choice["sect_blocks_per_sm"] in (4, 8, 16, 32)
    assert choice["rdm_blocks_per_sm"] in (2, 4, 8, 16)
    assert choice["sweep_blocks_per_sm"] in (1, 2, 4, 8)
    st.prepare_hf(p["occ"])
    E, g = st.energy_grad(ham, p["ops"], theta)
    tE, tg = TOL[dtype]
    assert abs(E - Eref) <= tE and np.max(np.abs(g - gref)) <= tg
    rdm_ref = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], theta, psi0))
    assert np.max(np.abs(st.rdm1() - rdm_ref)) <= (1e-12 if dtype == "c128" else 2e-6)


def test_option_round_trip_and_range():
    st = sv.StateVector(8, "c64")
    for opt, val in ((sv.SV_OPT_ROT_BLOCKS_PER_SM, 16), (sv.SV_OPT_SECT_BLOCKS_PER_SM, 4),
                     (sv.SV_OPT_RDM_BLOCKS_PER_SM, 2), (sv.SV_OPT_AB_CHUNK, 6), (sv.SV_OPT_EXPECT_VARIANT, 3)):
        st.set_option(opt, val)
        assert st.option(opt) == val
    with pytest.raises(sv.SvError):
        st.set_option(sv.SV_OPT_ROT_BLOCKS_PER_SM, 0)
    with pytest.raises(sv.SvError):
        st.set_option(sv.SV_OPT_RDM_BLOCKS_PER_SM, 65)
    st.set_option(sv.SV_OPT_POOL_VARIANT, 1)
    assert st.option(sv.SV_OPT_POOL_VARIANT) == 1
    with pytest.raises(sv.SvError):
        st.set_option(sv.SV_OPT_POOL_VARIANT, 3)
    assert st.option(sv.SV_OPT_L2_FETCH) == 32
    for v in (0, 64, 128, 32):
        st.set_option(sv.SV_OPT_L2_FETCH, v)
        assert st.option(sv.SV_OPT_L2_FETCH) == v
    with pytest.raises(sv.SvError):
        st.set_option(sv.SV_OPT_L2_FETCH, 48)


def test_batch_autotune_keeps_results():
    probs = inputs.batch_problems(48)
    theta = np.concatenate([q["theta"] for q in probs])
    b = sv.Batch(probs, "c64")
    e1, g1 = b.energy_grad(theta)
    grid = b.autotune(theta)
    assert grid >= 1
    e2, g2 = b.energy_grad(theta)
    # the block size changes the order of the per-instance sums: equal to complex64 rounding
    assert np.max(np.abs(e1 - e2)) <= 1e-5
    assert max(float(np.max(np.abs(x - y))) if len(x) else 0.0 for x, y in zip(g1, g2)) <= 1e-5
    e3, g3 = b.energy_grad(theta)                     # and a rerun with the tuned choice is bit-identical
    assert np.array_equal(e2, e3) and all(np.array_equal(x, y) for x, y in zip(g2, g3))
    b.close()
