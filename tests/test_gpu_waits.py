"""Failure detection without a GPU fault: the bounded waits of the tensor-core
expectation kernels (k_same_tc, k_ab_tc).

A test hook (SV_OPT_TEST_STALL) makes a kernel's producer issue nothing -- no copy,
no tensor-memory store, no MMA -- so its consumers' first mbarrier waits run out
(after SV_OPT_WAIT_POLLS polls) with nothing in flight: the path of a stuck
producer.  The kernel must set its error flag, free its tensor memory and return;
the call reports SV_ERR_CUDA, the handle refuses work until a state is prepared
again, and the same handle with the hook off then matches the oracle."""
import numpy as np
import pytest

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs, sv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


@pytest.fixture(scope="module")
def problem():
    n, na, nb = 16, 3, 4
    p = inputs.make_problem(n, 7, 40, seed=303)
    dense0 = inputs.random_sector_state(n, na, nb, np.random.default_rng(31))
    sec = oracle.Sector(n, na, nb)
    theta = p["theta"] * 5
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta,
                               dense0[sec.dets.astype(np.int64)])
    return dict(n=n, na=na, nb=nb, p=p, dense0=dense0.astype(np.complex64), theta=theta, E=Eref, g=gref)


@pytest.mark.parametrize("storage", ["sector", "dense"])
@pytest.mark.parametrize("variant,stall", [(4, 1), (5, 1), (5, 2), (5, 3)])
def test_bounded_wait_runs_out_reports_and_recovers(problem, storage, variant, stall):
    P = problem
    p = P["p"]
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = sv.StateVector(P["n"], "c64", sector=(P["na"], P["nb"]) if storage == "sector" else None)
    st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
    st.set_option(sv.SV_OPT_WAIT_POLLS, 4096)
    st.set_option(sv.SV_OPT_TEST_STALL, stall)
    st.prepare_state(P["dense0"], P["na"], P["nb"])
    with pytest.raises(sv.SvError) as e:
        st.energy_grad(ham, p["ops"], P["theta"])
    assert e.value.status == 3 and "bounded wait" in str(e.value)
    with pytest.raises(sv.SvError) as e2:        # failed handle: no work until a state is prepared again
        st.energy(ham)
    assert e2.value.status == 5
    st.set_option(sv.SV_OPT_TEST_STALL, 0)
    st.set_option(sv.SV_OPT_WAIT_POLLS, 1 << 22)
    for _ in range(2):                           # and the error flag was cleared: two good calls in a row
        st.prepare_state(P["dense0"], P["na"], P["nb"])
        E, g = st.energy_grad(ham, p["ops"], P["theta"])
        assert abs(E - P["E"]) <= 1e-5
        assert np.max(np.abs(g - P["g"])) <= 1e-5
    st.close()
    ham.close()


def test_wait_options_validated():
    st = sv.StateVector(8, "c64")
    for opt, bad in ((sv.SV_OPT_WAIT_POLLS, 0), (sv.SV_OPT_WAIT_POLLS, (1 << 30) + 1), (sv.SV_OPT_TEST_STALL, 4),
                     (sv.SV_OPT_TEST_STALL, -1)):
        with pytest.raises(sv.SvError) as e:
            st.set_option(opt, bad)
        assert e.value.status == 1
    assert st.option(sv.SV_OPT_WAIT_POLLS) == 1 << 22 and st.option(sv.SV_OPT_TEST_STALL) == 0
