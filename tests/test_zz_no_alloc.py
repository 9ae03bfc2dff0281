"""sv_rdm1_noalloc: the 1-RDM computed with the library's fixed device scratch array
instead of any allocation, for callers that cannot allocate device memory.

Collected last on purpose (file name): if it fails, a run that stops at the first
failure has already run every other test.  It builds its own states, so it passes
alone in a fresh process as well as after the other tests."""
import math

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


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-6)])
def test_rdm1_noalloc_matches_sv_rdm1_on_two_calls(dtype, tol):
    n, na, nb = 14, 3, 2
    p = inputs.make_problem(n, 4, 60, seed=501)
    rng = np.random.default_rng(4)
    v = inputs.random_sector_state(n, na, nb, rng)
    st = sv.StateVector(n, dtype)
    st.set_layout(np.arange(n))            # qubit order in device memory, as the entry point expects
    st.prepare_state(v.astype(np.complex64 if dtype == "c64" else np.complex128), na, nb)
    st.apply_ansatz(p["ops"], p["theta"] * 5)
    ref = st.rdm1()                        # the existing entry point
    ptr = sv.sv_state_device_ptr(st.handle)
    first = sv.sv_rdm1_noalloc(ptr, n, st.dtype, na, nb)
    second = sv.sv_rdm1_noalloc(ptr, n, st.dtype, na, nb)
    assert np.max(np.abs(first - ref)) <= tol
    assert np.max(np.abs(second - ref)) <= tol
    # and against the CPU oracle's 1-RDM of the same state (complex128, literal operators)
    sec = oracle.Sector(n, na, nb)
    psi = A.apply_ansatz(sec, p["ops"], p["theta"] * 5, v[sec.dets.astype(np.int64)])
    assert np.max(np.abs(first - A.rdm1(sec, psi))) <= tol
    # a closed-shell HF-based state of another size in between reuses the same scratch
    q = inputs.config_problem(2)
    st2 = sv.StateVector(q["n_qubits"], dtype)
    st2.set_layout(np.arange(q["n_qubits"]))   # qubit order in device memory (the automatic layout off)
    st2.prepare_hf(q["occ"])
    st2.apply_ansatz(q["ops"], q["theta"])
    ref2 = st2.rdm1()
    got2 = sv.sv_rdm1_noalloc(sv.sv_state_device_ptr(st2.handle), q["n_qubits"], st2.dtype, q["na"], q["nb"])
    assert np.max(np.abs(got2 - ref2)) <= tol
    assert np.max(np.abs(sv.sv_rdm1_noalloc(ptr, n, st.dtype, na, nb) - ref)) <= tol


def test_rdm1_noalloc_sector_near_the_scratch_limit():
    """A sector that fills most of the fixed array (26 qubits, 5 + 5 electrons:
    1287^2 = 1,656,369 determinants, 6.6 MB of sector list plus the partial sums of
    8 MiB), so the data at the array's end is used: two calls match sv_rdm1 and the
    oracle's 1-RDM."""
    n, na, nb = 26, 5, 5
    assert math.comb(13, 5) ** 2 == 1656369
    p = inputs.make_problem(n, na + nb, 24, seed=611)
    theta = p["theta"] * 6
    st = sv.StateVector(n, "c128")
    st.set_layout(np.arange(n))
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], theta)
    ref = st.rdm1()
    got = [st.rdm1_noalloc(na, nb) for _ in range(2)]
    sec = oracle.Sector(n, na, nb)
    orc = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], theta, A.hf_state(sec, p["occ"])))
    for g in got:
        assert np.max(np.abs(g - ref)) <= 1e-12
        assert np.max(np.abs(g - orc)) <= 1e-12


def test_rdm1_noalloc_ordered_after_the_handles_stream():
    """A handle on a non-blocking torch stream: the 1-RDM taken right after
    apply_ansatz, with no host synchronisation in between, through the state's own
    stream, sees the rotated state (matches the oracle)."""
    import torch
    n, na, nb = 16, 2, 2
    p = inputs.config_problem(2)
    stream = torch.cuda.Stream()
    st = sv.StateVector(n, "c128", stream)
    st.set_layout(np.arange(n))
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"] * 4)   # queued on `stream`, not waited for
    got = st.rdm1_noalloc(na, nb)
    sec = oracle.Sector(n, na, nb)
    orc = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], p["theta"] * 4, A.hf_state(sec, p["occ"])))
    assert np.max(np.abs(got - orc)) <= 1e-12


def test_rdm1_noalloc_rejects_sectors_beyond_its_scratch():
    st = sv.StateVector(28, "c64")
    with pytest.raises(sv.SvError) as e:
        sv.sv_rdm1_noalloc(sv.sv_state_device_ptr(st.handle), 28, sv.SV_C64, 5, 5)   # 4,008,004 determinants
    assert e.value.status == 1 and "scratch" in str(e.value)
