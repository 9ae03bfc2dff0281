"""Full-size parity at 30 qubits (config 5), in the launch configuration bench.py times,
for both state storages (the dense 2^30 vector and the compact sector matrix).

Expected values come from tests/golden/config5_oracle.json, written by
tests/golden/make_golden.py with the CPU oracle only: the energy, all 200 gradient
entries, the 1-RDM and psi(theta) at 4,000+ sampled determinants (seeded choice
plus the largest-weight ones)."""
import json
import os

import numpy as np
import pytest

from paper_2405_11567_gb300 import inputs, sv

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"c128": dict(E=1e-10, g=1e-9, rdm=1e-11, amp=1e-11), "c64": dict(E=1e-5, g=1e-5, rdm=2e-6, amp=2e-6),
       "r64": dict(E=1e-10, g=1e-9, rdm=1e-11, amp=1e-11), "r32": dict(E=1e-5, g=1e-5, rdm=2e-6, amp=2e-6)}


@pytest.fixture(scope="module")
def golden():
    from paper_2405_11567_gb300 import build
    build.build()
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, "golden", "config5_oracle.json")) as f:
        g = json.load(f)
    p = inputs.config_problem(5)
    assert mg.same_inputs(mg.fingerprint(p), g["fingerprint"]), \
        "this machine's generator draws other inputs than the golden file's"
    return p, g


@pytest.mark.parametrize("storage", ["dense", "sector"])
@pytest.mark.parametrize("dtype", ["c64", "c128", "r32", "r64"])
def test_config5_energy_gradient_rdm_and_state(golden, dtype, storage):
    p, g = golden
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    st = sv.StateVector(p["n_qubits"], dtype, sector=None if storage == "dense" else (p["na"], p["nb"]))
    st.prepare_hf(p["occ"])
    E, grad = st.energy_grad(ham, p["ops"], p["theta"])
    rdm = st.rdm1()
    t = TOL[dtype]
    assert abs(E - g["energy"]) <= t["E"], (E, g["energy"])
    assert np.max(np.abs(grad - np.array(g["gradient"]))) <= t["g"]
    ref_rdm = np.array(g["rdm1_re"]) + 1j * np.array(g["rdm1_im"])
    assert np.max(np.abs(rdm - ref_rdm)) <= t["rdm"]
    amps = st.amplitudes(np.array(g["sample_x"], dtype=np.uint64))
    ref = np.array(g["sample_re"]) + 1j * np.array(g["sample_im"])
    assert np.max(np.abs(amps - ref)) <= t["amp"]
    # amplitudes outside the sector stay exactly zero (a seeded sample of them)
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 1 << 30, size=20000, dtype=np.uint64)
    na = np.array([bin(int(x) & 0x15555555).count("1") for x in xs])
    nb = np.array([bin(int(x) & 0x2AAAAAAA).count("1") for x in xs])
    outside = xs[(na != 5) | (nb != 5)]
    assert np.count_nonzero(st.amplitudes(outside)) == 0
