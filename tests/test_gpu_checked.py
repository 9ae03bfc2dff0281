"""The checked build on the GPU (libsv_gb300_check.so, every kernel source compiled with
SV_CHECK=1): the sector sweeps, the 1-RDM rows, pool screening and the tensor-core
expectation (variant 5: gather tables, plane offsets) run through it in a separate process, match the oracle, and
record no out-of-range index (sv_check_status() == 0)."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    from paper_2405_11567_gb300 import build, inputs, sv
    import oracle
    from oracle import route_a as A
    build.build(check=True)
    assert sv.library_path() == build.LIB_CHECK
    n = 20
    p = inputs.make_problem(n, 6, 40, seed=4242)
    na, nb = p["na"], p["nb"]
    sec = oracle.Sector(n, na, nb)
    psi0 = A.hf_state(sec, p["occ"])
    theta = p["theta"] * 5
    Eref, gref = A.energy_grad(sec, p["h"], p["eri"], p["e_nuc"], p["ops"], theta, psi0)
    psi = A.apply_ansatz(sec, p["ops"], theta, psi0)
    rdm_ref = A.rdm1(sec, psi)
    pool = inputs.uccsd_pool(n, 6)[::7]
    sig = A.hamiltonian_apply(sec, p["h"], p["eri"], p["e_nuc"], psi)
    nrm = np.vdot(psi, psi).real
    pref = np.array([2 * np.vdot(sig, A.generator_apply(sec, op, psi)).real / nrm for op in pool])
    ham = sv.Hamiltonian(p["h"], p["eri"], p["e_nuc"])
    for variant in (5, 3):
        st = sv.StateVector(n, "c64", sector=(na, nb))
        st.set_option(sv.SV_OPT_EXPECT_VARIANT, variant)
        st.prepare_hf(p["occ"])
        E, g = st.energy_grad(ham, p["ops"], theta)
        assert abs(E - Eref) <= 1e-5 and np.max(np.abs(g - gref)) <= 1e-5, (variant, E, Eref)
        assert np.max(np.abs(st.rdm1() - rdm_ref)) <= 2e-6, variant
        _, pg = st.pool_gradients(ham, pool)
        assert np.max(np.abs(pg - pref)) <= 1e-5, variant
        st.close()
    status = sv.sv_check_status()
    assert status == 0, hex(status)
    print("checked build: clean")
""")


def test_checked_build_runs_clean_and_matches_the_oracle():
    env = dict(os.environ, SV_GB300_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CODE.format(root=ROOT)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build: clean" in r.stdout
