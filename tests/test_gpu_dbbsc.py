"""Strategy-2 self-consistent loop (host loop over the C-ABI) against the same loop
driven by the CPU oracle, plus the identities the scheme fixes."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from oracle import route_a as A
from paper_2405_11567_gb300 import inputs, sv
from paper_2405_11567_gb300.dbbsc import OccupationFunctional, dipole, spin_summed, strategy2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2405_11567_gb300 import build
    build.build()
    sv.lib()


def _oracle_strategy2(p, functional, tol):
    """The same scheme on the CPU oracle: solve with h + v, stop when two eigenvalues agree
    to tol, E_2 = EPS + E[n] - sum v n with v the potential of the last solve."""
    sec = oracle.Sector(p["n_qubits"], p["na"], p["nb"])
    psi0 = A.hf_state(sec, p["occ"])
    theta = np.zeros(len(p["ops"]))
    v = np.zeros_like(p["h"])
    prev = None
    for _ in range(20):
        hv = p["h"] + v
        res = minimize(lambda t: A.energy_grad(sec, hv, p["eri"], p["e_nuc"], p["ops"], t, psi0), theta, jac=True,
                       method="BFGS", options=dict(gtol=1e-10))
        theta, eps = res.x, res.fun
        n = spin_summed(A.rdm1(sec, A.apply_ansatz(sec, p["ops"], theta, psi0))).real
        if prev is not None and abs(eps - prev) < tol:
            return eps + functional.energy(n) - float(np.sum(v * n)), n
        prev = eps
        v = functional.potential(n)
    raise AssertionError("oracle loop did not converge")


def test_strategy2_matches_oracle_loop_and_identity():
    p = inputs.config_problem(1)
    f = OccupationFunctional(kappa=-0.05)
    st = sv.StateVector(p["n_qubits"], "c128")
    out = strategy2(st, p["h"], p["eri"], p["e_nuc"], p["occ"], p["ops"], np.zeros(len(p["ops"])), f,
                    tol=1e-7, delta_hf=0.0125, vqe_gtol=1e-10)
    assert out["converged"] and len(out["history"]) >= 2
    n = spin_summed(out["rdm"]).real
    # E_2 = EPS + E[n] - sum v n + dHF  equals  <H> + E[n] + dHF at self-consistency
    assert abs(out["E2"] - (out["energy_H"] + f.energy(n) + 0.0125)) < 1e-9
    E2_ref, n_ref = _oracle_strategy2(p, f, 1e-7)
    assert abs(out["E2"] - 0.0125 - E2_ref) < 1e-7
    assert np.max(np.abs(n - n_ref)) < 1e-6


def test_dipole_is_the_rdm_contraction():
    p = inputs.make_problem(12, 4, 40, seed=77)
    rng = np.random.default_rng(1)
    d = rng.normal(size=(6, 6))
    d = d + d.T
    st = sv.StateVector(12, "c64")
    st.prepare_hf(p["occ"])
    st.apply_ansatz(p["ops"], p["theta"] * 4)
    sec = oracle.Sector(12, 2, 2)
    g = A.rdm1(sec, A.apply_ansatz(sec, p["ops"], p["theta"] * 4, A.hf_state(sec, p["occ"])))
    ref = float(np.real(np.sum(d * (g[0] + g[1])))) + 0.3
    assert abs(dipole(st.rdm1(), d, 0.3) - ref) < 1e-5
