"""Strategy 2 of the paper (Methodology, "Strategy 2: Self-consistent basis-set
correction") as a host loop over the C-ABI, and one-body properties from the 1-RDM.

The self-consistent scheme minimises <Psi|H|Psi> + E[n_Psi] (Eq. E2B): the
ansatz is optimised for the effective Hamiltonian H~[n] = H + V[n] (Eqs.
HBPsi=EPsi, HtildeBn), with V[n] the one-body potential dE/dn of the density
functional, the potential is rebuilt from the new density, and the loop stops
when two successive eigenvalues differ by less than 0.1 mHa (about two
iterations in the paper).  The final energy is
    E_2 = EPS + E[n] - sum_pq v_pq n_pq + Delta E_HF
(the equation after HtildeBn), with n_pq the spin-summed 1-RDM, which the
state-vector path supplies (Strategy 2, equation for n_{pq,sigma}).

The paper's functional is the PBE-based basis-set correlation correction
evaluated on real-space grids with the basis functions; neither is available
here, so ``functional`` is any object with ``energy(gamma)`` and
``potential(gamma)`` on the orbital-basis density matrix.  ``OccupationFunctional``
is a synthetic stand-in of that shape (a smooth local function of the natural
occupations), used by the tests.  The dipole moment is the expectation value of a
one-body operator (Results, "Dipole Moments"): sum_pq d_pq n_pq plus the nuclear
part.
"""
import numpy as np

from .adapt import vqe
from .sv import Hamiltonian, StateVector


class OccupationFunctional:
    """Synthetic density functional of the orbital occupations: E[n] = kappa sum_p n_pp^(4/3).

    potential(gamma)[p, q] = dE/dn_pq = (4/3) kappa n_pp^(1/3) delta_pq, with n the
    spin-summed 1-RDM.  A stand-in with the shape (and sign convention) of a
    correlation-like correction; not the paper's functional.
    """

    def __init__(self, kappa: float = -0.02):
        self.kappa = float(kappa)

    def energy(self, gamma) -> float:
        n = np.clip(np.real(np.diag(gamma)), 0.0, None)
        return float(self.kappa * np.sum(n ** (4.0 / 3.0)))

    def potential(self, gamma) -> np.ndarray:
        n = np.clip(np.real(np.diag(gamma)), 0.0, None)
        return np.diag(4.0 / 3.0 * self.kappa * n ** (1.0 / 3.0))


def spin_summed(rdm):
    """n_pq = n_pq,alpha + n_pq,beta from the [2, N, N] spin-resolved 1-RDM."""
    return np.asarray(rdm)[0] + np.asarray(rdm)[1]


def dipole(rdm, d_ints, nuclear=0.0) -> float:
    """One-body expectation value sum_pq d_pq n_pq + nuclear (real symmetric d)."""
    n = spin_summed(rdm)
    return float(np.real(np.sum(np.asarray(d_ints) * n)) + nuclear)


def strategy2(state: StateVector, h, eri, e_nuc: float, occ, ops, theta0, functional,
              tol: float = 1e-4, max_iter: int = 20, delta_hf: float = 0.0, vqe_gtol: float = 1e-8):
    """Self-consistent basis-set-corrected VQE with a fixed ansatz ``ops``.

    Returns dict(E2, eps, history, theta, rdm, potential, energy_H, converged):
    ``eps`` the last eigenvalue of H~, ``energy_H`` = <psi|H|psi> of the final state.
    """
    h = np.asarray(h, dtype=np.float64)
    theta = np.asarray(theta0, dtype=np.float64).copy()
    v = np.zeros_like(h)
    eps_prev, history, converged = None, [], False
    ham_bare = Hamiltonian(h, eri, e_nuc)
    for _ in range(max_iter):
        ham_t = Hamiltonian(h + v, eri, e_nuc)          # H~[n] = H + V[n]: one-body update
        state.prepare_hf(occ)
        eps, theta, _ = vqe(state, ham_t, ops, theta, gtol=vqe_gtol)
        ham_t.close()
        rdm = state.rdm1()
        n = spin_summed(rdm).real
        history.append(eps)
        if eps_prev is not None and abs(eps - eps_prev) < tol:
            converged = True
            v_used = v
            break
        eps_prev = eps
        v_used = v
        v = functional.potential(n)
    n = spin_summed(rdm).real
    E2 = eps + functional.energy(n) - float(np.sum(v_used * n)) + delta_hf
    energy_H = state.energy(ham_bare)
    ham_bare.close()
    return dict(E2=E2, eps=eps, history=history, theta=theta, rdm=rdm, potential=v_used, energy_H=energy_H,
                converged=converged)
