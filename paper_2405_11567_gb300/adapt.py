"""VQE and ADAPT-VQE drivers over the C-ABI ("Computational Details": ADAPT-VQE
with an operator pool, started from the HF state, converged to 1e-6 Ha).

Both are host loops: every energy, gradient and pool screening runs in the
library's kernels (``sv_energy_grad``, ``sv_pool_gradients``); the optimiser is
scipy's BFGS on the exact adjoint gradients.
"""
import numpy as np
from scipy.optimize import minimize

from .sv import Hamiltonian, StateVector


def vqe(state: StateVector, ham: Hamiltonian, ops, theta0, gtol: float = 1e-6, maxiter: int = 1000):
    """Minimise E(theta) for the ansatz ``ops`` on the reference recorded on ``state``.

    Returns (E, theta, scipy result); on return the state holds psi(theta).
    """
    ops = np.ascontiguousarray(np.asarray(ops, dtype=np.int32).reshape(-1, 5))
    theta0 = np.asarray(theta0, dtype=np.float64).reshape(-1)
    if len(ops) == 0:
        return state.energy(ham), theta0, None

    def fun(t):
        E, g = state.energy_grad(ham, ops, t)
        return E, g

    res = minimize(fun, theta0, jac=True, method="BFGS", options=dict(gtol=gtol, maxiter=maxiter))
    E, _ = state.energy_grad(ham, ops, res.x)
    return E, res.x, res


def adapt_vqe(state: StateVector, ham: Hamiltonian, occ, pool, max_ops: int = 100, grad_tol: float = 1e-4,
              energy_tol: float = 1e-6, vqe_gtol: float = 1e-7):
    """Grow an ansatz from ``pool`` on the HF reference ``occ``.

    Each iteration screens the pool on the current state (the largest
    |dE/dtheta| at zero angle is appended, angle 0), then re-optimises all angles.
    Stops when the largest pool gradient is below ``grad_tol``, when an iteration
    lowers the energy by less than ``energy_tol`` (1e-6 Ha in the paper), or after
    ``max_ops`` operators.  Returns dict(energy, ops, theta, history, grad_norms).
    """
    pool = np.ascontiguousarray(np.asarray(pool, dtype=np.int32).reshape(-1, 5))
    ops = np.zeros((0, 5), dtype=np.int32)
    theta = np.zeros(0)
    state.prepare_hf(occ)
    E = state.energy(ham)
    history, gmax = [E], []
    for _ in range(max_ops):
        state.prepare_hf(occ)
        if len(ops):
            state.apply_ansatz(ops, theta)
        _, g = state.pool_gradients(ham, pool)
        k = int(np.argmax(np.abs(g)))
        gmax.append(float(abs(g[k])))
        if abs(g[k]) < grad_tol:
            break
        ops = np.vstack([ops, pool[k:k + 1]])
        theta = np.append(theta, 0.0)
        E_new, theta, _ = vqe(state, ham, ops, theta, gtol=vqe_gtol)
        history.append(E_new)
        done = abs(E - E_new) < energy_tol
        E = E_new
        if done:
            break
    return dict(energy=E, ops=ops, theta=theta, history=history, grad_norms=gmax)
