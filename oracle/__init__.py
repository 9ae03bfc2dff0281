"""CPU oracle for the state-vector hot path of arXiv:2405.11567.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference leg may import this package; the library under
``paper_2405_11567_gb300`` never does, and this package never imports it.

Two independent routes, both complex128 / float64:

* route A (:mod:`oracle.route_a`, C core in ``sv_oracle.c``): determinant space
  of the fixed (N_alpha, N_beta) sector, every operator applied literally with
  the Jordan-Wigner sign rule; works up to 30 qubits (slowly).
* route B (:mod:`oracle.route_b`): dense 2^n matrices built from Kronecker
  products of 2x2 matrices, ``scipy`` matrix exponentials and eigensolvers;
  n <= 12 only.  It shares nothing with route A.

Pins (tests/test_oracle_*.py, ``-m "not gpu"``) tie both routes to facts that
the mathematics fixes (closed forms, textbook special cases, invariants,
brute force) and to the paper's Table IV.  Functions without such a pin say
"parity unpinned" in their docstring.
"""
from .route_a import (  # noqa: F401
    Sector, hf_state, apply_ansatz, rotate, generator_apply, hamiltonian_apply,
    energy, energy_grad, rdm1, num_threads,
)
