"""FP64 CPU oracle for the two-component dipolar eGPE ground-state solver.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It never imports the CUDA package, and the CUDA package never imports it; the
two share no code.  Inputs reach both sides from
``paper_2510_24543_gb300.inputs`` (seeded generators with none of the method's
arithmetic), passed in as arrays by the caller.

Every function follows the paper (arXiv:2510.24543, "An efficient
preconditioned conjugate-gradient solver for a two-component dipolar
Bose-Einstein condensate") in its own order and notation; readings where the
paper is silent or garbled are named in each docstring.  All functions are
pinned by tests against closed forms, invariants, brute force or library
routines (``tests/test_oracle_pins.py``).  Parity status per function:

* energy/gradient, Hamiltonian, LHY, dipolar term, kinetic term: pinned (LHY
  also by Euler's identity n1 mu1 + n2 mu2 = 5/2 F of its degree-5/2 density)
* line-search coefficients E', E'': pinned (finite differences along the exact
  geodesic)
* preconditioner shift alpha_i and P_V: pinned (harmonic closed form; a
  single-component plane-wave state whose kinetic, dipolar and LHY terms have
  closed forms)
* beta (HS+ and PR+): pinned (hand-built fields with exactly known inner
  products: values, the max(., 0) clamp, zero-denominator restarts)
* P_Delta, projection, retraction, NCG loop: pinned (plane waves, invariants,
  harmonic closed form, descent, symmetry, agreement with ITE)
* ITE reference: pinned (harmonic closed form, agreement with NCG)
* parameter derivatives dE/d(g, g_dd, kappa, eta_s, trap): pinned (central
  differences of the energy, Hellmann-Feynman at a converged ground state)
* the paper's Table I energies: parity unpinned (the paper's physical
  parameters for that table are incomplete)
"""
from .egpe import (  # noqa: F401
    Grid, Params, SolveOpts, Evaluation,
    gauss_legendre_01, inner, kinetic_apply, trap_potential, dipolar_potentials,
    lhy_density_and_mu, evaluate, energy_grad, line_coeffs, line_coeffs_detail,
    preconditioner_shift, precondition, project, retract, cg_beta, ncg_solve, ite_solve,
    lhy_eta_derivatives, param_grad, PARAM_NAMES, PRECOND_MODES,
)
