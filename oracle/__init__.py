"""FP64 CPU oracle for the finite-temperature PEPS-VMC cooling step (arXiv:2409.05285).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA library
under ``paper_2409_05285_gb300/csrc`` and never imports it.

Every routine is a plain, slow statement of what the method computes, in float64,
citing the passage of the paper it follows (Sec. II "Method", Eqs. 1-13, App. A).
Library primitives (numpy einsum / QR / SVD / eigh) serve as single steps; there is
no blocking, fusion or reordering beyond the stated definitions.

Modules:
  philox       counter-based random numbers (Salmon et al., SC'11), used for the
               initial-state perturbation (App. A) and the Metropolis decisions.
  lattice      square lattice, OBC bond dimensions, parameter layout, bonds of Eq. 12.
  peps         PEPS of the vectorised density matrix (Eq. 4); exact contraction;
               boundary-MPS contraction at bond chi; amplitude, E_loc (Eq. 9), O_k (Eq. 8).
  sampler      Metropolis sampling of |rho|^p, p = 2 (normal) or 1 (reweighted, Eq. A1).
  direct       direct (autoregressive) sampling from double-layer marginals and its
               reweighted form p_4 with the adaptive diagonal factor b_d (Eqs. A2-A7).
  simple_update  bond-gate evolution with bond weights (the simple-update warm start of
               App. A) and its conversion to PEPS parameters.
  sr           weights, Eq. 6/7/10 reductions, CG solve, parameter update (Eq. 5).
  observables  energy (Eq. 11), specific heat, susceptibility (Eq. 13).
  ed           exact diagonalisation and full-state imaginary-time evolution (Eqs. 1-3).
  hubbard_ed   exact diagonalisation of the Fermi-Hubbard model (Eq. 14): energy, double
               occupancy and next-nearest-neighbour spin correlation (checks for a
               fermionic PEPS).
  fermion      the vectorised fermionic thermal state in the doubled Fock space (system and
               ancilla modes, the identity |I>, calH = H(c) + H(d)), its evolution, local
               energies and observables, and the amplitudes of a fermionic (Grassmann-graded)
               PEPS of sixteen local states.
  fermion_vmc  Metropolis sampling of the fermionic PEPS (pair and hop moves, Philox
               uniforms), the SR step on its samples (Eqs. 5-10) and the fermionic
               estimators (energy, double occupancy, density).

Parity status: every function here is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, brute force or exact diagonalisation (see tests/test_oracle_*.py).
"""
