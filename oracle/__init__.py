"""Plain CPU oracle for the nested shift-invert MINRES method (Kutsuzawa & Todo,
arXiv:2203.09732).

This package is TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The CUDA product path never calls into it, and it shares no code with the
CUDA path: it has its own basis enumeration (brute force, ascending integers),
an explicit sparse Hamiltonian assembled from Eq. (1), the textbook MINRES of
Algorithm 2, the shift-invert Lanczos of Algorithm 1 and a direct twist sum.
Everything is FP64 (complex128 for the twist).

Conventions (the paper is silent on them, Sec. II and Sec. III):
  * site j (1-based) is bit j-1 of the state word; bit = 1 means spin up
    (Sz_j = +1/2);
  * the Sz = 0 sector states are ranked in ascending integer order;
  * J = 1 and the chain is periodic, bond (L, 1) included.

Modules:
  basis        Sz = 0 sector enumeration and ranking (Sec. I, Eq. (1)).
  hamiltonian  explicit sparse H, diagonal, preconditioners (Eq. (1), Sec. II).
  minres       Algorithm 2 (Appendix A).
  lanczos      Algorithm 1 (Sec. II) with full reorthogonalisation.
  twist        twist overlap z = <psi|U_twist|psi> (Sec. III).
  rng          SplitMix64 counter-based generator for the Lanczos start vector.
  observables  entanglement entropy and level spacing ratio (Sec. IV B).

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
closed forms, a Kronecker-product construction in the full 2^L space, brute
force on tiny inputs and exact invariants from the paper.
"""
