"""CPU oracle for two-site TDVP (2TDVP) of a vibronic Hamiltonian.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, complex128
statement of what the CUDA path computes. Only the tests, the smoke check in
`__graft_entry__` and the CPU-baseline leg of `bench.py` may import it; the
product library never does, and it shares no code with the CUDA path (both
read their inputs from the `vibmodels` generator module, which holds no part
of the method).

Modules
  vibronic  local operators, the Hamiltonian's term list (Sec. 2.2), sparse
            dense-basis H and exact propagation for tiny systems, closed forms
  mpo       finite-state-automaton MPO builder from the term list (Eq. MPO)
  tdvp      MPS, environments, H_eff,2 / H_eff,1 application
            (Eqs. one-site Hamiltonian 1, two-site Hamiltonian), Krylov
            exponential (Eq. Krylov subspace), truncated split (Sec. 2.1.1,
            DBSS), the symmetric 2TDVP sweep (Sec. 2.1.2) and observables
  global_krylov  MPO x MPS application, MPS compression and sums, the global
            Krylov time step and pre-steps before one-site TDVP (Sec. 2.1.2)
  gradient  dP_k(t)/dg of the populations with respect to the linear
            couplings (Duhamel formula in the eigenbasis; tiny systems)

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: dense projections, library routines (scipy expm/eigh/SVD), closed
forms and exact state-vector propagation.
"""
