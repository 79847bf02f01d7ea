"""Plain FP64 CPU oracle for state-averaged PNO-EOM-CCSD (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  The product (the CUDA library and its Python binding) never imports
it, and it shares no code with the product: the only common module is the
seeded input generator, which holds none of the method's arithmetic.

Modules
-------
hamiltonian   integrals from density-fitting factors, HF-consistent one-electron
              operator, T1 dressing of the Hamiltonian
bruteforce    determinant-space Hamiltonian, similarity transform, FCI/CISD
ccsd          closed-shell CCSD residual, CCSD solver, MP1 amplitudes
eom           EOM-CCSD sigma: Jacobian-vector definition and explicit terms
pno           CIS, CIS(D) doubles, state-averaged pair densities, PNOs/OSVs,
              projector and packed PNO vector layout
davidson      non-symmetric Davidson solver with the PNO-space preconditioner
pno_direct    the PNO-space sigma evaluated pair by pair from projected blocks and DF
              factors, without canonical R2/sigma2 or three- and four-virtual integrals
              ("O2"; pinned against pno.PNOSigma)

Parity status: every function here is pinned by a test under ``tests/``
against brute force, a closed form, an invariant or a textbook special case,
except the truncation-trend checks (reported only).
"""
