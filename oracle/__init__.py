"""Plain CPU FP64 oracle for two-level additive Schwarz preconditioned GMRES
applied to the lowest-order Nedelec discretisation of
curl curl E - (k^2 + i xi) E = F on the unit cube with PEC boundary conditions
(Bonazzoli, Dolean, Graham, Spence, Tournier, arXiv:1711.03789).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import, call or execute anything in this
package. It shares no code with the CUDA path and never imports it.

Modules:
    mesh    -- uniform Kuhn mesh, edges, PEC-interior DOF numbering (Sec. 2.2, Eq. 1.4)
    fem     -- Whitney element matrices, assembly of K, M, A_xi, load vector (Eq. 2.2, Sec. 2.2)
    dd      -- subdomains, restriction R^l, minors, coarse space R^0, A^0, AS apply (Sec. 3, Eq. 3.1-3.4)
    gmres   -- right-preconditioned restarted GMRES with MGS Arnoldi and Givens rotations (Sec. 6.1)
    problem -- build / factor / solve, mirroring the library's three calls

Every function states the passage of the paper it follows. Where the paper is
silent the reading taken is stated in the docstring; all such readings are
collected in the design notes of the repository.

Parity pins (tests/test_oracle_*.py) tie each function to closed forms,
invariants, special cases and brute force; none compares the oracle with
itself.
"""
