"""FP64 CPU oracle for the unitary-matrix simulation method (test infrastructure).

This package is test infrastructure, not part of the product: only the test
suite, the smoke check and the bench's CPU-baseline / reference leg may import
it.  It shares no code with the CUDA path and imports nothing from it.

It is plain numpy in complex128 and follows the paper step by step:

* ``gates``       - gate matrices: Table 1 (H, X, Y, Z, R_phi), S and T
                    (named in Sec. 5.2), the controlled form of eq. 7 / eq. 8,
                    the textbook rotations used by the synthetic workloads, and
                    custom k-qubit unitaries (Sec. 5.2 operation interface).
* ``kron_route``  - the unitary-matrix method itself: circuit steps (Sec. 5.2),
                    the step unitary as a Kronecker product of the step's
                    factors (Algorithm 2, eq. 9s1) with controlled gates as
                    projector sums (eq. 7), the per-step matrix-vector product
                    (eq. 11) and the circuit-unitary chain (Algorithm 1).
* ``fsv_route``   - the independent per-gate state-vector update of eq. 12
                    (Appendix A), used to cross-check the method and to compute
                    columns of large circuit unitaries.
* ``observables`` - probabilities |amplitude|^2, their sum, and marginals.
* ``collapse``    - simulateAndCollapse (Sec. 5.2): inverse-CDF sampling of an
                    outcome from the probabilities, and the measure / reset
                    instructions of the operation interface.

Every function is pinned by the tests under ``tests/test_oracle_*.py``
against values the paper prints, closed forms and brute force.
"""
