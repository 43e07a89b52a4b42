"""CPU oracle of the CT-AUX submatrix-update hot path.

TEST INFRASTRUCTURE.  This package is a plain, slow, float64 restatement of
what the CUDA path computes, written from the paper (plain CT-AUX with dense
LU determinant ratios; see oracle/ctaux.py for the readings it follows), plus
exact diagonalisation (oracle/ed.py) that pins it.  Only tests/,
__graft_entry__.smoke() and the CPU-baseline leg of bench.py may import it.
The product path (paper_1010_3690_gb300) never imports, links or runs it, and
the two share no code; the only shared module is the seeded input generator
package `workloads`, which holds none of the method's arithmetic.
"""
