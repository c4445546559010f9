"""CPU FP64 oracle for preconditioned MINRES on symmetrised BLTT systems (arXiv 2307.07749).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (neither imports the other); both take their inputs from ``workloads``.

Everything here is plain, slow and written to be checked against the paper by eye:

* ``operators``  - the BLTT operator A (eq. amatdef), the time reversal Y (Sec. 2), the Laplacian,
                   the DST-I matrix U and the eigenvalues of the blocks (Sec. 3), all from their
                   definitions; dense assembly for tiny sizes.  General commuting blocks given
                   as matrices (Assumption 1 (i)) get their common eigenbasis from one generic
                   combination of the blocks and their block sum as written.
* ``precond``    - the ABAC preconditioner P_alpha = |C_alpha| (Defs. 2-3, eqs. calphaabsdef,
                   precdef): a dense route (C_alpha assembled, principal square root by a Schur
                   method) and the paper's three-step structured route (Sec. 5.1).
* ``minres``     - textbook preconditioned MINRES (Elman-Silvester-Wathen, the solver the
                   convergence Lemma of Sec. 4.2 refers to), zero initial guess (Sec. 5.2).
* ``timestep``   - block forward substitution, the exact solution of A u = f.
* ``mlp``        - FP64 forward/backward/Adam of the 4-32-32-1 alpha predictor.

Every function's docstring cites the passage it follows.  Functions without an independent pin
say "parity unpinned" in their docstring.
"""
from .operators import (laplacian, laplacian_eigenvalues, dst1_matrix, apply_U, block_eigenvalues,
                        bltt_matvec, assemble_A, assemble_Y, assemble_C_alpha, assumption_margin)
from .precond import (alpha_circulant_eigs, precond_apply, precond_dense, sqrt_C_alpha_dense,
                      precond_apply_one_pass_alpha1)
from .minres import minres, solve
from .timestep import timestep_solve

__all__ = [
    "laplacian", "laplacian_eigenvalues", "dst1_matrix", "apply_U", "block_eigenvalues",
    "bltt_matvec", "assemble_A", "assemble_Y", "assemble_C_alpha", "assumption_margin",
    "alpha_circulant_eigs", "precond_apply", "precond_dense", "sqrt_C_alpha_dense",
    "precond_apply_one_pass_alpha1", "minres", "solve", "timestep_solve",
]
