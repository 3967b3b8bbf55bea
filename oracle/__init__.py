"""CPU FP64 oracle (test infrastructure only).

Only the tests, the smoke check (`__graft_entry__.smoke`) and the benchmark's CPU
baseline leg may import this package.  It is a plain, slow, independently written
restatement of what the CUDA path computes; it shares no code with it.

Parity status: every function here is pinned by the CPU tests in
tests/test_oracle_pins.py against closed forms, invariants, brute force or
convergence rates; none is "parity unpinned".
"""
from .fem_oracle import *  # noqa: F401,F403
from .fem_oracle import (MASS, DIFFUSION, HexGridMesh, HexMesh, hex_numbering, Problem, Rule3D, rule, gauss_legendre, gll_points,
                         lagrange, elem_dofs, boundary_dofs, num_dofs, node_coords, trilinear, qp_factors,
                         element_matrices, assemble_csr, constrain, action_elementwise, action_rows,
                         diagonal_elementwise, qp_coords, rhs_from_qp, sine_solution, sine_source, jacobi_pcg,
                         l2_error, dense_bruteforce, elements_of_dof)
