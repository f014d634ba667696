"""CPU complex128 oracle for deflated multi-shift GMRES.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The CUDA library never calls it and has no fallback to it.

The oracle is plain and slow on purpose: numpy/scipy in complex128, no
blocking, fusion or reordering beyond what the paper's algorithms state, so it
can be checked against the paper by eye.  It shares no code with the CUDA path;
both are fed from ``workloads`` (seeded input generation only).

Contents
  operators  : CSR matvec and the Wilson-Dirac hopping operator (Sec. 4,
               Example 7; conventions fixed in the module docstring).
  krylov     : Arnoldi with classical Gram-Schmidt + one reorthogonalisation,
               GMRES-Sh (Sec. 2.1), harmonic Ritz vectors and GMRES-DR(m,k)-Sh
               (Sec. 2.2, Sec. 3), the Minres projection and GMRES(m)-Proj(k)
               (Sec. 2.3), GMRES-Proj-Sh with the extra right-hand side and the
               correction phase (Sec. 4), the projection over selected approximate
               eigenvectors (Sec. 4, Theorem 1, Example 4), related right-hand
               sides (Sec. 5).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute-force definitions on tiny inputs, dense LU, or
the paper's printed numbers; none is "parity unpinned".
"""
from .operators import CSROperator, WilsonOperator, gamma_matrices, gamma5  # noqa: F401
from .krylov import (  # noqa: F401
    arnoldi_cgs2_step,
    gmres_sh_dense_step,
    fom_sh_dense_step,
    ritz,
    harmonic_ritz,
    select_smallest,
    gmres_dr_sh,
    minres_projection,
    gmres_proj_sh,
    extra_rhs_solve,
    correct_solutions,
    related_rhs_projection,
    kept_eigenpairs,
    eigvec_projection,
    solve_all_rhs,
)
