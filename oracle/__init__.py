"""FP64 CPU oracle for the recursive moving-PML sweeping preconditioner.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, step-by-step
restatement of Liu & Ying, "Recursive Sweeping Preconditioner for the 3D
Helmholtz Equation" (arXiv 1502.07266) in complex double precision.  Only the
test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  The CUDA library never calls it and shares no code with it: the
two meet only through the seeded inputs of
``paper_1502_07266_gb300.workloads``.

Modules
  operator  PML profile (Section 2), the 7-point nonsymmetric scheme (Eq.
            system) assembled on an arbitrary box, and its matrix-free form.
  sweep     moving-PML auxiliary problems, the quasi-1D block LDU
            (Section 3 recursion applied along x1), Algorithm 3/4 (inner
            sweep along x2), Algorithm 5/6 (outer sweep along x3), and the
            non-recursive Algorithm 2 with exact quasi-2D solves.
  exact     the exact block LDU of Section 3 with dense plane blocks and the
            half-space Green's-function identity.
  krylov    right-preconditioned restarted GMRES (Section 4 solver).
  adjoint   transpose identity and the velocity gradient.

Every reading of the paper that is not fixed by the text is stated in the
docstring of the function that makes it.
"""
