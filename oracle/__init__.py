"""FP64 CPU oracle for the nonrigid SENSE operator (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow, obviously-correct reference that the CUDA
path is checked against.  Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
library under ``paper_2501_16713_gb300`` never does, and it shares no code with
that library (no kernels, tables, helpers or constants).

Every function follows a passage of Jang, Malave & Nishimura, "Image-Space
Gridding for Nonrigid Motion-Corrected MR Image Reconstruction"
(arXiv 2501.16713), cited by section and equation:

* kernel.py     - the interpolation kernel c and its Fourier transform C
                  (Notations table; deapodization, "k-space Gridding").
* operators.py  - k-space gridding and its inverse (Eqs. for the gridding
                  process and inverse gridding), image-space gridding T_j and
                  T_j^H (image-space gridding process diagrams), coil
                  sensitivities, the nonrigid SENSE operator A_j = G_j S T_j and
                  its adjoint, the stacked model (stacked SENSE equation).
* references.py - exact definitions the gridded operators approximate (the
                  displacement-field warp equation evaluated by trigonometric
                  interpolation, and the non-uniform DFT), closed forms for
                  constant and integer displacements, the rigorous aliasing
                  bound, and dense matrices built factor by factor.
* solvers.py    - conjugate gradients on the normal equations of the stacked
                  model with a Tikhonov term.

Readings of the paper where it is silent are stated where they are used.
"""

from .kernel import bessel_i0, bessel_i0m1, beatty_beta, kb_kernel, kb_kernel_ft  # noqa: F401
from . import operators, references, solvers  # noqa: F401
