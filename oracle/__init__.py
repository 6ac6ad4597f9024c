"""Plain CPU oracle for the discrete Jacobi polynomial transform (arXiv:1901.07275).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA library (no kernels, headers, tables or helpers); the two meet only on
seeded inputs produced by ``paper_1901_07275_gb300.synthetic``.

It computes the *definition* of the transform directly -- no phase functions,
no low-rank factorisation and no FFT -- so that every fast result has a plain,
checkable reference:

* orthonormal Jacobi polynomials by the three-term recurrence of the Jacobi
  matrix (the polynomials behind the modified functions of Sec. 1, Eq.
  ``eq:modifiedjac``);
* Gauss--Jacobi nodes and Christoffel weights (Sec. 1, Eqs. ``eq:GJquadrule``
  and ``introduction:modrule``);
* the weighted uniform matrix ``W J`` (Sec. 3.1, Eqs. ``tf:transout``,
  ``tf:transexp``), the unweighted nonuniform ``J`` (Sec. 3.1, end), and
  their d-dimensional tensor products (Sec. 3.2--3.3, Eqs. ``eq:2Djac``,
  ``eq:3Djac``) applied by dense mode products.

The second-kind functions ``Q~`` (Sec. 1, Eq. ``eq:jacnonosci2``) for the second-kind
transform are in ``second_kind.py``: the Stieltjes transform of the weight by adaptive
quadrature and the same three-term recurrence under the principal-value integral.

Recurrences and Newton iterations run in ``numpy.longdouble`` (80-bit extended
on x86-64, IEEE binary128 on aarch64); dense summations run in float64.
Every function is pinned by ``tests/test_oracle_pins.py`` against closed forms,
library routines and brute force.  No function here is "parity unpinned".
"""

from .jacobi import (  # noqa: F401
    recurrence_coefficients,
    orthonormal_jacobi,
    gauss_jacobi,
    gauss_jacobi_nodes_at,
    modified_jacobi,
    uniform_matrix,
    uniform_rows,
    nonuniform_matrix,
    axis_matrix,
    forward,
    adjoint,
    forward_sampled,
)
from .second_kind import (  # noqa: F401
    stieltjes,
    stieltjes_t,
    second_kind_h,
    modified_second_kind,
    uniform_matrix_q,
    nonuniform_matrix_q,
    axis_matrix_q,
)
