"""GB300-native fast Jacobi polynomial transforms (Bremer, Pang and Yang, arXiv:1901.07275).

``Transform`` applies the forward, adjoint and inverse d-dimensional transforms
through libjt, a C-ABI library of hand-written sm_103a kernels (``include/jt.h``);
``binding`` is the same ABI with its C names; ``build`` compiles the library in-tree.
"""

from .transform import Batch, Transform, jacobi_fn  # noqa: F401

__all__ = ["Batch", "Transform", "jacobi_fn"]
