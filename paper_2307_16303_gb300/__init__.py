"""GB300-native HODLR3D kernel-matrix product (arXiv 2307.16303).

The compute path is the CUDA library ``libh3d.so`` (C ABI in ``include/h3d.h``);
``paper_2307_16303_gb300.api`` is a thin ctypes binding over it.  Importing this
package does not load the library; the binding does, and fails loudly when the
library has not been built.
"""

__all__ = ["api", "inputs"]
