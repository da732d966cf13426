"""GB300-native B-KFAC preconditioning hot path (arXiv 2210.08494).

``bkfac`` is the ctypes binding of the C-ABI library ``libbkfac.so``
(``include/bkfac.h``), built in-tree by ``build``.  ``synth`` draws the seeded
synthetic inputs.  Importing the package does not load the CUDA library; the
first call into ``bkfac`` does (and raises if it cannot).
"""

__all__ = ["bkfac", "build", "synth"]
