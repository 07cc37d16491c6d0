"""DNN-MG fine-level correction step on one GB300 GPU.

The hot path (prolongation, residual and patch features, GRU patch network,
averaging, right-hand side and restriction; the correction step of Algorithm 2 of
arXiv 2008.11520) is hand-written CUDA for sm_103a in ``csrc/`` behind the C
ABI of ``include/dnnmg.h`` (``libdnnmg.so``).  ``dnnmg`` is its thin ctypes
binding, ``synth`` the seeded synthetic inputs, ``build`` the nvcc build.
Import ``paper_2008_11520_gb300.dnnmg`` explicitly: it needs torch and the
built library and fails loudly without them.
"""

from . import synth  # noqa: F401
