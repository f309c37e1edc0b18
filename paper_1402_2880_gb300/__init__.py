"""GB300 (sm_103a) sparse SCF hot path: libsscf and its Python binding.

The compute path is the CUDA library ``libsscf.so`` built from ``csrc/`` by
``build.build()``; ``Context`` marshals arguments to its C-ABI. There is no
CPU fallback: using the package without the built library raises.
"""
from ._lib import (  # noqa: F401
    SSCF_FP64,
    SSCF_MIXED,
    SSCF_ORTHO_ALL,
    SSCF_ORTHO_OCC,
    Context,
    SscfError,
    group_molecules,
    load,
)
