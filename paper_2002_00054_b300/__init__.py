"""B300 (sm_103a) Behler-Parrinello neural-network potential hot path (arXiv 2002.00054).

The compute path is the CUDA library libnnp.so (C ABI in include/nnp.h); this
package is its thin Python binding.  ``NNP`` is imported lazily so that the
build script can run without torch.
"""


def __getattr__(name):
    if name == "NNP":
        from .nnp import NNP
        return NNP
    if name == "NNPError":
        from ._capi import NNPError
        return NNPError
    raise AttributeError(name)
