"""GB300-native tensor-product--Thomas Poisson/Helmholtz solver (CUDA, sm_103a).

The compute path lives in libtpt.so (csrc/, C ABI in include/tpt.h); this
package is its Python binding.  Attribute access loads the library and raises
ImportError when it has not been built (there is no CPU fallback); the
``build`` submodule works without it.
"""
_EXPORTS = ("Plan", "Batch", "Cache", "Server", "make_desc", "grid_tanh", "field_to_device", "field_to_host", "AUTO", "GEMM", "FFT",
            "PERIODIC", "NEUMANN", "DIRICHLET", "DIRICHLET_NODE", "NONE", "grid_faces", "FP64", "MIXED_BF16", "MIXED_BF16X3", "MIXED_TF32")
__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
