"""GB300 (sm_103a) runtime for stencil programs in the style of the Open Earth
Compiler paper: parse a stencil program (paper §IV), infer its ranges (§V-B),
and run it as fused or stage-by-stage CUDA kernels behind the C ABI of
liboec (include/oec.h). The CUDA library is required; there is no CPU path.
"""

from . import programs  # noqa: F401  (program texts; no compute)


def __getattr__(name):
    # the binding is imported lazily so that `inputs` and `programs` load
    # without the CUDA library
    if name in ("Program", "Field", "Batch", "device_field"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
