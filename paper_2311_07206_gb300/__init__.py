"""GB300 (sm_103a) adaptive spectral deferred correction for P1 finite-element
monodomain systems with Aliev-Panfilov kinetics.

The compute path is the CUDA library ``libsdc_gb300.so`` (C ABI in
``include/sdc.h``); this package is its thin ctypes binding plus the build
script.  Importing the package does not load the library; ``binding.load()``
does, and raises if the library has not been built.
"""

from .binding import (  # noqa: F401
    Batch,
    Context,
    SdcError,
    default_options,
    load,
    radau,
    sdc_stats,
)

__all__ = ["Batch", "Context", "SdcError", "default_options", "load", "radau", "sdc_stats"]
