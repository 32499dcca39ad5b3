"""GB300 (sm_103a) ADER-DG / ADER-WENO hot path for the 1D Euler equations.

The compute path is the CUDA library libader_gb300.so behind the C ABI of
include/ader.h; ``capi.Context`` is its thin Python binding (torch supplies the
device memory and the stream).
"""
from .capi import (ADER_ERR_ARG, ADER_ERR_CUDA, ADER_ERR_NOMEM, ADER_ERR_NONPHYSICAL,  # noqa: F401
                   ADER_ERR_NOT_CONVERGED, ADER_ERR_STATE, ADER_ERR_TIMEOUT, ADER_OK, AderError,
                   Context, Context2D, Context3D, default_options, exported_symbols, load)

__all__ = ["Context", "Context2D", "Context3D", "AderError", "load", "default_options", "exported_symbols"]
