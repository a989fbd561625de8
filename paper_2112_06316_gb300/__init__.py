"""GB300-native IFGF-accelerated combined-field (CFIE) operator.

The hot path of Jimenez, Bauinger & Bruno's IFGF-accelerated CFIE solver: the
apply of the discrete combined-field operator that GMRES calls once per
iteration, as hand-written sm_103a CUDA behind the C ABI of ``include/ifgf.h``.
Python only marshals arguments (``binding``); PyTorch supplies device memory
and streams.
"""
from .binding import (  # noqa: F401
    FP64,
    LAYER_COMBINED,
    LAYER_DOUBLE,
    LAYER_SINGLE,
    MIXED,
    Group,
    IFGFError,
    IFGFOperator,
    Params,
    Plan,
    lib,
    rp_correction,
    supported_orders,
)
from .autograd import IFGFApply, ifgf_apply  # noqa: F401
