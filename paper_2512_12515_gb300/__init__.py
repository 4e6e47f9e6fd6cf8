"""GB300-native (sm_103a) particle-particle RPA hot path.

The computation lives in ``libpprpa_gb300.so`` (hand-written CUDA behind a
C ABI, see include/pprpa.h); this package only marshals arguments.
Importing it loads the library and fails loudly when it has not been built.
"""
from ._lib import (  # noqa: F401
    AB,
    CHANNEL_HH,
    CHANNEL_PP,
    Context,
    DEVICE,
    HOST,
    METHOD_DAVIDSON,
    METHOD_FULL,
    PREC_BF16,
    PREC_BF16_SPLIT,
    PREC_FP64,
    PREC_FP8,
    PprpaError,
    SINGLET,
    TRIPLET,
    kernel_launches,
    load,
)

load()

from .autograd import PPRPARoots  # noqa: E402,F401
