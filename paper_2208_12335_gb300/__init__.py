"""GB300 (sm_103a) batched real-space grid integration for numeric
atom-centred orbitals: basis evaluation, H integration with sparse scatter,
density, adjoint.  The compute path is ``libfgi.so`` (hand-written CUDA);
this package only binds its C ABI (``include/fgi.h``)."""
from .fgi import (FGI_BF16, FGI_FP64, FGI_SPLIT_BF16, Context, FGIError, HIntegrate,  # noqa: F401
                  integrate, lib, load_library, SYMBOLS, LIB_PATH)
