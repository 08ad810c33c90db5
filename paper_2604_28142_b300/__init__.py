"""B300 (sm_103a) gather-and-refine scoring for multivector retrieval.

The compute runs in the CUDA library `libtachiom.so` built from `csrc/`; this
package only marshals arguments to its C ABI (include/tachiom.h). There is no
CPU fallback: loading fails loudly if the library is missing.
"""
from .binding import (  # noqa: F401
    PREC_BF16,
    PREC_FP8,
    PREC_FP32,
    FLAG_CAPACITY,
    FLAG_SELECT_TIES,
    FLAG_TOPC_RESCUED,
    TachiomError,
    Index,
    Server,
    SearchParams,
    lib,
    lib_path,
    profile_enable,
    pq_encode,
    pq_train,
    profile_read,
    tac_allot,
    tac_cluster,
    tc_available,
)
