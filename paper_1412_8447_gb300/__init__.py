"""GB300 (sm_103a) CUR and interpolative decompositions of Voronin &
Martinsson (arXiv:1412.8447).

The computation lives in ``libcurid.so`` (hand-written CUDA kernels behind the
C ABI of ``include/curid.h``); this package is its thin Python binding.
"""
from ._binding import (  # noqa: F401
    BatchedID, CURFunction, CuridError, HostStream, LIB_PATH, PHASES, Result, STATUS_NAMES, Srft,
    cpqr,
    inflight, set_concurrency, set_timeout,
    cur, cur_adjoint, cur_complex, cur_differentiable, cur_outputs, cur_sparse, gaussian, id_col, id_row,
    interp_tikhonov, interp_tsvd, last_status, load_library, profile, profile_read, sketch_matrix,
    sparse_operand, srft_draw, srft_omega, srft_sketch, tsid,
)
