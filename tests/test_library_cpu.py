"""CPU-side checks of the C-ABI library: it builds, loads, exports every
entry point that include/curid.h declares, and rejects bad arguments on the
host before touching a GPU.  Also pins the numpy Philox reference."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import paper_1412_8447_gb300 as curid
from paper_1412_8447_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_8447_gb300.build import build
    build()
    return curid.load_library()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^curid_status\s+(curid_\w+)\s*\(", txt, re.M))
    return names


def test_header_symbols_exported(lib):
    names = declared_symbols()
    assert len(names) >= 13
    for n in sorted(names):
        assert hasattr(lib, n), n
    # the binding's signature table covers every declared entry point
    assert names <= set(B.SIGNATURES)


def test_null_handle_rejected_on_host(lib):
    vp = ctypes.c_void_p
    assert lib.curid_set_stream(None, None) == B.INVALID_ARG
    assert lib.curid_set_workspace(None, None, 0) == B.INVALID_ARG
    assert lib.curid_last_status(None, None) == B.INVALID_ARG
    assert lib.curid_create(None, 0) == B.INVALID_ARG
    sk = B.Sketch(-1, 0, 0, None, 0)
    assert lib.curid_id_col(None, 0, vp(1), 10, 10, 10, 2, 0.0, sk, vp(1), vp(1), 8) == B.INVALID_ARG
    assert lib.curid_cur(None, 0, vp(1), 10, 10, 10, 2, 0.0, sk, vp(1), vp(1), vp(1), None, None,
                         None, 0, None, 0) == B.INVALID_ARG
    b = ctypes.c_size_t(0)
    assert lib.curid_workspace_size(None, 0, 10, 10, 2, sk, ctypes.byref(b)) == B.INVALID_ARG
    assert lib.curid_srft_omega(None, 1, 10, 4, vp(1), vp(1), vp(1), 10) == B.INVALID_ARG
    assert lib.curid_srft_draw(None, 10, 4, 1, vp(1), vp(1)) == B.INVALID_ARG
    assert lib.curid_cur_corrected(None, 0, vp(1), 10, 10, 10, 2, 0.0, sk, vp(1), vp(1), vp(1),
                                   None, None, None, 0, None, 0) == B.INVALID_ARG
    assert lib.curid_interp_tikhonov(None, 0, vp(1), 10, vp(1), 10, 2, 0.5, vp(1), 8) \
        == B.INVALID_ARG
    assert lib.curid_interp_tsvd(None, 0, vp(1), 10, vp(1), 10, 2, 1e-3, vp(1), 8) \
        == B.INVALID_ARG
    assert lib.curid_interp_tikhonov_workspace_size(None, 0, 10, 2, ctypes.byref(b)) \
        == B.INVALID_ARG
    assert lib.curid_interp_tsvd_workspace_size(None, 0, 10, 2, ctypes.byref(b)) \
        == B.INVALID_ARG
    sp = B.Sparse(0, vp(1), None, None, vp(1), None, None)
    sk1 = B.Sketch(5, 0, 0, None, 0)
    assert lib.curid_sparse_workspace_size(None, 0, 10, 10, 2, sk1, ctypes.byref(b)) \
        == B.INVALID_ARG
    assert lib.curid_cur_sparse(None, 0, 10, 10, ctypes.byref(sp), 2, sk1, 0, vp(1), vp(1),
                                vp(1), None, None, None, 0, None, 0) == B.INVALID_ARG
    assert lib.curid_complex_workspace_size(None, 0, 10, 10, 2, sk, ctypes.byref(b)) \
        == B.INVALID_ARG
    assert lib.curid_cur_complex(None, 0, vp(1), 10, 10, 10, 2, sk, vp(1), vp(1), vp(1), None,
                                 0) == B.INVALID_ARG
    assert lib.curid_srft_sketch(None, 1, vp(1), 10, 10, 10, 4, vp(1), vp(1), vp(1), 10) \
        == B.INVALID_ARG


def test_sketch_struct_matches_header():
    """The binding's curid_sketch has the header's fields in the header's
    order (the structure is passed by value through the C ABI)."""
    txt = open(os.path.join(ROOT, "include", "curid.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} curid_sketch;", txt).group(1)
    names = re.findall(r"(\w+)\s*;", body)
    assert names == [f[0] for f in B.Sketch._fields_]
    # int, int, uint64, pointer, int (+ padding), pointer, pointer on LP64
    assert ctypes.sizeof(B.Sketch) == 48


def test_philox_known_answers():
    from oracle.philox import philox4x32_10
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "philox_kat.json")))
    for v in g["vectors"]:
        c = np.array([[int(x, 16) for x in v["ctr"]]], dtype=np.uint64)
        out = philox4x32_10(c, [int(x, 16) for x in v["key"]])[0]
        assert ["%08x" % x for x in out] == v["out"]


def test_philox_gaussian_moments():
    from oracle.philox import gaussian
    z = gaussian(400, 500, 12345).ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.05
