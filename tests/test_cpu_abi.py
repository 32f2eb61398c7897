"""CPU-only checks of the C-ABI library: it loads without a GPU, exports every
function include/svf.h declares, and its host-side validation answers with
the documented error codes (no kernel is launched)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "svf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(svf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_08528_b300 import build
    build.build()
    from paper_2601_08528_b300 import _lib
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_2601_08528_b300 import _lib
    assert set(_lib.SYMBOLS) <= set(names)


def test_buffer_sizes_and_validation(lib):
    from paper_2601_08528_b300 import _lib as L
    p = L.Params(96, L.F32, L.IP, 32, 1_000_000, L.PRUNE_RNG, 8, 3, 0, 1)
    s = L.Sizes()
    assert lib.svf_buffer_sizes(C.byref(p), 10_000, C.byref(s)) == 0
    assert s.vecs == 1_000_000 * 96 * 4
    assert s.vecs_bf16 == 1_000_000 * 96 * 2
    assert s.vecs_fp8 == 1_000_000 * 128
    assert s.graph == 1_000_000 * 32 * 4
    assert s.del_bits >= 1_000_000 // 8 and s.workspace > 0 and s.status >= 64 * 8
    for bad in (dict(d=100), dict(R=48), dict(n_cap=1 << 30), dict(repair_c=17), dict(dtype=L.U8, lowp=1),
                dict(metric=7)):
        q = L.Params(96, L.F32, L.IP, 32, 1000, L.PRUNE_RNG, 8, 0, 0, 1)
        for k, v in bad.items():
            setattr(q, k, v)
        assert lib.svf_buffer_sizes(C.byref(q), 10, C.byref(s)) == L.SVF_EINVAL
        assert lib.svf_last_error()


def test_null_and_size_checks_before_any_launch(lib):
    from paper_2601_08528_b300 import _lib as L
    assert lib.svf_search(None, None, 0, None, None, None, None) == L.SVF_EINVAL
    assert lib.svf_insert(None, None, 5, 64, 32, None, None) == L.SVF_EINVAL
    assert lib.svf_knn(None, 10, 100, 0, 0, None, 5, None, 10, None, None, None, None) == L.SVF_EINVAL
    assert lib.svf_mlp_partial_floats(4096) == 16 * 1154
    assert lib.svf_mlp_grad(None, None, 8, None, 10, None, None, None, None, None) == L.SVF_EINVAL


def test_oracle_and_library_share_no_code():
    """The oracle (test infrastructure) and the CUDA path are separate: no
    file of one includes or imports the other."""
    pkg = os.path.join(ROOT, "paper_2601_08528_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include)\s+\S*", txt).__str__(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2601_08528_b300" not in txt and "svf.h" not in txt, f
