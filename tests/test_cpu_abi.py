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


def test_static_knn_validation_before_any_cuda_call(lib):
    """svf_knn_static answers bad arguments with SVF_EINVAL and a message on
    both error paths, before it touches a device (none exists here)."""
    from paper_2601_08528_b300 import _lib as L
    cap = lib.svf_knn_static_capacity()
    assert cap == 1 << 20
    P = C.c_void_p(16)  # never dereferenced: every case below fails validation first
    cases = [
        dict(n=0), dict(d=100), dict(d=0), dict(k=0), dict(k=129), dict(dtype=L.BF16), dict(metric=5),
        dict(nq=cap // 128 + 1, k=128), dict(nq=cap // 10 + 1), dict(X=None), dict(Q=None), dict(out=None), dict(nq=-1),
    ]
    for c in cases:
        a = dict(X=P, n=100, d=16, dtype=L.F32, metric=L.L2, Q=P, nq=4, k=10, out=P)
        a.update(c)
        rc = lib.svf_knn_static(a["X"], a["n"], a["d"], a["dtype"], a["metric"], a["Q"], a["nq"], None, a["k"],
                                a["out"], None, None)
        assert rc == L.SVF_EINVAL, c
        msg = lib.svf_knn_static_error()
        assert msg.startswith(b"svf_knn_static: "), c
        assert lib.svf_last_error() == msg, c
    assert b"exceeds" in (lib.svf_knn_static(P, 100, 16, 0, 0, P, cap // 128 + 1, None, 128, P, None, None)
                          and lib.svf_knn_static_error())
    # an empty batch is a no-op that needs no pointers
    assert lib.svf_knn_static(None, 100, 16, 0, 0, None, 0, None, 10, None, None, None) == L.SVF_OK


def test_gather_probe_validation_before_any_cuda_call(lib):
    """svf_gather_probe answers bad arguments with SVF_EINVAL before touching
    the device (the pointers below are never dereferenced)."""
    from paper_2601_08528_b300 import _lib as L
    P = 0x10000  # 16-byte aligned, never read: every case fails validation first
    st = C.c_int64(0)
    ms = C.c_float(0.0)
    cases = [dict(table=None), dict(table=P + 8), dict(pitch=100), dict(row_bytes=8), dict(row_bytes=144),
             dict(row_bytes=2048, pitch=2048), dict(n=0), dict(n=1 << 31), dict(rows=0), dict(warps=2),
             dict(warps=6), dict(warps=68), dict(status=None)]
    for c in cases:
        a = dict(table=P, n=1000, pitch=128, row_bytes=112, rows=1000, warps=24, status=P)
        a.update(c)
        rc = lib.svf_gather_probe(a["table"], a["n"], a["pitch"], a["row_bytes"], a["rows"], a["warps"], 1,
                                  a["status"], C.byref(st), C.byref(ms), None)
        assert rc == L.SVF_EINVAL, c
