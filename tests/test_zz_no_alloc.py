"""svf_knn_static: the allocation-free kNN entry point (collected last).

Callers that cannot call cudaMalloc (a plugin inside a framework that owns
the device memory, a latency-critical loop) use svf_knn_static, whose scratch
is a fixed device array inside the library.  Its output must equal svf_knn's
(which uses a caller-allocated buffer) on two calls in a row: the second call
reuses the array and must not see the first call's keys.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _static_fn():
    import paper_2601_08528_b300 as svf
    lib = svf.load()
    f = lib.svf_knn_static
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    f.restype = I32
    f.argtypes = [P, I64, I32, I32, I32, P, I64, P, I32, P, P, P]
    lib.svf_knn_static_error.restype = C.c_char_p
    lib.svf_knn_static_capacity.restype = I64
    return svf, lib, f


def _p(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("mix,metric,k", [("u8", "l2", 10), ("unit96", "ip", 32)])
def test_static_knn_matches_allocating_knn_twice(mix, metric, k):
    svf, lib, f = _static_fn()
    assert lib.svf_knn_static_capacity() == 1 << 20
    X = torch.from_numpy(synth.sample(mix, 6000, 501)).cuda()
    dt = 1 if mix == "u8" else 0
    mt = 1 if metric == "ip" else 0
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (nq, seed) in enumerate([(333, 502), (97, 503)]):
        Q = torch.from_numpy(synth.sample(mix, nq, seed)).cuda()
        ref_ids, ref_d = svf.knn(X, Q, k, metric)
        ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
        dist = torch.empty_like(ref_d)
        rc = f(_p(X), X.shape[0], X.shape[1], dt, mt, _p(Q), nq, None, k, _p(ids), _p(dist), stream)
        assert rc == 0, lib.svf_knn_static_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_ids.cpu().numpy(), err_msg=f"call {call}")
        if dt == 1:
            np.testing.assert_array_equal(dist.cpu().numpy(), ref_d.cpu().numpy())
        else:
            np.testing.assert_allclose(dist.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_static_knn_rejects_oversized_batches():
    svf, lib, f = _static_fn()
    X = torch.zeros((100, 16), dtype=torch.float32, device="cuda")
    Q = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    ids = torch.empty((1, 128), dtype=torch.int32, device="cuda")
    rc = f(_p(X), 100, 16, 0, 0, _p(Q), (1 << 20) // 128 + 1, None, 128, _p(ids), None, None)
    assert rc == -1 and b"exceeds" in lib.svf_knn_static_error()
