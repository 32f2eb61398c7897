"""Failure handling on the GPU without a fault: every device wait in the
library is a bounded poll of an mbarrier.  A warp waits on a barrier nothing
arrives at; the wait must give up, report SVF_ETIMEOUT through the status
words, and leave the context usable for the next call."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def svf():
    import paper_2601_08528_b300 as svf
    svf.load()
    return svf


def test_bounded_wait_reports_timeout_and_context_survives(svf, orc):
    from paper_2601_08528_b300 import _lib as L
    lib = L.load()
    status = torch.zeros(2, dtype=torch.int64, device="cuda")
    secs = C.c_double(0.0)
    polls = 1 << 16
    rc = lib.svf_selftest_wait_timeout(polls, status.data_ptr(), C.byref(secs),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.SVF_ETIMEOUT
    st = status.cpu().numpy()
    assert st[0] == -L.SVF_ETIMEOUT and st[1] == polls + 1  # error code, then the poll count at which it gave up
    # the production limit stays a bounded wait: report its scale from this run
    assert lib.svf_wait_limit() >= polls
    assert secs.value < 60.0
    print(f"bounded wait: {polls} polls gave up after {secs.value * 1e3:.2f} ms; the library's limit of "
          f"{lib.svf_wait_limit()} polls scales to about {secs.value * lib.svf_wait_limit() / polls:.2f} s")
    # the context is intact: a search right after matches the oracle
    X = synth.sample("tiny", 2000, 901)
    Q = synth.sample("tiny", 50, 902)
    st_o = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st_o, 32)
    ix = svf.Index(X.shape[1], 2000, dtype="f32", metric="l2", R=32, max_batch=2000)
    ix.attach(torch.from_numpy(X).cuda(), torch.from_numpy(g.view(np.int32)))
    ids, _ = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=64, T=32, seed=4))
    o = orc.search(st_o, 2000, g, None, Q, 10, 64, 32, 4)
    same = (ids.cpu().numpy().astype(np.int64) == o["ids"].astype(np.int64)).all(1)
    assert same.mean() >= 0.9
