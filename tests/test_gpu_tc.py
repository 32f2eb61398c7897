"""Tensor-core (tcgen05) exact kNN against the SIMT scan and the oracle."""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def svf():
    import paper_2601_08528_b300 as svf
    svf.load()
    return svf


@pytest.mark.parametrize("mix,metric,n,nq,k", [("unit96", "ip", 5000, 300, 10), ("tiny", "l2", 7001, 129, 10),
                                               ("unit96", "ip", 40000, 1000, 32), ("serve128", "l2", 20011, 300, 10),
                                               # past the seed-pass threshold (2^17 rows), ragged last tile
                                               ("unit96", "ip", 200003, 300, 10), ("serve128", "l2", 150001, 200, 10)])
def test_tc_knn_equals_oracle(svf, orc, mix, metric, n, nq, k):
    X = synth.sample(mix, n, 801)
    Q = synth.sample(mix, nq, 802)
    ids, dist, fb = svf.knn_tc(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), k, metric)
    st = orc.Store.from_vectors(X, metric)
    oi, od, og = orc.knn(st, Q, k)
    gi = P.as_u32(ids.cpu().numpy())
    same = (gi == oi).all(1)
    assert not (~same & (og > P.TOL)).any(), f"{(~same & (og > P.TOL)).sum()} unambiguous queries differ"
    sc = P.dist_scale(X, Q, oi.astype(np.int64), metric)
    assert (np.abs(dist.cpu().numpy()[same] - od[same]) <= P.TOL * sc[same]).all()
    assert fb <= 0.1 * nq, fb  # queries the certificate sent to the SIMT scan


@pytest.mark.parametrize("mix,metric,n,nq,k", [
    ("tiny", "l2", 1, 3, 10),       # a single row: one real result, the rest padded
    ("tiny", "l2", 5, 17, 10),      # fewer rows than k
    ("tiny", "l2", 300, 1, 32),     # one query, the largest k
    ("serve128", "l2", 1000, 5, 32),  # the largest dimension (128)
    ("unit96", "ip", 257, 130, 1),  # ragged row and query tiles, k = 1
])
def test_tc_knn_edge_cases(svf, orc, mix, metric, n, nq, k):
    X = synth.sample(mix, n, 811)
    Q = synth.sample(mix, nq, 812)
    ids, dist, _ = svf.knn_tc(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), k, metric)
    oi, od, og = orc.knn(orc.Store.from_vectors(X, metric), Q, k)
    gi = P.as_u32(ids.cpu().numpy())
    real = min(n, k)
    assert (gi[:, real:] == 0xFFFFFFFF).all() and np.isinf(dist.cpu().numpy()[:, real:]).all()
    same = (gi[:, :real] == oi[:, :real]).all(1)
    assert not (~same & (og > P.TOL)).any()
    sc = P.dist_scale(X, Q, oi[:, :real].astype(np.int64), metric)
    assert (np.abs(dist.cpu().numpy()[same, :real] - od[same, :real]) <= P.TOL * sc[same]).all()


def test_tc_knn_empty_and_invalid(svf):
    X = torch.from_numpy(synth.sample("tiny", 100, 821)).cuda()
    ids, dist, fb = svf.knn_tc(X, X[:0], 10, "l2")
    assert ids.shape == (0, 10) and fb == 0
    with pytest.raises(Exception):
        svf.knn_tc(X, X[:4], 33, "l2")  # k above 32
    with pytest.raises(Exception):
        svf.knn_tc(X[:, :15].contiguous(), X[:4, :15].contiguous(), 10, "l2")  # d not a multiple of 16
