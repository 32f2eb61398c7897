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
