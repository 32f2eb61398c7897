"""Precision forms (BF16 / FP8-E4M3 traversal, exact FP32 re-rank) and the
learned early stop, against the FP64 oracle (C ABI)."""
import ctypes as C

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


_cache = {}


def setup(orc, mix, n, R, metric, seed):
    key = (mix, n, R, metric, seed)
    if key not in _cache:
        X = synth.sample(mix, n, seed)
        st = orc.Store.from_vectors(X, metric)
        g, _ = orc.build_graph(st, R)
        _cache[key] = (X, st, g)
    return _cache[key]


def make_index(svf, X, g, metric, R, lowp=("bf16", "fp8")):
    ix = svf.Index(X.shape[1], X.shape[0], dtype="u8" if X.dtype == np.uint8 else "f32", metric=metric, R=R,
                   lowp=lowp if X.dtype != np.uint8 else (), max_batch=1000)
    ix.attach(torch.from_numpy(X).cuda(), torch.from_numpy(g.view(np.int32)))
    return ix


# ---------------------------------------------------------------- precision forms
@pytest.mark.parametrize("prec,metric,mix", [("bf16", "ip", "unit96"), ("fp8", "ip", "unit96"),
                                             ("bf16", "l2", "tiny"), ("fp8", "l2", "tiny")])
def test_lowp_traversal_parity(svf, orc, prec, metric, mix):
    X, st, g = setup(orc, mix, 3000, 32, metric, 601)
    Q = synth.sample(mix, 300, 602)
    ix = make_index(svf, X, g, metric, 32)
    lst = orc.Store.from_vectors(X, metric, dtype=prec)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=64, T=32, precision=prec, seed=4))
    o = orc.search(lst, 3000, g, None, Q, 10, 64, 32, 4)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), o, X, Q, metric)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_rerank_is_exact_fp32_over_the_final_pool(svf, orc, prec):
    X, st, g = setup(orc, "unit96", 3000, 32, "ip", 611)
    Q = synth.sample("unit96", 200, 612)
    ix = make_index(svf, X, g, "ip", 32)
    lst = orc.Store.from_vectors(X, "ip", dtype=prec)
    L = 64
    ids, dist = ix.search(torch.from_numpy(Q).cuda(),
                          svf.SearchConfig(k=10, L=L, T=32, precision=prec, rerank=True, seed=4))
    o = orc.search(lst, 3000, g, None, Q, 10, L, 32, 4, want_pool=True)
    # oracle: exact FP64 distances of the whole final pool, re-sorted by (dist, id)
    ref = P.rerank_ref(orc, st, Q, o, 10)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), ref, X, Q, "ip")


def test_lowp_recall_is_won_back_by_rerank(svf, orc):
    X, st, g = setup(orc, "unit96", 3000, 32, "ip", 611)
    Q = synth.sample("unit96", 300, 613)
    ix = make_index(svf, X, g, "ip", 32)
    ti, td, _ = orc.knn(st, Q, 10)
    rec = {}
    for name, cfg in {"fp32": svf.SearchConfig(k=10, L=128, T=64),
                      "fp8": svf.SearchConfig(k=10, L=128, T=64, precision="fp8"),
                      "fp8+rr": svf.SearchConfig(k=10, L=128, T=64, precision="fp8", rerank=True)}.items():
        ids, _ = ix.search(torch.from_numpy(Q).cuda(), cfg)
        gi = P.as_u32(ids.cpu().numpy())
        rec[name] = P.recall(gi, ti, td, orc.dist_ids(st, Q, gi))
    assert rec["fp8+rr"] >= rec["fp8"] and rec["fp8+rr"] >= rec["fp32"] - 0.01


# ---------------------------------------------------------------- learned stop
def _lib(svf):
    return svf.load()


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def test_trace_features_match_oracle(svf, orc):
    X, st, g = setup(orc, "u8", 4000, 64, "l2", 621)
    Q = synth.sample("u8", 100, 622)
    ix = make_index(svf, X, g, "l2", 64)
    T = 48
    feat = torch.zeros((100, T, 16), dtype=torch.float32, device="cuda")
    meta = torch.zeros((100, 2), dtype=torch.int32, device="cuda")
    ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=64, T=T, seed=8), trace_feat=feat,
              trace_meta=meta)
    o = orc.search_ex(st, 4000, g, None, Q, 10, 64, T, 8, trace=True)
    m = meta.cpu().numpy()
    np.testing.assert_array_equal(m[:, 0], o["n_feat"])
    np.testing.assert_array_equal(m[:, 1], o["t_last"])
    f = feat.cpu().numpy()
    for q in range(100):
        nf = o["n_feat"][q]
        np.testing.assert_allclose(f[q, :nf], o["feat"][q, :nf], rtol=2e-5, atol=2e-6)


def _fake_trace(seed, nq, T):
    rng = np.random.default_rng(seed)
    feat = rng.standard_normal((nq, T, 16)).astype(np.float32)
    ran = rng.integers(1, T + 1, nq)
    t_last = np.array([rng.integers(-1, r) for r in ran])
    meta = np.stack([ran, t_last], 1).astype(np.int32)
    ids = np.concatenate([q * T + np.arange(r) for q, r in enumerate(ran)]).astype(np.int32)
    return feat, meta, ids


def test_mlp_forward_backward_match_oracle(svf, orc):
    lib = _lib(svf)
    T = 20
    feat, meta, ids = _fake_trace(631, 300, T)
    rng = np.random.default_rng(632)
    batch = ids[rng.permutation(len(ids))[:2048]]
    prm = np.concatenate([rng.standard_normal(1024) * 0.3, rng.standard_normal(64) * 0.1,
                          rng.standard_normal(64) * 0.3, [0.05]]).astype(np.float32)
    net = orc.MLP(prm[:1024].reshape(64, 16), prm[1024:1088], prm[1088:1152], float(prm[1152]))
    q, t = batch // T, batch % T
    F = feat[q, t].astype(np.float64)
    y = (t >= meta[q, 1]).astype(np.float64)
    loss_o, g_o = orc.mlp_backward(net, F, y)
    z_o, _ = orc.mlp_forward(net, F)

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    f_d, m_d, b_d, p_d = dev(feat), dev(meta), dev(batch), dev(prm)
    grad = torch.empty(1153, dtype=torch.float32, device="cuda")
    part = torch.empty(int(lib.svf_mlp_partial_floats(len(batch))), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    assert lib.svf_mlp_grad(_p(f_d), _p(m_d), T, _p(b_d), len(batch), _p(p_d), _p(grad), _p(part), _p(loss),
                            None) == 0
    z = torch.empty(len(batch), dtype=torch.float32, device="cuda")
    Fd = dev(F.astype(np.float32))
    assert lib.svf_mlp_forward(_p(p_d), _p(Fd), len(batch), _p(z), None) == 0
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    go = np.concatenate([g_o["W1"].ravel(), g_o["b1"], g_o["w2"], [g_o["b2"]]])
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))
    assert abs(float(loss.item()) - loss_o) <= 1e-5 * max(1.0, abs(loss_o))
    np.testing.assert_allclose(z.cpu().numpy(), z_o, rtol=1e-5, atol=1e-5)
    # the same batch twice gives bit-identical gradients (fixed reduction order)
    g1 = grad.clone()
    lib.svf_mlp_grad(_p(f_d), _p(m_d), T, _p(b_d), len(batch), _p(p_d), _p(grad), _p(part), _p(loss), None)
    torch.cuda.synchronize()
    assert torch.equal(g1, grad)


def test_adam_step_and_pack(svf, orc):
    lib = _lib(svf)
    rng = np.random.default_rng(641)
    p0 = rng.standard_normal(1153).astype(np.float32)
    g = rng.standard_normal(1153).astype(np.float32)
    p, gr = torch.from_numpy(p0.copy()).cuda(), torch.from_numpy(g).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    assert lib.svf_mlp_adam(_p(p), _p(gr), _p(m), _p(v), 1, C.c_float(0.01), C.c_float(0.9), C.c_float(0.999),
                            C.c_float(1e-8), None) == 0
    torch.cuda.synchronize()
    # first bias-corrected Adam step moves every weight by lr * sign(g)
    np.testing.assert_allclose(p.cpu().numpy(), p0 - 0.01 * np.sign(g), rtol=1e-5, atol=1e-6)
    packed = torch.empty(1160, dtype=torch.int16, device="cuda")
    assert lib.svf_mlp_pack(_p(p), _p(packed), None) == 0
    torch.cuda.synchronize()
    codes = packed.cpu().numpy().view(np.uint16)
    want = np.array([orc.bf16_encode(float(x)) for x in p.cpu().numpy()], dtype=np.uint16)
    np.testing.assert_array_equal(codes[:1153], want)
    assert (codes[1153:] == 0).all()


@pytest.mark.parametrize("t_every", [1, 3])
def test_stop_decisions_match_oracle(svf, orc, t_every):
    X, st, g = setup(orc, "u8", 4000, 64, "l2", 621)
    Q = synth.sample("u8", 200, 651)
    ix = make_index(svf, X, g, "l2", 64)
    lib = _lib(svf)
    rng = np.random.default_rng(652)
    prm = np.concatenate([rng.standard_normal(1024) * 0.5, rng.standard_normal(64) * 0.2,
                          rng.standard_normal(64) * 0.5, [-0.3]]).astype(np.float32)
    p_d = torch.from_numpy(prm).cuda()
    packed = torch.empty(1160, dtype=torch.int16, device="cuda")
    assert lib.svf_mlp_pack(_p(p_d), _p(packed), None) == 0
    net = orc.MLP(prm[:1024].reshape(64, 16), prm[1024:1088], prm[1088:1152], float(prm[1152])).rounded_bf16()
    tau, T = 0.6, 64
    ids, dist = ix.search(torch.from_numpy(Q).cuda(),
                          svf.SearchConfig(k=10, L=64, T=T, seed=8, mlp=packed, tau=tau, t_min=4, t_every=t_every))
    o = orc.search_ex(st, 4000, g, None, Q, 10, 64, T, 8, net=net, tau=tau, t_min=4, t_every=t_every)
    gi = P.as_u32(ids.cpu().numpy())
    same = (gi == o["ids"]).all(1)
    near = o["margin"] <= 1e-3  # the FP32 logit met the threshold within rounding
    assert not (~same & ~near).any(), f"{(~same & ~near).sum()} queries differ away from the threshold"
    stopped = o["stop_iter"] > 0
    assert stopped.mean() > 0.3 and same.mean() > 0.9
    assert ((o["stop_iter"][stopped] - 4) % t_every == 0).all()


def test_learned_stop_saves_iterations(svf, orc):
    """Train on traces of the plain search, calibrate tau for <= 0.2 pt recall
    loss, and show the average number of iterations drops."""
    from paper_2601_08528_b300 import learned
    X = synth.sample("unit96", 60000, 661)
    Qtr = torch.from_numpy(synth.sample("unit96", 12000, 662)).cuda()
    Qev = torch.from_numpy(synth.sample("unit96", 2000, 663)).cuda()
    ix = svf.Index(96, 60000, dtype="f32", metric="ip", R=32, lowp=("fp8",), max_batch=60000)
    ix.build(torch.from_numpy(X).cuda())
    cfg = svf.SearchConfig(k=10, L=64, T=96, precision="fp8", rerank=True)
    gt_cal, _ = svf.knn(ix.vectors()[:60000], Qtr[:2000], 10, "ip")
    gt_ev, _ = svf.knn(ix.vectors()[:60000], Qev, 10, "ip")
    feat, meta = learned.capture_traces(ix, Qtr[2000:], cfg)
    ids = learned.sample_ids(meta, cfg.T)
    net = learned.train(feat, meta, cfg.T, ids, epochs=3)
    tau, r0, r1 = learned.calibrate(ix, net, Qtr[:2000], gt_cal, cfg)
    assert tau < 1.0
    ix.stats_reset()
    base, _ = ix.search(Qev, cfg)
    it0 = ix.stats()["search_iters"]
    ix.stats_reset()
    import dataclasses
    stop, _ = ix.search(Qev, dataclasses.replace(cfg, mlp=net.packed, tau=tau, t_min=net.t_min))
    it1 = ix.stats()["search_iters"]
    r_base, r_stop = learned.recall_at_k(base, gt_ev), learned.recall_at_k(stop, gt_ev)
    assert r_stop >= r_base - 0.004  # calibrated for 0.2 pt on other queries
    assert it1 < 0.9 * it0, (it0, it1)
