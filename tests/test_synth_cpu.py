"""Seeded input generators (no method arithmetic): determinism and the
component samplers of the serving streams."""
import numpy as np

import synth


def test_window_components_stay_in_the_moving_window():
    C, W, speed = 4096, 64, 4.0
    draw = synth.window_components(C, W, speed, 7)
    perm = np.random.default_rng(7).permutation(C)
    rng = np.random.default_rng(1)
    for t in (0.0, 0.6, 3.2, 1500.0):
        comps = draw(rng, t, 500)
        start = int(np.floor(t * speed))
        allowed = set(perm[(start + np.arange(W)) % C].tolist())
        assert set(comps.tolist()) <= allowed
        assert len(set(comps.tolist())) > W // 2  # spread over the window


def test_given_components_feed_the_generator_in_order():
    labels = np.arange(300) % 16
    X = synth.sample_chunked("tiny", 300, 11, component_sampler=synth.given_components(labels), workers=1)
    Y = synth.sample_chunked("tiny", 300, 11, component_sampler=synth.given_components(labels), workers=1)
    assert X.shape == (300, 128) and np.array_equal(X, Y)
    # rows drawn for the same component sit near the same centre
    c = synth.centres(synth.MIXTURES["tiny"])
    near = np.argmin(((X[:, None, :] - c[None, :, :]) ** 2).sum(-1), axis=1)
    assert (near == labels).mean() > 0.95
