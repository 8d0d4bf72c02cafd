"""View sampling (Sec. 4.3): the Python oracle pinned by the generator's
published outputs and by properties K-means and uniform draws must have;
then the library's host-side sampler against the oracle, bit for bit
(no device needed)."""
import json
import os

import numpy as np
import pytest

from oracle import views as ov
from paper_2504_12905_gb300 import synthetic as syn

HERE = os.path.dirname(os.path.abspath(__file__))


def _w2c(cams):
    return [list(map(float, c["world_to_cam"])) for c in cams]


def test_splitmix64_published_sequences():
    with open(os.path.join(HERE, "golden", "splitmix64.json")) as f:
        g = json.load(f)
    assert ov.SplitMix64(0).next() == int(g["seed_0"][0], 16)
    s = ov.SplitMix64(1234567)
    assert [s.next() for _ in range(5)] == g["seed_1234567"]


def test_uniform_views_are_distinct_sorted_and_uniform():
    n, k, steps = 24, 8, 3000
    counts = np.zeros(n)
    for step in range(steps):
        v = ov.uniform_views(n, k, seed=7, step=step)
        assert len(v) == k and len(set(v)) == k and v == sorted(v) and 0 <= v[0] and v[-1] < n
        counts[v] += 1
    p = k / n
    assert np.all(np.abs(counts - steps * p) <= 5 * np.sqrt(steps * p * (1 - p)))
    assert ov.uniform_views(5, 0, 1, 0) == [0, 1, 2, 3, 4] == ov.uniform_views(5, 9, 1, 3)


def _groups():
    """Three tight groups of five cameras: positions around three points,
    all looking at the origin."""
    rng = np.random.default_rng(3)
    cams = []
    for centre in ([3.0, 0.0, 0.5], [-1.5, 2.6, 0.5], [-1.5, -2.6, 0.5]):
        for _ in range(5):
            eye = np.array(centre) + rng.normal(0.0, 0.05, 3)
            cams.append(syn.look_at_camera(eye, 32, 32))
    return np.array(cams, dtype=syn.CAMERA_DTYPE)


def test_kmeans_recovers_separated_groups():
    feats = ov.camera_features(_w2c(_groups()))
    labels, iters = ov.kmeans(feats, 3, seed=11)
    groups = [set(labels[5 * g:5 * g + 5]) for g in range(3)]
    assert all(len(s) == 1 for s in groups) and len(set.union(*groups)) == 3
    assert iters < 100


@pytest.mark.parametrize("k", [1, 5, 8, 24])
def test_kmeans_fixed_point(k):
    """At convergence every camera is nearest to its own cluster's mean."""
    feats = ov.camera_features(_w2c(syn.hemisphere_cameras(24, 3.0, 32, 32)))
    labels, iters = ov.kmeans(feats, k, seed=5)
    assert iters < 100
    F = np.array(feats)
    lab = np.array(labels)
    cen = np.array([F[lab == c].mean(axis=0) if (lab == c).any() else np.full(6, np.inf) for c in range(k)])
    d = ((F[:, None, :] - cen[None, :, :]) ** 2).sum(-1)
    assert np.all(d[np.arange(len(F)), lab] <= d.min(axis=1) + 1e-12)
    if k == 24:
        assert len(set(labels)) == 24
    if k == 1:
        assert set(labels) == {0}


def test_features_are_normalised():
    feats = np.array(ov.camera_features(_w2c(syn.ring_cameras(12, 3.0, 32, 32))))
    pos, dirs = feats[:, :3], feats[:, 3:]
    assert np.allclose(pos.mean(axis=0), 0.0, atol=1e-12)
    assert np.isclose(np.linalg.norm(pos, axis=1).max(), 1.0)
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-6)
    # a ring camera at radius 3 looks at the origin: its +z axis is -position / |position|
    assert np.allclose(dirs, -pos / np.linalg.norm(pos, axis=1, keepdims=True), atol=1e-6)


def test_cluster_draw_takes_one_per_cluster_uniformly():
    labels = [0, 0, 0, 1, 1, 2, 0, 1, 2, 2, 2, 2]
    counts = np.zeros(len(labels))
    steps = 4000
    for step in range(steps):
        v = ov.cluster_draw(labels, 3, seed=9, step=step)
        assert sorted({labels[i] for i in v}) == [0, 1, 2] and len(v) == 3
        counts[v] += 1
    for c in range(3):
        m = [i for i, l in enumerate(labels) if l == c]
        p = 1.0 / len(m)
        assert np.all(np.abs(counts[m] - steps * p) <= 5 * np.sqrt(steps * p * (1 - p)))


# ---- the library's sampler against the oracle ----------------------------

def _camera_sets():
    rng = np.random.default_rng(21)
    return {
        "ring24": syn.ring_cameras(24, 3.0, 64, 64),
        "hemisphere96": syn.hemisphere_cameras(96, 3.0, 64, 64),
        "orbit100": syn.orbit_cameras(rng, 100, 3.0, 64, 64),
        "groups15": _groups(),
    }


@pytest.fixture(scope="module")
def lmrs():
    from paper_2504_12905_gb300 import build
    build.build()
    from paper_2504_12905_gb300 import lmrs as m
    return m


@pytest.mark.parametrize("name", ["ring24", "hemisphere96", "orbit100", "groups15"])
@pytest.mark.parametrize("k", [1, 3, 8, 16, 32])
def test_library_sampler_equals_oracle(lmrs, name, k):
    cams = _camera_sets()[name]
    seed = 0xC0FFEE + k
    labels_ref, iters_ref = ov.kmeans(ov.camera_features(_w2c(cams)), k, seed)
    smp = lmrs.ViewSampler(cams, k, seed)
    labels, kk, iters = smp.labels()
    assert kk == min(k, len(cams)) and iters == iters_ref
    np.testing.assert_array_equal(labels, labels_ref)
    for step in range(20):
        np.testing.assert_array_equal(smp.draw(step), ov.cluster_draw(labels_ref, kk, seed, step))
    smp.close()


def test_library_uniform_views_equal_oracle(lmrs):
    for n, k in [(24, 8), (100, 12), (7, 7), (5, 0), (96, 32)]:
        for step in range(15):
            np.testing.assert_array_equal(lmrs.lmrs_uniform_views(n, k, 123, step), ov.uniform_views(n, k, 123, step))
