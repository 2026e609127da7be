"""Geometry of the GPU contact case at the bodies' extremes (CPU only): each
body's farthest point from its origin reaches into the cube, so that the
particles it contacts lie near the edge of the body's bounding ball. The signed
distances here are numpy restatements of the primitives' definitions."""
import numpy as np

from paper_2503_05046_gb300 import scenes
from test_gpu_parity import extremes_scene


def _sdf(b, x):
    y = (x - b["p"]) @ b["R"]  # body frame: R^T (x - p) for each row
    prm = b["params"]
    if b["shape"] == scenes.SPHERE:
        return np.linalg.norm(y, axis=1) - prm[0]
    if b["shape"] == scenes.BOX:
        q = np.abs(y) - prm[:3]
        return np.linalg.norm(np.maximum(q, 0.0), axis=1) + np.minimum(q.max(1), 0.0)
    if b["shape"] == scenes.CAPSULE:
        o = y.copy()
        o[:, 2] -= np.clip(y[:, 2], -prm[0], prm[0])
        return np.linalg.norm(o, axis=1) - prm[1]
    return y[:, 2]  # half-space


def _bound(b):
    prm = b["params"]
    return {scenes.SPHERE: prm[0], scenes.BOX: np.linalg.norm(prm[:3]),
            scenes.CAPSULE: prm[0] + prm[1]}[b["shape"]]


def test_extreme_points_reach_into_the_cube():
    sc = extremes_scene()
    x = sc["groups"][0]["x"].astype(np.float64)
    assert _sdf(sc["bodies"][0], x).min() > 0.0  # nothing touches the ground
    for b in sc["bodies"][1:]:
        R = b["R"]
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-12) and np.linalg.det(R) > 0
        phi = _sdf(b, x)
        inside = phi < 0.0
        assert inside.sum() >= 3, b["shape"]
        # every contacted particle lies inside the body's bounding ball, and
        # the deepest-reaching ones lie in its outer tenth
        r = np.linalg.norm(x[inside] - b["p"], axis=1)
        assert r.max() <= _bound(b) * (1 + 1e-9)
        assert r.max() >= 0.9 * _bound(b), (b["shape"], r.max(), _bound(b))
