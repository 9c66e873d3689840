"""Host-side checks of the synthetic workloads and of the schedule autotuner.

The scene generators stand in for the scenes of the paper's numerical study (Sec. 6): their shapes
and sizes are what the measurements quote, so their structure is pinned here
by geometry (closed, consistently wound surfaces; Euler characteristic;
volumes and areas against closed forms) and by counts.  The autotuner is
driven with a fake renderer and fake CUDA events so that its selection logic
runs without a GPU.
"""
import collections
import math

import numpy as np
import pytest

from paper_2605_08916_gb300 import scenes as S


def _directed_edges(tris):
    t = np.asarray(tris, np.int64)
    return np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])


def _closed_and_consistent(tris):
    """Every edge is used once in each direction: a closed, consistently
    oriented 2-manifold."""
    e = collections.Counter(map(tuple, _directed_edges(tris)))
    return all(n == 1 and e.get((b, a), 0) == 1 for (a, b), n in e.items())


def _signed_volume(verts, tris):
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64)
    return float(np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])).sum() / 6.0)


@pytest.mark.parametrize("n_theta,n_phi", [(2, 3), (5, 8), (40, 60)])
def test_uv_sphere_is_a_closed_outward_sphere(n_theta, n_phi):
    c, r = np.array([0.3, -1.0, 2.0]), 1.7
    verts, tris, normals = S.uv_sphere(c, r, n_theta, n_phi)
    assert len(tris) == 2 * n_phi * (n_theta - 1)
    assert len(verts) == 2 + n_phi * (n_theta - 1)
    assert _closed_and_consistent(tris)
    n_edges = len(_directed_edges(tris)) // 2
    assert len(verts) - n_edges + len(tris) == 2            # Euler characteristic of S^2
    np.testing.assert_allclose(np.linalg.norm(verts - c, axis=1), r, rtol=1e-12)
    np.testing.assert_allclose(normals, (verts - c) / r, rtol=0, atol=1e-12)
    # outward winding: positive volume, below the sphere's (inscribed polytope)
    vol = _signed_volume(verts - c, tris)
    assert 0 < vol < 4.0 / 3.0 * math.pi * r ** 3
    if n_theta >= 40:
        assert vol > 0.99 * 4.0 / 3.0 * math.pi * r ** 3


def test_furnace_box_is_closed_and_faces_inward():
    s = S.furnace_box(albedo=0.3, emission=2.0)
    assert s.n_tris == 12
    # the box's six quads share corner vertices only by position: merge them
    key = {tuple(p): i for i, p in enumerate(map(tuple, s.verts))}
    ids = np.array([[key[tuple(s.verts[k])] for k in t] for t in s.tris])
    assert _closed_and_consistent(ids)
    assert _signed_volume(s.verts, s.tris) == pytest.approx(-8.0, rel=1e-6)   # 2 x 2 x 2, wound inward
    m = s.materials[s.tri_mat]
    assert np.all(m[:, 0] == S.MAT_DIFFUSE)
    np.testing.assert_array_equal(m[:, 1:4], np.float32(0.3))
    np.testing.assert_array_equal(m[:, 6:9], 2.0)


def test_cornell_box_structure():
    for metal in (False, True):
        s = S.cornell_box(1, 32, 24, glossy=True, metal=metal)
        assert (s.width, s.height) == (32, 24)
        kinds = s.materials[s.tri_mat][:, 0]
        light = kinds == S.MAT_EMITTER
        assert 0 < light.sum() < s.n_tris
        assert np.all(s.materials[s.tri_mat[light]][:, 6:9] > 0)
        assert (kinds == S.MAT_CONDUCTOR).any() == metal
        # the camera eye lies inside the bounding box of the geometry in x and y
        lo, hi = s.verts.min(0), s.verts.max(0)
        assert np.all(s.camera[:2] > lo[:2]) and np.all(s.camera[:2] < hi[:2])


@pytest.mark.parametrize("target", [5_000, 20_000, 100_000])
def test_procedural_scene_size_and_determinism(target):
    a = S.procedural_scene(3, 64, 48, target_tris=target, n_objects=8)
    b = S.procedural_scene(3, 64, 48, target_tris=target, n_objects=8)
    c = S.procedural_scene(4, 64, 48, target_tris=target, n_objects=8)
    assert abs(a.n_tris - target) <= 0.01 * target
    for f in ("verts", "tris", "tri_mat", "materials", "camera"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.verts, c.verts)
    kinds = set(np.unique(a.materials[a.tri_mat][:, 0]).astype(int))
    assert S.MAT_EMITTER in kinds and kinds <= {0, 1, 2, 3, 4}
    # no degenerate triangles (zero area would give no geometric normal)
    v = a.verts.astype(np.float64)
    t = a.tris
    area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)
    assert area.min() > 0


def test_procedural_batch_splits_chains_by_pixels():
    total = 100_003
    batch = S.procedural_batch(6, total, 7, (1_000, 5_000), (32, 96), (3, 6))
    assert len(batch) == 6
    chains = np.array([n for _, _, n in batch])
    px = np.array([s.width * s.height for s, _, _ in batch], np.float64)
    assert chains.sum() == total
    assert np.all(np.abs(chains[:-1] - total * px[:-1] / px.sum()) < 1)
    for s, L, _ in batch:
        assert s.width == s.height and s.width % 16 == 0 and 32 <= s.width <= 96
        assert 3 <= L <= 6
        assert 900 <= s.n_tris <= 5_100
    again = S.procedural_batch(6, total, 7, (1_000, 5_000), (32, 96), (3, 6))
    assert [(s.n_tris, s.width, L, n) for s, L, n in again] == \
           [(s.n_tris, s.width, L, n) for s, L, n in batch]


def test_pss_dim():
    # the film pair, then a BSDF pair and a light pair per scattering vertex
    assert [S.pss_dim(L) for L in (1, 2, 4, 12)] == [2, 6, 14, 46]


# --- the schedule autotuner, with fake CUDA timing -------------------------

class _Clock:
    t = 0.0


class _FakeStream:
    def __init__(self, clock):
        self.clock = clock

    def synchronize(self):
        pass


class _FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream):
        self.t = stream.clock.t

    def synchronize(self):
        pass

    def elapsed_time(self, end):
        return end.t - self.t


def _cost(opts, F):
    """Fake ms per Restore step with one strict minimum."""
    return (1.0 + 0.1 * (opts["traverse_blocks"] != 6) + 0.01 * abs(opts["refill"] - 16)
            + 0.2 * (opts["tail_bounce"] != 4) + 0.05 * (F != 4))


class _FakeRenderer:
    def __init__(self, clock):
        self.clock = clock
        self.opts = {}
        self.inits = []

    def set_option(self, key, value):
        self.opts[key] = value

    def init_chains(self, n, seed, params):
        self.inits.append((n, seed, params))

    def frame(self, F):
        self.clock.t += F * _cost(self.opts, F)


def test_autotune_picks_and_applies_the_fastest_schedule(monkeypatch):
    import torch
    from paper_2605_08916_gb300 import autotune as AT
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    clock = _Clock()
    r, stream = _FakeRenderer(clock), _FakeStream(clock)
    cands = AT.default_candidates()
    best, table = AT.autotune(r, stream, 1234, 5, "prm", steps=8, reps=2)
    assert best == dict(traverse_blocks=6, refill=16, steps_per_frame=4, tail_bounce=4)
    assert {k: r.opts[k] for k in ("traverse_blocks", "refill", "tail_bounce")} == \
           {k: best[k] for k in ("traverse_blocks", "refill", "tail_bounce")}
    assert len(table) == len(cands) and r.inits == [(1234, 5, "prm")] * len(cands)
    for ms, c in table:
        opts = {k: c[k] for k in ("traverse_blocks", "refill", "tail_bounce")}
        assert ms == pytest.approx(_cost(opts, c["steps_per_frame"]))
