"""Instanced scenes: the flattening that defines them (both the library and
the oracle render the flattened scene).

Pins: a normal carried by the inverse transpose stays perpendicular to the
edges carried by the map itself (n^T A^-1 A e = n^T e = 0) for random
affine maps; the identity map reproduces the mesh; the instanced procedural
layout flattens to the flat procedural generator's scene up to float32
rounding of the vertex positions (same triangles, materials and order).
"""
import numpy as np

from paper_2605_08916_gb300 import scenes as S


def _box_mesh_with_face_normals():
    v, t, n = [], [], []
    for f in S._box_faces((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), bottomless=False):
        f = np.asarray(f)
        fn = np.cross(f[1] - f[0], f[2] - f[0])
        fn /= np.linalg.norm(fn)
        k = len(v)
        v.extend(f)
        n.extend([fn] * 4)
        t.extend([[k, k + 1, k + 2], [k, k + 2, k + 3]])
    return S.Mesh(np.array(v, np.float32), np.array(t, np.int32), np.zeros(len(t), np.int32),
                  np.array(n, np.float32))


def test_flatten_carries_normals_by_the_inverse_transpose():
    rng = np.random.default_rng(3)
    mesh = _box_mesh_with_face_normals()
    insts = []
    for _ in range(6):
        A = rng.normal(size=(3, 3)) + 2.0 * np.eye(3)
        t = rng.normal(size=3) * 5
        insts.append((0, -1, np.concatenate([A, t[:, None]], 1).ravel().tolist()))
    isc = S.InstancedScene([mesh], insts, np.stack([S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))]),
                           np.zeros(10, np.float32), 8, 8)
    flat = isc.flatten()
    v = flat.verts.astype(np.float64)
    n = flat.normals.astype(np.float64)
    per = len(mesh.tris)
    for i, tri in enumerate(flat.tris):
        e1, e2 = v[tri[1]] - v[tri[0]], v[tri[2]] - v[tri[0]]
        for k in tri:
            nk = n[k] / np.linalg.norm(n[k])
            assert abs(nk @ e1) <= 1e-5 * np.linalg.norm(e1)
            assert abs(nk @ e2) <= 1e-5 * np.linalg.norm(e2)
        # the winding normal A e1 x A e2 = det(A) A^-T (e1 x e2): same side
        # as the carried normal exactly when det(A) > 0
        det = np.linalg.det(np.asarray(insts[i // per][2]).reshape(3, 4)[:, :3])
        assert (np.cross(e1, e2) @ n[tri[0]] > 0) == (det > 0)


def test_identity_instances_reproduce_the_meshes():
    mesh = _box_mesh_with_face_normals()
    ident = [1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0]
    isc = S.InstancedScene([mesh], [(0, -1, ident), (0, 0, ident)],
                           np.stack([S.material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))]), np.zeros(10, np.float32), 8, 8)
    flat = isc.flatten()
    assert np.array_equal(flat.verts[:len(mesh.verts)], mesh.verts)
    assert np.array_equal(flat.verts[len(mesh.verts):], mesh.verts)
    assert np.array_equal(flat.tris[len(mesh.tris):], mesh.tris + len(mesh.verts))
    assert np.allclose(flat.normals[:len(mesh.verts)], mesh.normals, atol=1e-7)


def _tri_set(sc):
    key = np.concatenate([sc.verts[sc.tris].reshape(-1, 9), sc.tri_mat[:, None].astype(np.float32)], 1)
    return key[np.lexsort(key.T[::-1])]


def test_instanced_procedural_layout_flattens_to_the_flat_generator():
    flat = S.procedural_scene(1, 64, 36, target_tris=60000, n_objects=40)
    isc = S.procedural_scene_instanced(1, 64, 36, target_tris=60000, n_objects=40, terrain_chunks=1)
    f = isc.flatten()
    assert f.n_tris == flat.n_tris and len(isc.instances) == 42
    assert np.array_equal(f.tris, flat.tris)
    assert np.array_equal(f.tri_mat, flat.tri_mat)
    assert np.array_equal(f.materials, flat.materials)
    assert np.allclose(f.verts, flat.verts, rtol=0, atol=2e-5)
    # terrain tiles: the same triangles (exact terrain vertices), regrouped
    tiled = S.procedural_scene_instanced(1, 64, 36, target_tris=60000, n_objects=40, terrain_chunks=3).flatten()
    assert tiled.n_tris == flat.n_tris
    a, b = _tri_set(tiled), _tri_set(f)
    assert np.array_equal(a, b)
