"""Seeded synthetic inputs: scenes (triangle soups, materials, cameras) and
analytic target densities.

This module only *generates inputs*.  It holds none of the method's
arithmetic (no path sampling, no Restore step, no RNG of the method): both
the CUDA library and the FP64 oracle receive the arrays built here and
compute everything else on their own.  Randomness here comes from numpy's
PCG64 with fixed seeds, which is unrelated to the Philox4x32-10 stream that
the method itself draws (that stream is implemented separately on each side).

The paper's test scenes (Sec. 6, "Test scenes") are third-party datasets and
are not available; the generators below are the synthetic stand-ins:

* ``cornell_box``      room + two axis-aligned boxes + one quad light
                       (Lambertian, or GGX-coated "glossy" boxes)
* ``caustic_scene``    tessellated glass sphere on a diffuse floor, lit
                       through a small aperture of an occluding light box
* ``procedural_scene`` fBm-displaced terrain grid + many tessellated
                       spheres/boxes with mixed materials
* ``gaussian_mixture`` analytic target on the torus (invariance tests)
* ``StepDensity``      a torus density with a jump (or a smoothed one),
                       for the bias of unadjusted moves across a jump

Material record layout (float32 x 12, shared by both sides):
``[type, albedo_r, albedo_g, albedo_b, roughness, ior, emit_r, emit_g,
emit_b, f0, 0, 0]`` with type 0 diffuse, 1 glossy (GGX coat over a
Lambertian base), 2 smooth dielectric, 3 black emitter, 4 rough conductor.
A conductor record holds the real part eta of its complex index of
refraction (RGB) in the albedo slots and the imaginary part k (RGB) in slots
9..11: ``[4, eta_rgb, roughness, 0, emit_rgb, k_rgb]``.  Any material may
carry emission; emission is one-sided along the triangle's winding normal
``cross(v1 - v0, v2 - v0)``.

Camera record (float32 x 10): ``eye[3], look[3], up[3], vfov_degrees``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAT_DIFFUSE = 0
MAT_GLOSSY = 1
MAT_DIELECTRIC = 2
MAT_EMITTER = 3
MAT_CONDUCTOR = 4
MAT_FLOATS = 12


def material(kind, albedo=(0.0, 0.0, 0.0), roughness=0.0, ior=1.5,
             emission=(0.0, 0.0, 0.0), f0=0.04):
    m = np.zeros(MAT_FLOATS, np.float32)
    m[0] = kind
    m[1:4] = albedo
    m[4] = roughness
    m[5] = ior
    m[6:9] = emission
    m[9] = f0
    return m


def conductor(eta, k, roughness, emission=(0.0, 0.0, 0.0)):
    """Rough conductor record: complex index eta + i k per RGB channel and
    GGX roughness (alpha)."""
    m = np.zeros(MAT_FLOATS, np.float32)
    m[0] = MAT_CONDUCTOR
    m[1:4] = eta
    m[4] = roughness
    m[6:9] = emission
    m[9:12] = k
    return m


@dataclasses.dataclass
class Scene:
    """A triangle soup with per-triangle materials, a pinhole camera and an
    image size.  ``normals`` (per vertex) is optional; when given, shading
    normals are interpolated over each triangle."""
    verts: np.ndarray          # float32 [nv, 3]
    tris: np.ndarray           # int32 [nt, 3]
    tri_mat: np.ndarray        # int32 [nt]
    materials: np.ndarray      # float32 [nm, 12]
    camera: np.ndarray         # float32 [10]
    width: int
    height: int
    normals: np.ndarray | None = None   # float32 [nv, 3] or None
    name: str = "scene"

    @property
    def n_tris(self):
        return int(self.tris.shape[0])

    def check(self):
        assert self.verts.dtype == np.float32 and self.verts.ndim == 2 and self.verts.shape[1] == 3
        assert self.tris.dtype == np.int32 and self.tris.ndim == 2 and self.tris.shape[1] == 3
        assert self.tri_mat.dtype == np.int32 and self.tri_mat.shape == (self.tris.shape[0],)
        assert self.materials.dtype == np.float32 and self.materials.shape[1] == MAT_FLOATS
        assert self.camera.dtype == np.float32 and self.camera.shape == (10,)
        assert self.tris.min() >= 0 and self.tris.max() < self.verts.shape[0]
        assert self.tri_mat.min() >= 0 and self.tri_mat.max() < self.materials.shape[0]
        if self.normals is not None:
            assert self.normals.dtype == np.float32 and self.normals.shape == self.verts.shape
        return self


class _Builder:
    def __init__(self):
        self.v = []
        self.t = []
        self.m = []
        self.mats = []
        self.n = []
        self.nv = 0

    def add_material(self, m):
        self.mats.append(np.asarray(m, np.float32))
        return len(self.mats) - 1

    def add_mesh(self, verts, tris, mat, normals=None):
        verts = np.asarray(verts, np.float64)
        tris = np.asarray(tris, np.int64)
        self.v.append(verts)
        self.t.append(tris + self.nv)
        self.m.append(np.full(len(tris), mat, np.int64))
        self.n.append(None if normals is None else np.asarray(normals, np.float64))
        self.nv += len(verts)

    def add_quad(self, p0, p1, p2, p3, mat):
        """Quad p0-p1-p2-p3 (counter-clockwise seen from the front side)."""
        self.add_mesh(np.array([p0, p1, p2, p3], np.float64), np.array([[0, 1, 2], [0, 2, 3]]), mat)

    def build(self, camera, width, height, name):
        verts = np.concatenate(self.v).astype(np.float32)
        tris = np.concatenate(self.t).astype(np.int32)
        tri_mat = np.concatenate(self.m).astype(np.int32)
        normals = None
        if any(n is not None for n in self.n):
            parts = []
            for v, n in zip(self.v, self.n):
                parts.append(np.zeros_like(v) if n is None else n)
            normals = np.concatenate(parts).astype(np.float32)
        return Scene(verts, tris, tri_mat, np.stack(self.mats).astype(np.float32),
                     np.asarray(camera, np.float32), int(width), int(height), normals, name).check()


def _box_faces(lo, hi, bottomless=True, inward=False):
    """Faces of an axis-aligned box as quads (front side facing outward unless
    ``inward``).  Returns a list of 4-corner arrays."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    faces = [
        [(x0, y1, z0), (x0, y1, z1), (x1, y1, z1), (x1, y1, z0)],  # +y top
        [(x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)],  # +z
        [(x1, y0, z0), (x0, y0, z0), (x0, y1, z0), (x1, y1, z0)],  # -z
        [(x1, y0, z1), (x1, y0, z0), (x1, y1, z0), (x1, y1, z1)],  # +x
        [(x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0)],  # -x
    ]
    if not bottomless:
        faces.append([(x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)])  # -y bottom
    faces = [np.array(f, np.float64) for f in faces]
    if inward:
        faces = [f[::-1].copy() for f in faces]
    return faces


def cornell_box(seed=1, width=64, height=64, glossy=False, light_radiance=15.0, metal=False):
    """Closed room (6 walls, 12 triangles, camera inside), two bottomless
    axis-aligned boxes (2 x 10 triangles) and one quad area light (2 triangles)
    under the ceiling, facing down.  Wall / box albedo per face and channel is
    U[0.2, 0.8]; with ``glossy`` the boxes get a GGX coat (roughness
    U[0.05, 0.3], F0 = 0.04); with ``metal`` they are rough conductors
    (eta U[0.2, 1.6], k U[2, 4] per channel, roughness U[0.05, 0.3])."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    # room [-1,1] x [0,2] x [-1,3]; walls face inward
    room = _box_faces((-1.0, 0.0, -1.0), (1.0, 2.0, 3.0), bottomless=False, inward=True)
    for f in room:
        b.add_quad(*f, b.add_material(material(MAT_DIFFUSE, rng.uniform(0.2, 0.8, 3))))
    boxes = [((-0.75, 0.0, -0.65), (-0.15, 1.2, -0.05)), ((0.1, 0.0, 0.0), (0.7, 0.6, 0.6))]
    for lo, hi in boxes:
        for f in _box_faces(lo, hi, bottomless=True):
            alb = rng.uniform(0.2, 0.8, 3)
            if metal:
                m = conductor(rng.uniform(0.2, 1.6, 3), rng.uniform(2.0, 4.0, 3), rng.uniform(0.05, 0.3))
            elif glossy:
                m = material(MAT_GLOSSY, alb, roughness=rng.uniform(0.05, 0.3), f0=0.04)
            else:
                m = material(MAT_DIFFUSE, alb)
            b.add_quad(*f, b.add_material(m))
    y = 1.98
    lm = b.add_material(material(MAT_EMITTER, emission=(light_radiance,) * 3))
    # facing down: counter-clockwise seen from below
    b.add_quad((-0.25, y, -0.25), (0.25, y, -0.25), (0.25, y, 0.25), (-0.25, y, 0.25), lm)
    cam = [0.0, 1.0, 2.9, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 40.0]
    kind = '-metal' if metal else '-glossy' if glossy else ''
    return b.build(cam, width, height, f"cornell{kind}-{width}x{height}")


def uv_sphere(center, radius, n_theta, n_phi):
    """Tessellated sphere with outward winding and per-vertex normals.
    Triangle count = 2 * n_phi * (n_theta - 1)."""
    c = np.asarray(center, np.float64)
    verts = [c + (0.0, radius, 0.0)]
    for i in range(1, n_theta):
        th = math.pi * i / n_theta
        for j in range(n_phi):
            ph = 2 * math.pi * j / n_phi
            verts.append(c + radius * np.array([math.sin(th) * math.cos(ph), math.cos(th),
                                                -math.sin(th) * math.sin(ph)]))
    verts.append(c + (0.0, -radius, 0.0))
    verts = np.array(verts)
    tris = []
    top, bot = 0, len(verts) - 1

    def ring(i, j):
        return 1 + (i - 1) * n_phi + (j % n_phi)

    for j in range(n_phi):
        tris.append((top, ring(1, j), ring(1, j + 1)))
    for i in range(1, n_theta - 1):
        for j in range(n_phi):
            a, b_, c_, d_ = ring(i, j), ring(i + 1, j), ring(i + 1, j + 1), ring(i, j + 1)
            tris.append((a, b_, c_))
            tris.append((a, c_, d_))
    for j in range(n_phi):
        tris.append((bot, ring(n_theta - 1, j + 1), ring(n_theta - 1, j)))
    tris = np.array(tris, np.int64)
    normals = (verts - c) / radius
    # make the winding outward for every triangle
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cr = np.cross(v1 - v0, v2 - v0)
    flip = np.einsum("ij,ij->i", cr, (v0 + v1 + v2) / 3 - c) < 0
    tris[flip] = tris[flip][:, ::-1]
    return verts, tris, normals


def caustic_scene(seed=1, width=512, height=512, n_theta=100, n_phi=100, aperture=0.05,
                  light_radiance=50.0):
    """Glass sphere (``2 n_phi (n_theta - 1)`` triangles, IOR 1.5, smooth
    shading normals) on a diffuse floor inside a diffuse room.  The area light
    sits inside an occluding box whose bottom face has a square aperture of
    ``aperture`` times the face's area."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    room = _box_faces((-3.0, 0.0, -3.0), (3.0, 4.0, 4.0), bottomless=False, inward=True)
    for f in room:
        b.add_quad(*f, b.add_material(material(MAT_DIFFUSE, rng.uniform(0.4, 0.8, 3))))
    glass = b.add_material(material(MAT_DIELECTRIC, ior=1.5))
    sv, st, sn = uv_sphere((0.0, 0.8, 0.0), 0.8, n_theta, n_phi)
    b.add_mesh(sv, st, glass, sn)
    # light box: half-size s, centred above the sphere, bottom face at y0
    s, y0, y1 = 0.6, 2.6, 3.2
    occ = b.add_material(material(MAT_DIFFUSE, (0.05, 0.05, 0.05)))
    for f in _box_faces((-s, y0, -s), (s, y1, s), bottomless=True, inward=False):
        b.add_quad(*f, occ)
    # bottom face with a centred square hole of side a: (2a)^2 = aperture (2s)^2
    a = s * math.sqrt(aperture)
    ring = [((-s, -s), (s, -a)), ((-s, a), (s, s)), ((-s, -a), (-a, a)), ((a, -a), (s, a))]
    for (xa, za), (xb, zb) in ring:
        # facing down (outward from the box)
        b.add_quad((xa, y0, za), (xb, y0, za), (xb, y0, zb), (xa, y0, zb), occ)
    # inner side of the bottom face (facing up into the box) so light cannot leak
    for (xa, za), (xb, zb) in ring:
        b.add_quad((xa, y0 + 1e-3, za), (xa, y0 + 1e-3, zb), (xb, y0 + 1e-3, zb), (xb, y0 + 1e-3, za), occ)
    lm = b.add_material(material(MAT_EMITTER, emission=(light_radiance,) * 3))
    yl = y1 - 0.05
    b.add_quad((-0.5 * s, yl, -0.5 * s), (0.5 * s, yl, -0.5 * s), (0.5 * s, yl, 0.5 * s),
               (-0.5 * s, yl, 0.5 * s), lm)
    cam = [0.0, 1.6, 3.8, 0.0, 0.7, 0.0, 0.0, 1.0, 0.0, 45.0]
    return b.build(cam, width, height, f"caustic-{width}x{height}")


def _fbm(x, z, rng_phases, octaves=6):
    h = np.zeros_like(x)
    amp, freq = 1.0, 1.0
    for o in range(octaves):
        px, pz, ang = rng_phases[o]
        ca, sa = math.cos(ang), math.sin(ang)
        u = ca * x - sa * z
        w = sa * x + ca * z
        h += amp * (np.sin(freq * u + px) * np.cos(freq * w + pz))
        amp *= 0.5
        freq *= 2.03
    return h


def procedural_scene(seed=1, width=1280, height=720, target_tris=1_000_000, n_objects=200,
                     object_res=(12, 16)):
    """fBm-displaced terrain grid plus ``n_objects`` tessellated spheres and
    boxes, flattened into one triangle soup.  Materials per object are drawn
    from the seed: one third Lambertian, one third GGX glossy, one third
    dielectric.  Four quad area lights hang above the terrain.  The terrain
    resolution is chosen so that the total triangle count is close to
    ``target_tris``."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    ext = 20.0
    nt_th, nt_ph = object_res
    sphere_tris = 2 * nt_ph * (nt_th - 1)
    n_sph = n_objects // 2
    n_box = n_objects - n_sph
    obj_tris = n_sph * sphere_tris + n_box * 12
    light_tris = 8
    terr_tris = max(2, target_tris - obj_tris - light_tris)
    g = max(2, int(round(math.sqrt(terr_tris / 2.0))))
    xs = np.linspace(-ext, ext, g + 1)
    X, Z = np.meshgrid(xs, xs, indexing="xy")
    phases = [(rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi), rng.uniform(0, math.pi))
              for _ in range(8)]
    Y = 1.2 * _fbm(X * 0.25, Z * 0.25, phases)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    idx = np.arange((g + 1) * (g + 1)).reshape(g + 1, g + 1)
    a = idx[:-1, :-1].ravel()
    bb = idx[:-1, 1:].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[1:, :-1].ravel()
    # up-facing winding: (a, d, c), (a, c, bb)
    tris = np.concatenate([np.stack([a, d, c], 1), np.stack([a, c, bb], 1)])
    terr = b.add_material(material(MAT_DIFFUSE, (0.45, 0.42, 0.38)))
    b.add_mesh(verts, tris, terr)

    def height_at(x, z):
        return float(1.2 * _fbm(np.array([x * 0.25]), np.array([z * 0.25]), phases)[0])

    def obj_material():
        r = rng.integers(0, 3)
        if r == 0:
            return material(MAT_DIFFUSE, rng.uniform(0.2, 0.8, 3))
        if r == 1:
            return material(MAT_GLOSSY, rng.uniform(0.2, 0.8, 3), roughness=rng.uniform(0.05, 0.3))
        return material(MAT_DIELECTRIC, ior=1.5)

    for k in range(n_objects):
        x, z = rng.uniform(-0.8 * ext, 0.8 * ext, 2)
        size = rng.uniform(0.3, 1.2)
        y = height_at(x, z)
        m = b.add_material(obj_material())
        if k < n_sph:
            sv, st, sn = uv_sphere((x, y + size, z), size, nt_th, nt_ph)
            b.add_mesh(sv, st, m, sn)
        else:
            lo = (x - size, y - 0.2, z - size)
            hi = (x + size, y + 1.6 * size, z + size)
            for f in _box_faces(lo, hi, bottomless=False):
                b.add_quad(*f, m)
    # four area lights above the terrain (facing down)
    for (cx, cz) in [(-8.0, -8.0), (8.0, -8.0), (-8.0, 8.0), (8.0, 8.0)]:
        lm = b.add_material(material(MAT_EMITTER, emission=rng.uniform(20.0, 40.0, 3)))
        h, s = 14.0, 2.5
        b.add_quad((cx - s, h, cz - s), (cx + s, h, cz - s), (cx + s, h, cz + s), (cx - s, h, cz + s), lm)
    cam = [0.0, 9.0, 24.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 50.0]
    return b.build(cam, width, height, f"procedural-{target_tris}-{width}x{height}")


@dataclasses.dataclass
class Mesh:
    """Object-space triangle mesh of an instanced scene."""
    verts: np.ndarray              # [nv, 3] float32
    tris: np.ndarray               # [nt, 3] int32
    tri_mat: np.ndarray            # [nt] int32
    normals: np.ndarray = None     # [nv, 3] float32 or None (flat)


@dataclasses.dataclass
class InstancedScene:
    """Meshes placed by instances (mesh index, material or -1 for the mesh's
    own, row-major 3 x 4 object-to-world affine map).  The scene is its
    flattening (``flatten``), which both sides render."""
    meshes: list
    instances: list
    materials: np.ndarray
    camera: np.ndarray
    width: int
    height: int
    name: str = "instanced"

    @property
    def n_tris(self):
        return sum(len(self.meshes[m].tris) for m, _, _ in self.instances)

    def flatten(self):
        """The flat scene: instance after instance, vertex p -> ((a0 p.x +
        a1 p.y) + a2 p.z) + t per row in FP64 rounded to float32; normals by
        the inverse transpose (the inverse by cofactors over the
        determinant); a mesh without normals gets zero (flat) normals."""
        V, T, M, N = [], [], [], []
        any_n = any(self.meshes[m].normals is not None for m, _, _ in self.instances)
        vb = 0
        for mesh_i, mat, xf in self.instances:
            mesh = self.meshes[mesh_i]
            A = np.asarray(xf, np.float32).astype(np.float64).reshape(3, 4)
            p = mesh.verts.astype(np.float64)
            w = np.empty_like(p)
            for r in range(3):
                w[:, r] = A[r, 0] * p[:, 0] + A[r, 1] * p[:, 1] + A[r, 2] * p[:, 2] + A[r, 3]
            V.append(w.astype(np.float32))
            T.append(mesh.tris.astype(np.int64) + vb)
            M.append(np.full(len(mesh.tris), mat) if mat >= 0 else mesh.tri_mat.astype(np.int64))
            if any_n:
                if mesh.normals is None:
                    N.append(np.zeros_like(p, dtype=np.float32))
                else:
                    Mi = _inverse3(A[:, :3])
                    n = mesh.normals.astype(np.float64)
                    nw = np.empty_like(n)
                    for r in range(3):
                        nw[:, r] = Mi[0, r] * n[:, 0] + Mi[1, r] * n[:, 1] + Mi[2, r] * n[:, 2]
                    N.append(nw.astype(np.float32))
            vb += len(p)
        return Scene(np.concatenate(V), np.concatenate(T).astype(np.int32), np.concatenate(M).astype(np.int32),
                     np.asarray(self.materials, np.float32), np.asarray(self.camera, np.float32), self.width,
                     self.height, np.concatenate(N) if any_n else None, self.name + "-flat").check()


def _inverse3(a):
    """Inverse of a 3 x 3 matrix by cofactors over the determinant (FP64)."""
    a00, a01, a02 = a[0]
    a10, a11, a12 = a[1]
    a20, a21, a22 = a[2]
    c00 = a11 * a22 - a12 * a21
    c01 = a12 * a20 - a10 * a22
    c02 = a10 * a21 - a11 * a20
    det = a00 * c00 + a01 * c01 + a02 * c02
    return np.array([[c00 / det, (a02 * a21 - a01 * a22) / det, (a01 * a12 - a02 * a11) / det],
                     [c01 / det, (a00 * a22 - a02 * a20) / det, (a02 * a10 - a00 * a12) / det],
                     [c02 / det, (a01 * a20 - a00 * a21) / det, (a00 * a11 - a01 * a10) / det]])


def procedural_scene_instanced(seed=1, width=1280, height=720, target_tris=1_000_000, n_objects=200,
                               object_res=(12, 16), terrain_chunks=4):
    """The procedural scene's layout (same seed draws, same terrain, same
    lights) with its objects as instances: one unit sphere mesh and one unit
    box mesh placed by scale-and-translate maps, one material per instance;
    the terrain (as terrain_chunks x terrain_chunks tiles, so that no one
    mesh's hierarchy is deep) and the lights are meshes with the identity
    map.  With terrain_chunks = 1 its flattening lists the triangles in the
    flat generator's order."""
    rng = np.random.default_rng(seed)
    ext = 20.0
    nt_th, nt_ph = object_res
    sphere_tris = 2 * nt_ph * (nt_th - 1)
    n_sph = n_objects // 2
    n_box = n_objects - n_sph
    obj_tris = n_sph * sphere_tris + n_box * 12
    terr_tris = max(2, target_tris - obj_tris - 8)
    g = max(2, int(round(math.sqrt(terr_tris / 2.0))))
    xs = np.linspace(-ext, ext, g + 1)
    X, Z = np.meshgrid(xs, xs, indexing="xy")
    phases = [(rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi), rng.uniform(0, math.pi))
              for _ in range(8)]
    Y = 1.2 * _fbm(X * 0.25, Z * 0.25, phases)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    idx = np.arange((g + 1) * (g + 1)).reshape(g + 1, g + 1)
    a = idx[:-1, :-1].ravel()
    bb = idx[:-1, 1:].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[1:, :-1].ravel()
    mats = [material(MAT_DIFFUSE, (0.45, 0.42, 0.38))]
    ident = [1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0]
    meshes, instances = [], []
    cuts = np.linspace(0, g, terrain_chunks + 1).round().astype(int)
    for ci in range(terrain_chunks):
        for cj in range(terrain_chunks):
            r0, r1, c0, c1 = cuts[ci], cuts[ci + 1], cuts[cj], cuts[cj + 1]
            sub = idx[r0:r1 + 1, c0:c1 + 1]
            remap = sub.ravel()
            loc = np.arange(remap.size).reshape(sub.shape)
            la, lb, lc, ld = loc[:-1, :-1].ravel(), loc[:-1, 1:].ravel(), loc[1:, 1:].ravel(), loc[1:, :-1].ravel()
            t = np.concatenate([np.stack([la, ld, lc], 1), np.stack([la, lc, lb], 1)])
            meshes.append(Mesh(verts[remap].astype(np.float32), t.astype(np.int32), np.zeros(len(t), np.int32)))
            instances.append((len(meshes) - 1, -1, ident))
    sphere_mesh, box_mesh = len(meshes), len(meshes) + 1
    sv, st, sn = uv_sphere((0.0, 0.0, 0.0), 1.0, nt_th, nt_ph)
    meshes.append(Mesh(sv.astype(np.float32), st.astype(np.int32), np.zeros(len(st), np.int32),
                       sn.astype(np.float32)))
    bv, bt = [], []
    for f in _box_faces((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), bottomless=False):
        k = len(bv)
        bv.extend(f)
        bt.extend([[k, k + 1, k + 2], [k, k + 2, k + 3]])
    meshes.append(Mesh(np.array(bv, np.float32), np.array(bt, np.int32), np.zeros(len(bt), np.int32)))

    def height_at(x, z):
        return float(1.2 * _fbm(np.array([x * 0.25]), np.array([z * 0.25]), phases)[0])

    def obj_material():
        r = rng.integers(0, 3)
        if r == 0:
            return material(MAT_DIFFUSE, rng.uniform(0.2, 0.8, 3))
        if r == 1:
            return material(MAT_GLOSSY, rng.uniform(0.2, 0.8, 3), roughness=rng.uniform(0.05, 0.3))
        return material(MAT_DIELECTRIC, ior=1.5)

    for k in range(n_objects):
        x, z = rng.uniform(-0.8 * ext, 0.8 * ext, 2)
        size = rng.uniform(0.3, 1.2)
        y = height_at(x, z)
        mats.append(obj_material())
        m = len(mats) - 1
        if k < n_sph:
            instances.append((sphere_mesh, m, [size, 0.0, 0.0, x, 0.0, size, 0.0, y + size, 0.0, 0.0, size, z]))
        else:
            lo = np.array([x - size, y - 0.2, z - size])
            hi = np.array([x + size, y + 1.6 * size, z + size])
            cc, hh = (lo + hi) / 2, (hi - lo) / 2
            instances.append((box_mesh, m, [hh[0], 0.0, 0.0, cc[0], 0.0, hh[1], 0.0, cc[1], 0.0, 0.0, hh[2], cc[2]]))
    lv, lt, lm = [], [], []
    for (cx, cz) in [(-8.0, -8.0), (8.0, -8.0), (-8.0, 8.0), (8.0, 8.0)]:
        mats.append(material(MAT_EMITTER, emission=rng.uniform(20.0, 40.0, 3)))
        h, sz = 14.0, 2.5
        k = len(lv)
        lv.extend([(cx - sz, h, cz - sz), (cx + sz, h, cz - sz), (cx + sz, h, cz + sz), (cx - sz, h, cz + sz)])
        lt.extend([[k, k + 1, k + 2], [k, k + 2, k + 3]])
        lm.extend([len(mats) - 1] * 2)
    meshes.append(Mesh(np.array(lv, np.float32), np.array(lt, np.int32), np.array(lm, np.int32)))
    instances.append((len(meshes) - 1, -1, ident))
    cam = [0.0, 9.0, 24.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 50.0]
    return InstancedScene(meshes, instances, np.stack(mats).astype(np.float32), np.asarray(cam, np.float32),
                          int(width), int(height), f"procedural-instanced-{target_tris}-{width}x{height}")


def procedural_batch(n_scenes=64, total_chains=1 << 21, seed=2605, tris_range=(1_000, 200_000),
                     size_range=(128, 512), L_range=(4, 16)):
    """The multi-scene workload: ``n_scenes`` variants of the procedural
    scene (scene seed 1..n) with triangle counts log-uniform over
    ``tris_range``, square images with sides uniform over ``size_range``
    (multiples of 16), path lengths uniform over ``L_range``, and
    ``total_chains`` split in proportion to the pixel counts.  Returns
    [(scene, max_path_len, n_chains), ...]."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_scenes):
        tris = int(round(math.exp(rng.uniform(math.log(tris_range[0]), math.log(tris_range[1])))))
        side = int(rng.integers(size_range[0] // 16, size_range[1] // 16 + 1)) * 16
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        specs.append((i + 1, tris, side, L))
    px = np.array([side * side for _, _, side, _ in specs], np.float64)
    chains = np.floor(total_chains * px / px.sum()).astype(np.int64)
    chains[-1] += total_chains - chains.sum()
    out = []
    for (sseed, tris, side, L), n in zip(specs, chains):
        n_obj = int(max(2, min(200, round(tris / 1000))))
        out.append((procedural_scene(sseed, side, side, target_tris=tris, n_objects=n_obj), L, int(n)))
    return out


def furnace_box(albedo=0.5, emission=1.0, width=8, height=8):
    """Closed room whose walls all reflect (Lambertian, ``albedo``) and emit
    (``emission``, facing inward).  Radiance is the same everywhere: truncated
    after n segments it equals sum_{k<n} albedo^k * emission."""
    b = _Builder()
    for f in _box_faces((-1.0, 0.0, -1.0), (1.0, 2.0, 1.0), bottomless=False, inward=True):
        b.add_quad(*f, b.add_material(material(MAT_DIFFUSE, (albedo,) * 3, emission=(emission,) * 3)))
    cam = [0.0, 1.0, 0.5, 0.0, 1.0, -1.0, 0.0, 1.0, 0.0, 60.0]
    return b.build(cam, width, height, "furnace")


def glass_furnace(camera_inside=False, emission=1.0, ior=1.5, n_theta=12, n_phi=16, width=8, height=8):
    """A glass body inside a closed room whose walls are black emitters
    (radiance ``emission``, facing inward).  The glass is a UV sphere of
    radius 1 at (0, 1, 0) with flat facets (no shading normals).  The camera
    sits at the sphere's centre (``camera_inside``) or between the sphere and
    a wall.  Every path that reaches a wall ends there, so its contribution
    is fixed by the radiance scaling of the refractions it went through."""
    b = _Builder()
    wall = b.add_material(material(MAT_EMITTER, emission=(emission,) * 3))
    for f in _box_faces((-3.0, -2.0, -3.0), (3.0, 4.0, 3.0), bottomless=False, inward=True):
        b.add_quad(*f, wall)
    sv, st, _ = uv_sphere((0.0, 1.0, 0.0), 1.0, n_theta, n_phi)
    b.add_mesh(sv, st, b.add_material(material(MAT_DIELECTRIC, ior=ior)))
    if camera_inside:
        cam = [0.0, 1.0, 0.0, 0.3, 1.2, -1.0, 0.0, 1.0, 0.0, 70.0]
    else:
        cam = [0.0, 1.0, 2.7, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 50.0]
    return b.build(cam, width, height, "glass-furnace-" + ("inside" if camera_inside else "outside"))


def glass_slab_stripes(thickness=1.0, stripe=0.05, ior=1.5, width=8, height=8):
    """A camera at the origin looking down -z at a closed glass slab
    (z in [-1 - thickness, -1], 60 x 60 wide).  Black emitter stripes of width
    ``stripe`` along x lie behind the slab at z = -4 (facing +z) and behind
    the camera at z = +3 (facing -z); stripe k (x in [k s, (k + 1) s]) emits
    ``stripe_radiance(k, side)``.  Where a refracted or reflected ray lands,
    and therefore the path's contribution, follows from Snell's law and the
    mirror law in closed form."""
    b = _Builder()
    glass = b.add_material(material(MAT_DIELECTRIC, ior=ior))
    z0, z1 = -1.0 - thickness, -1.0
    for f in _box_faces((-30.0, -30.0, z0), (30.0, 30.0, z1), bottomless=False, inward=False):
        b.add_quad(*f, glass)
    n = int(round(6.0 / stripe))
    for side, z in ((0, -4.0), (1, 3.0)):
        for k in range(-n, n):
            xa, xb = k * stripe, (k + 1) * stripe
            m = b.add_material(material(MAT_EMITTER, emission=(stripe_radiance(k, side),) * 3))
            if side == 0:   # facing +z
                b.add_quad((xa, -6.0, z), (xb, -6.0, z), (xb, 6.0, z), (xa, 6.0, z), m)
            else:           # facing -z
                b.add_quad((xa, -6.0, z), (xa, 6.0, z), (xb, 6.0, z), (xb, -6.0, z), m)
    cam = [0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 0.0, 1.0, 0.0, 60.0]
    return b.build(cam, width, height, "glass-slab-stripes")


def stripe_radiance(k, side):
    """Radiance of stripe k of ``glass_slab_stripes`` (side 0 behind the slab,
    1 behind the camera): neighbouring stripes always differ."""
    return 1.0 + (k % 7) + 10.0 * side


def parallel_squares(half_light=0.5, height=1.0, albedo=0.5, radiance=1.0, glossy=False,
                     roughness=0.2, width=1, height_px=1):
    """A large receiving floor (y = 0) under a square emitter of half-side
    ``half_light`` at ``height`` facing down.  The camera looks straight down
    at the floor point on the emitter's axis through a hole-free path (the
    camera sits just below the light plane, off to the side of nothing:
    the light is one-sided so the camera sees only the floor)."""
    b = _Builder()
    kind = MAT_GLOSSY if glossy else MAT_DIFFUSE
    fm = b.add_material(material(kind, (albedo,) * 3, roughness=roughness, f0=0.04))
    L = 50.0
    b.add_quad((-L, 0.0, -L), (-L, 0.0, L), (L, 0.0, L), (L, 0.0, -L), fm)
    lm = b.add_material(material(MAT_EMITTER, emission=(radiance,) * 3))
    s = half_light
    b.add_quad((-s, height, -s), (s, height, -s), (s, height, s), (-s, height, s), lm)
    cam = [0.0, 0.5 * height, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 1e-3]
    return b.build(cam, width, height_px, "parallel-squares")


@dataclasses.dataclass
class Mixture:
    """Isotropic Gaussian mixture on the torus T^d (K = 0 means a constant
    density ``const``).  Component k has weight w[k], mean mu[k] (in
    [0.25, 0.75]^d) and standard deviation sig[k]."""
    d: int
    w: np.ndarray
    mu: np.ndarray
    sig: np.ndarray
    width: int = 16
    height: int = 16
    const: float = 1.0

    @property
    def K(self):
        return int(len(self.w))


def gaussian_mixture(seed=1, d=4, K=3, sig_range=(0.03, 0.05), width=16, height=16):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, K)
    w /= w.sum()
    mu = rng.uniform(0.25, 0.75, (K, d))
    sig = rng.uniform(*sig_range, K)
    return Mixture(d, w, mu, sig, width, height)


def single_gaussian(center, sig, width=16, height=16):
    c = np.asarray(center, np.float64)
    return Mixture(len(c), np.array([1.0]), c[None, :], np.array([float(sig)]), width, height)


def constant_target(d=4, value=1.0, width=8, height=8):
    return Mixture(d, np.zeros(0), np.zeros((0, d)), np.zeros(0), width, height, const=float(value))


@dataclasses.dataclass
class StepDensity:
    """Density on the torus T^d with one jump per half period along x0:
    about c1 on x0 in (0, 1/2) and c2 on (1/2, 1), the jumps smoothed over a
    width ~w (w = 0: sharp), g(x) = c2 + (c1 - c2) (1 + tanh(q(x0) / w)) / 2
    with q(x0) = sin(2 pi x0) / (2 pi).  The pixel grid is width x height
    over (x0, x1); the default 2 x 1 grid puts each half in its own pixel."""
    d: int = 2
    c1: float = 1.0
    c2: float = 4.0
    w: float = 0.0
    width: int = 2
    height: int = 1


def pss_dim(max_path_len):
    """PSS dimension d = 2 + 4 (L - 1): the film pair plus, for each of the
    L - 1 scattering vertices, one BSDF pair and one light-sample pair."""
    return 2 + 4 * (int(max_path_len) - 1)


WORKLOADS = {
    # name: (scene builder kwargs, max path length, chains, steps, drift mode)
    "cornell-64-fd": dict(scene=lambda: cornell_box(1, 64, 64, glossy=False), L=4, chains=4096,
                          steps=256, drift="fd"),
    "cornell-glossy-256-adjoint": dict(scene=lambda: cornell_box(1, 256, 256, glossy=True), L=8,
                                       chains=65536, steps=256, drift="adjoint"),
    "caustic-20k-512": dict(scene=lambda: caustic_scene(1, 512, 512), L=10, chains=262144,
                            steps=64, drift="adjoint"),
    "procedural-1m-720p": dict(scene=lambda: procedural_scene(1, 1280, 720), L=12, chains=1 << 20,
                               steps=16, drift="adjoint"),
}
