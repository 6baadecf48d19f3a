"""Seeded synthetic scene generator (inputs only).

This module builds triangle meshes, material tables and pinhole cameras with
numpy.  It holds none of the method's arithmetic (no sampling, no intersection,
no estimator) and is the only code that both the CUDA library's tests and the
CPU oracle consume.  The paper's scenes (Section 9: Bitterli's bathroom, glass
of water and kitchen, lmc's Veach-Ajar and Torus, the swimming pool) are not
available; these seeded scenes stand in for them.

Material record (12 float32): [type, albedo r g b, emission r g b, phong
exponent, ior, 0, 0, 0]; type 0 Lambertian, 1 modified Phong, 2 smooth
dielectric.  Emission is one-sided: a triangle emits on the side its winding
normal (v1 - v0) x (v2 - v0) points to.

Camera (12 float32): origin o, forward f, right r, up u; the film point
(x0, x1) in [0,1)^2 looks along f + (2 x0 - 1) r + (1 - 2 x1) u, so x1 = 0 is
the top row.  Pixel (i, j) = (floor(x0 W), floor(x1 H)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LAMBERT, PHONG, DIELECTRIC = 0, 1, 2
MAT_FLOATS = 12


@dataclasses.dataclass
class SceneArrays:
    name: str
    verts: np.ndarray      # float32 [n_verts, 3]
    tris: np.ndarray       # uint32  [n_tris, 3]
    tri_mat: np.ndarray    # uint32  [n_tris]
    mats: np.ndarray       # float32 [n_mats, 12]
    camera: np.ndarray     # float32 [12]
    width: int
    height: int
    depth: int

    @property
    def D(self) -> int:
        """Primary-sample-space dimension: 2 film + 2 per bounce."""
        return 2 + 2 * self.depth

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def material(kind, albedo=(0, 0, 0), emission=(0, 0, 0), phong_n=0.0, ior=1.0):
    m = np.zeros(MAT_FLOATS, np.float32)
    m[0] = kind
    m[1:4] = albedo
    m[4:7] = emission
    m[7] = phong_n
    m[8] = ior
    return m


class _Builder:
    def __init__(self):
        self.v, self.t, self.m = [], [], []
        self.mats = []

    def add_material(self, m) -> int:
        self.mats.append(np.asarray(m, np.float32))
        return len(self.mats) - 1

    def tri(self, a, b, c, mat):
        base = sum(len(x) for x in self.v)
        self.v.append(np.asarray([a, b, c], np.float64))
        self.t.append(np.asarray([[base, base + 1, base + 2]], np.int64))
        self.m.append(np.asarray([mat], np.int64))

    def quad(self, center, e1, e2, normal, mat):
        """Axis-aligned (or any planar) quad centre +- e1/2 +- e2/2, winding so
        that the geometric normal points along ``normal``."""
        c, e1, e2, nrm = (np.asarray(a, np.float64) for a in (center, e1, e2, normal))
        if np.dot(np.cross(e1, e2), nrm) < 0:
            e1, e2 = e2, e1
        a = c - 0.5 * e1 - 0.5 * e2
        b = c + 0.5 * e1 - 0.5 * e2
        cc = c + 0.5 * e1 + 0.5 * e2
        d = c - 0.5 * e1 + 0.5 * e2
        self.tri(a, b, cc, mat)
        self.tri(a, cc, d, mat)

    def box(self, lo, hi, mat, inward=False):
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        c = 0.5 * (lo + hi)
        s = hi - lo
        sgn = -1.0 if inward else 1.0
        for ax in range(3):
            for side in (-1.0, 1.0):
                cen = c.copy()
                cen[ax] = lo[ax] if side < 0 else hi[ax]
                o1, o2 = [a for a in range(3) if a != ax]
                e1 = np.zeros(3)
                e1[o1] = s[o1]
                e2 = np.zeros(3)
                e2[o2] = s[o2]
                n = np.zeros(3)
                n[ax] = side * sgn
                self.quad(cen, e1, e2, n, mat)

    def mesh(self, verts, tris, mat):
        base = sum(len(x) for x in self.v)
        self.v.append(np.asarray(verts, np.float64))
        self.t.append(np.asarray(tris, np.int64) + base)
        self.m.append(np.full(len(tris), mat, np.int64))

    def build(self, name, camera, width, height, depth) -> SceneArrays:
        verts = np.concatenate(self.v).astype(np.float32) if self.v else np.zeros((0, 3), np.float32)
        tris = np.concatenate(self.t).astype(np.uint32) if self.t else np.zeros((0, 3), np.uint32)
        tm = np.concatenate(self.m).astype(np.uint32) if self.m else np.zeros((0,), np.uint32)
        mats = np.stack(self.mats).astype(np.float32) if self.mats else np.zeros((1, MAT_FLOATS), np.float32)
        return SceneArrays(name, np.ascontiguousarray(verts), np.ascontiguousarray(tris), np.ascontiguousarray(tm),
                           np.ascontiguousarray(mats), np.asarray(camera, np.float32), int(width), int(height),
                           int(depth))


def pinhole(origin, target, up, vfov_tan_half, aspect):
    o = np.asarray(origin, np.float64)
    f = np.asarray(target, np.float64) - o
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return np.concatenate([o, f, r * vfov_tan_half * aspect, u * vfov_tan_half]).astype(np.float32)


def uv_sphere(center, radius, n_lon, n_lat):
    """UV sphere with 2 * n_lon * (n_lat - 1) triangles, outward winding."""
    c = np.asarray(center, np.float64)
    verts = [c + np.array([0.0, radius, 0.0])]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * math.pi * j / n_lon
            verts.append(c + radius * np.array([math.sin(th) * math.cos(ph), math.cos(th), math.sin(th) * math.sin(ph)]))
    verts.append(c - np.array([0.0, radius, 0.0]))
    verts = np.asarray(verts)
    top, bot = 0, len(verts) - 1

    def ring(i, j):
        return 1 + (i - 1) * n_lon + (j % n_lon)

    tris = []
    for j in range(n_lon):
        tris.append([top, ring(1, j + 1), ring(1, j)])
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a, b = ring(i, j), ring(i, j + 1)
            cc, d = ring(i + 1, j), ring(i + 1, j + 1)
            tris.append([a, b, d])
            tris.append([a, d, cc])
    for j in range(n_lon):
        tris.append([bot, ring(n_lat - 1, j), ring(n_lat - 1, j + 1)])
    tris = np.asarray(tris)
    # make the winding outward (normal . (centroid - c) > 0)
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(v1 - v0, v2 - v0)
    flip = np.einsum("ij,ij->i", n, (v0 + v1 + v2) / 3.0 - c) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris


CORNELL_CAMERA_TAN = 0.5 / 1.3


def _cornell_room(b: _Builder, light_size: float, block=True):
    grey = b.add_material(material(LAMBERT, (0.7, 0.7, 0.7)))
    red = b.add_material(material(LAMBERT, (0.7, 0.0, 0.0)))
    green = b.add_material(material(LAMBERT, (0.0, 0.7, 0.0)))
    light = b.add_material(material(LAMBERT, (0.0, 0.0, 0.0), emission=(15.0, 15.0, 15.0)))
    b.quad((0.5, 0.0, 0.5), (1, 0, 0), (0, 0, 1), (0, 1, 0), grey)    # floor
    b.quad((0.5, 1.0, 0.5), (1, 0, 0), (0, 0, 1), (0, -1, 0), grey)   # ceiling
    b.quad((0.5, 0.5, 0.0), (1, 0, 0), (0, 1, 0), (0, 0, 1), grey)    # back wall
    b.quad((0.0, 0.5, 0.5), (0, 1, 0), (0, 0, 1), (1, 0, 0), red)     # left wall
    b.quad((1.0, 0.5, 0.5), (0, 1, 0), (0, 0, 1), (-1, 0, 0), green)  # right wall
    b.quad((0.5, 0.999, 0.5), (light_size, 0, 0), (0, 0, light_size), (0, -1, 0), light)
    if block:
        b.box((0.15, 0.0, 0.15), (0.4, 0.5, 0.4), grey)                 # tall block, 6 quads
    return grey


def cornell(width=64, height=64, depth=3) -> SceneArrays:
    """Cornell box: 12 axis-aligned quads (24 triangles) -- 5 walls (front open),
    one 0.2 x 0.2 area light (L_e = 15) below the ceiling, one 6-quad block.
    Lambertian albedo 0.7; left wall (0.7, 0, 0), right wall (0, 0.7, 0)."""
    b = _Builder()
    _cornell_room(b, 0.2)
    cam = pinhole((0.5, 0.5, 2.3), (0.5, 0.5, 0.0), (0, 1, 0), CORNELL_CAMERA_TAN, width / height)
    return b.build("cornell", cam, width, height, depth)


def cornell_spheres(width=512, height=512, depth=8, n_lon=100, n_lat=101) -> SceneArrays:
    """The Cornell box plus two UV spheres of 2 n_lon (n_lat - 1) = 20k triangles
    each (one modified-Phong glossy, exponent 50; one Lambertian), light
    shrunk to 0.05 x 0.05."""
    b = _Builder()
    _cornell_room(b, 0.05)
    gloss = b.add_material(material(PHONG, (0.7, 0.7, 0.7), phong_n=50.0))
    diff = b.add_material(material(LAMBERT, (0.7, 0.7, 0.7)))
    v, t = uv_sphere((0.7, 0.2, 0.35), 0.2, n_lon, n_lat)
    b.mesh(v, t, gloss)
    v, t = uv_sphere((0.4, 0.15, 0.7), 0.15, n_lon, n_lat)
    b.mesh(v, t, diff)
    cam = pinhole((0.5, 0.5, 2.3), (0.5, 0.5, 0.0), (0, 1, 0), CORNELL_CAMERA_TAN, width / height)
    return b.build("cornell_spheres", cam, width, height, depth)


def furnace(width=16, height=16, depth=8, albedo=0.5, emission=1.0) -> SceneArrays:
    """White furnace: closed unit cube, every face Lambertian with albedo rho and
    inward-facing emission L_e; the camera sits inside.  Every path has
    F = L_e (1 - rho^(depth+1)) / (1 - rho) in every channel."""
    b = _Builder()
    m = b.add_material(material(LAMBERT, (albedo,) * 3, emission=(emission,) * 3))
    b.box((0, 0, 0), (1, 1, 1), m, inward=True)
    cam = pinhole((0.5, 0.5, 0.5), (0.5, 0.5, 0.0), (0, 1, 0), 1.0, width / height)
    return b.build("furnace", cam, width, height, depth)


def empty(width=8, height=8, depth=2) -> SceneArrays:
    """No triangles: every path misses, F = 0 everywhere."""
    b = _Builder()
    b.add_material(material(LAMBERT, (0.5, 0.5, 0.5)))
    cam = pinhole((0, 0, 1), (0, 0, 0), (0, 1, 0), 0.5, width / height)
    return b.build("empty", cam, width, height, depth)


def glass_furnace(width=16, height=16, depth=6, albedo=0.5) -> SceneArrays:
    """A glass sphere (IOR 1.5) inside a furnace cube: exercises the dielectric
    sampler inside a closed scene (F is not constant)."""
    b = _Builder()
    m = b.add_material(material(LAMBERT, (albedo,) * 3, emission=(1.0, 1.0, 1.0)))
    g = b.add_material(material(DIELECTRIC, (1, 1, 1), ior=1.5))
    b.box((0, 0, 0), (1, 1, 1), m, inward=True)
    v, t = uv_sphere((0.5, 0.5, 0.25), 0.15, 24, 13)
    b.mesh(v, t, g)
    cam = pinhole((0.5, 0.5, 0.9), (0.5, 0.5, 0.0), (0, 1, 0), 0.6, width / height)
    return b.build("glass_furnace", cam, width, height, depth)


def _subdivided_box(lo, hi, s):
    """Axis-aligned box with every face split into an s x s grid of quads
    (12 s^2 triangles), outward winding."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    g = np.linspace(0.0, 1.0, s + 1)
    verts, tris = [], []
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for side in (0, 1):
            U, V = np.meshgrid(g, g, indexing="ij")
            p = np.zeros((s + 1, s + 1, 3))
            p[..., ax] = hi[ax] if side else lo[ax]
            p[..., o1] = lo[o1] + U * (hi[o1] - lo[o1])
            p[..., o2] = lo[o2] + V * (hi[o2] - lo[o2])
            base = sum(len(v) for v in verts)
            verts.append(p.reshape(-1, 3))
            idx = np.arange((s + 1) * (s + 1)).reshape(s + 1, s + 1) + base
            a, b, c, d = idx[:-1, :-1], idx[1:, :-1], idx[1:, 1:], idx[:-1, 1:]
            t = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
            # orient outward: normal along +ax on the hi side, -ax on the lo side
            n = np.zeros(3)
            n[ax] = 1.0 if side else -1.0
            v = np.concatenate(verts)
            nn = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]) @ n
            t[nn < 0] = t[nn < 0][:, [0, 2, 1]]
            tris.append(t)
    return np.concatenate(verts), np.concatenate(tris)


def random_boxes(seed, n_tris, width, height, depth) -> SceneArrays:
    """Seeded procedural interior: a closed room (grey walls, one ceiling
    light) holding random axis-aligned boxes whose faces are subdivided so the
    scene has about n_tris triangles; Lambertian and glossy boxes."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    wall = b.add_material(material(LAMBERT, (0.65, 0.65, 0.65)))
    light = b.add_material(material(LAMBERT, (0.0, 0.0, 0.0), emission=(12.0, 12.0, 12.0)))
    b.box((0, 0, 0), (1, 1, 1), wall, inward=True)
    lx, lz = rng.uniform(0.3, 0.7, size=2)
    b.quad((lx, 0.998, lz), (0.25, 0, 0), (0, 0, 0.25), (0, -1, 0), light)
    nb = int(rng.integers(6, 25))
    s = max(1, int(round(np.sqrt(max(n_tris - 14, 12) / (12.0 * nb)))))
    for _ in range(nb):
        size = rng.uniform(0.05, 0.3, size=3)
        lo = rng.uniform(0.02, 0.98 - size)
        lo[1] = rng.uniform(0.0, 0.6)
        hi = np.minimum(lo + size, 0.97)
        if rng.random() < 0.3:
            m = b.add_material(material(PHONG, tuple(rng.uniform(0.4, 0.9, 3)), phong_n=float(rng.uniform(10, 100))))
        else:
            m = b.add_material(material(LAMBERT, tuple(rng.uniform(0.2, 0.85, 3))))
        v, t = _subdivided_box(lo, hi, s)
        b.mesh(v, t, m)
    cam = pinhole((0.5, 0.45, 0.97), (0.5, 0.4, 0.0), (0, 1, 0), 0.75, width / height)
    return b.build(f"random_boxes_{seed}", cam, width, height, depth)


def batched_workload(seed=0, n_scenes=64):
    """The 64-scene batch: triangle count log-uniform in [1k, 200k], image side
    log-uniform in [128, 1024] rounded to a multiple of 16, depth uniform in
    {4..10}.  Returns a list of SceneArrays (one chain per pixel is the
    intended chain count)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scenes):
        n_tris = int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
        side = int(np.exp(rng.uniform(np.log(128), np.log(1024))))
        side = max(128, min(1024, 16 * int(round(side / 16))))
        depth = int(rng.integers(4, 11))
        out.append(random_boxes(seed * 1000 + k, n_tris, side, side, depth))
    return out


def caustic_slit(width=1024, height=1024, depth=10, n_lon=200, n_lat=201, slit=0.02) -> SceneArrays:
    """A glass UV sphere (IOR 1.5, 2 n_lon (n_lat - 1) = 80k triangles) over a
    diffuse floor, lit by an area light that shines through a `slit`-wide gap
    in an opaque occluder: the light reaches the scene only through the slit,
    and the sphere focuses it into a caustic on the floor."""
    b = _Builder()
    floor = b.add_material(material(LAMBERT, (0.8, 0.8, 0.8)))
    black = b.add_material(material(LAMBERT, (0.0, 0.0, 0.0)))
    glass = b.add_material(material(DIELECTRIC, (1.0, 1.0, 1.0), ior=1.5))
    light = b.add_material(material(LAMBERT, (0.0, 0.0, 0.0), emission=(50.0, 50.0, 50.0)))
    b.quad((0.5, 0.0, 0.5), (3.0, 0, 0), (0, 0, 3.0), (0, 1, 0), floor)
    b.quad((0.5, 2.0, 0.5), (0.6, 0, 0), (0, 0, 0.6), (0, -1, 0), light)
    z0, z1 = 0.5 - slit / 2, 0.5 + slit / 2
    lo_w = z0 - (-0.5)
    hi_w = 1.5 - z1
    for sgn in (1, -1):   # the occluder is opaque from both sides
        b.quad((0.5, 1.4, -0.5 + lo_w / 2), (2.0, 0, 0), (0, 0, lo_w), (0, sgn, 0), black)
        b.quad((0.5, 1.4, z1 + hi_w / 2), (2.0, 0, 0), (0, 0, hi_w), (0, sgn, 0), black)
    v, t = uv_sphere((0.5, 0.3, 0.62), 0.25, n_lon, n_lat)
    b.mesh(v, t, glass)
    cam = pinhole((0.5, 1.1, 2.3), (0.5, 0.15, 0.55), (0, 1, 0), 0.45, width / height)
    return b.build("caustic_slit", cam, width, height, depth)


def fbm_value_noise(x, z, seed, octaves=6, base=4.0, gain=0.5):
    """Fractal sum of seeded value noise on [0,1]^2: octave o samples a lattice
    of uniform values (spacing 1 / (base 2^o)) with smoothstep-weighted
    bilinear interpolation; weights gain^o, normalised to [0, 1]."""
    rng = np.random.default_rng(seed)
    x, z = np.asarray(x, np.float64), np.asarray(z, np.float64)
    h = np.zeros(np.broadcast(x, z).shape)
    amp, freq, norm = 1.0, float(base), 0.0
    for _ in range(octaves):
        n = int(np.ceil(freq)) + 2
        lat = rng.random((n, n))
        gx, gz = x * freq, z * freq
        i, j = np.floor(gz).astype(np.int64), np.floor(gx).astype(np.int64)
        fz, fx = gz - i, gx - j
        sz, sx = fz * fz * (3 - 2 * fz), fx * fx * (3 - 2 * fx)
        a = lat[i, j] + (lat[i, j + 1] - lat[i, j]) * sx
        b = lat[i + 1, j] + (lat[i + 1, j + 1] - lat[i + 1, j]) * sx
        h += amp * (a + (b - a) * sz)
        norm += amp
        amp *= gain
        freq *= 2.0
    return h / norm


def terrain(width=2048, height=2048, depth=12, n_grid=1000, n_lights=256, seed=5, relief=0.25) -> SceneArrays:
    """A grid terrain of n_grid^2 vertices over [0,1]^2 (2 (n_grid - 1)^2
    triangles, about 2M by default) displaced by seeded fBm value noise, lit
    only by n_lights small quad emitters (0.012 wide, facing down, 0.03 above
    the ground) with L_e log-uniform in [1, 100]; open sky."""
    b = _Builder()
    ground = b.add_material(material(LAMBERT, (0.6, 0.6, 0.6)))
    g = np.linspace(0.0, 1.0, n_grid)
    X, Z = np.meshgrid(g, g)                       # X along columns (j), Z along rows (i)
    Y = relief * fbm_value_noise(X, Z, seed)
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    i, j = np.meshgrid(np.arange(n_grid - 1), np.arange(n_grid - 1), indexing="ij")
    a = (i * n_grid + j).ravel()
    bb, c, d = a + 1, a + n_grid, a + n_grid + 1
    tris = np.concatenate([np.stack([a, c, bb], 1), np.stack([bb, c, d], 1)])   # normals point up
    b.mesh(verts, tris, ground)
    rng = np.random.default_rng(seed + 1)
    lx, lz = rng.uniform(0.05, 0.95, n_lights), rng.uniform(0.05, 0.95, n_lights)
    ly = relief * fbm_value_noise(lx, lz, seed) + 0.03
    le = np.exp(rng.uniform(np.log(1.0), np.log(100.0), n_lights))
    for k in range(n_lights):
        m = b.add_material(material(LAMBERT, (0.0, 0.0, 0.0), emission=(le[k], le[k], le[k])))
        b.quad((lx[k], ly[k], lz[k]), (0.012, 0, 0), (0, 0, 0.012), (0, -1, 0), m)
    cam = pinhole((0.5, 0.75, -0.35), (0.5, 0.05, 0.55), (0, 1, 0), 0.6, width / height)
    return b.build("terrain", cam, width, height, depth)


def by_name(name: str, **kw) -> SceneArrays:
    return {"cornell": cornell, "cornell_spheres": cornell_spheres, "furnace": furnace, "empty": empty,
            "glass_furnace": glass_furnace, "random_boxes": random_boxes, "caustic_slit": caustic_slit,
            "terrain": terrain}[name](**kw)
