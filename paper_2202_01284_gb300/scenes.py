"""Seeded synthetic scene generators (inputs only).

This module builds the procedural inputs that both the CUDA path and the FP64
oracle consume: triangle soups, per-shape material records, differentiable
parameter arrays (constant albedos, RGBA textures, roughness scalars), the
environment map and the pinhole cameras.  It holds none of the rendering
method's arithmetic (no sampling, no CDFs, no BSDF terms): every function here
only produces numbers that are then handed, unchanged, to both implementations.

The paper's benchmark scenes (Bitterli's Staircase, Living room and Glass of
water, Sec. 3.5) are not available, so the workloads below stand in for them:
  * ``cornell``      -- 36-triangle box with 5 constant albedos and a quad light.
  * ``cornell96``    -- the same room re-tessellated into 96 shapes with an
                        atlas-mapped 2048^2 RGBA texture and 96 roughness values.
  * ``spheres``      -- noise-displaced icospheres on a ground plane under an
                        environment map (sky gradient + sun disk), with a textured
                        diffuse, a rough GGX conductor and a smooth dielectric.
All arrays are float32 (the path's input precision) and fully determined by
their integer seeds.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
from typing import List, Optional

import numpy as np

# BSDF codes shared by both sides' marshalling code (numbers only).
BSDF_NONE = 0        # black: a path that reaches it stops (pure emitters)
BSDF_DIFFUSE = 1     # Lambertian, constant or textured albedo
BSDF_CONDUCTOR = 2   # rough GGX conductor with Schlick Fresnel
BSDF_DIELECTRIC = 3  # smooth dielectric interface
BSDF_BLEND = 4       # w * diffuse + (1 - w) * GGX(F0 = 0.04)


@dataclass
class Camera:
    origin: tuple
    target: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int


@dataclass
class Scene:
    """Triangle soup + per-shape material table + differentiable parameters."""
    vertices: np.ndarray            # [T,3,3] f32
    uvs: np.ndarray                 # [T,3,2] f32
    tri_shape: np.ndarray           # [T] i32
    # shape table (one record per shape)
    bsdf: np.ndarray                # [S] i32
    tex: np.ndarray                 # [S] i32  texture slot of the albedo, -1 = constant
    albedo_index: np.ndarray        # [S] i32  row of `albedo`, -1 = none
    rough_index: np.ndarray         # [S] i32  entry of `roughness`, -1 = fixed `alpha`
    alpha: np.ndarray               # [S] f32
    f0: np.ndarray                  # [S,3] f32
    eta: np.ndarray                 # [S] f32
    emission: np.ndarray            # [S,3] f32
    diffuse_weight: np.ndarray      # [S] f32 (blend only)
    # differentiable parameters
    albedo: np.ndarray              # [A,3] f32
    textures: List[np.ndarray]      # each [H,W,4] f32 (RGBA, alpha unused)
    roughness: np.ndarray           # [R] f32
    env: Optional[np.ndarray] = None  # [H,W,4] f32 equirectangular, row 0 = +y
    cameras: List[Camera] = field(default_factory=list)
    name: str = ""

    @property
    def n_tris(self) -> int:
        return int(self.vertices.shape[0])

    @property
    def n_shapes(self) -> int:
        return int(self.bsdf.shape[0])

    def translated(self, offsets) -> "Scene":
        """Copy with every shape's vertices moved by offsets[shape] ([S, 3])."""
        import copy
        off = np.asarray(offsets, np.float64).reshape(self.n_shapes, 3)
        s = copy.copy(self)
        v = self.vertices.astype(np.float64) + off[self.tri_shape][:, None, :]
        s.vertices = np.ascontiguousarray(v, dtype=np.float32)
        return s

    def camera_moved(self, offset) -> "Scene":
        """Copy with every camera's origin and target moved by offset ([3])."""
        import copy
        import dataclasses
        off = np.asarray(offset, np.float64).reshape(3)
        s = copy.copy(self)
        s.cameras = [dataclasses.replace(c, origin=tuple(float(x) for x in np.add(c.origin, off)),
                                         target=tuple(float(x) for x in np.add(c.target, off)))
                     for c in self.cameras]
        return s

    def with_params(self, albedo=None, textures=None, roughness=None) -> "Scene":
        import copy
        s = copy.copy(self)
        if albedo is not None:
            s.albedo = np.ascontiguousarray(albedo, dtype=np.float32)
        if textures is not None:
            s.textures = [np.ascontiguousarray(t, dtype=np.float32) for t in textures]
        if roughness is not None:
            s.roughness = np.ascontiguousarray(roughness, dtype=np.float32)
        return s


# ----------------------------------------------------------------------------
# small geometry helpers
# ----------------------------------------------------------------------------

def _quad(p0, p1, p2, p3):
    """Two triangles (p0,p1,p2), (p0,p2,p3); normal = (p1-p0) x (p2-p0)."""
    return [np.array([p0, p1, p2]), np.array([p0, p2, p3])]


_QUAD_UV = [np.array([[0, 0], [1, 0], [1, 1]], np.float32),
            np.array([[0, 0], [1, 1], [0, 1]], np.float32)]


def _box_faces(lo, hi):
    """Six outward-facing quads of an axis-aligned box, as corner lists."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    return [
        ((x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)),  # +z
        ((x1, y0, z0), (x0, y0, z0), (x0, y1, z0), (x1, y1, z0)),  # -z
        ((x1, y0, z1), (x1, y0, z0), (x1, y1, z0), (x1, y1, z1)),  # +x
        ((x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0)),  # -x
        ((x0, y1, z1), (x1, y1, z1), (x1, y1, z0), (x0, y1, z0)),  # +y
        ((x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)),  # -y
    ]


def _room_walls():
    """Inward-facing walls of the room [-1,1]x[0,2]x[-1,1], open at z=+1."""
    return {
        "floor": ((-1, 0, 1), (1, 0, 1), (1, 0, -1), (-1, 0, -1)),
        "ceiling": ((-1, 2, -1), (1, 2, -1), (1, 2, 1), (-1, 2, 1)),
        "back": ((-1, 0, -1), (1, 0, -1), (1, 2, -1), (-1, 2, -1)),
        "left": ((-1, 0, 1), (-1, 0, -1), (-1, 2, -1), (-1, 2, 1)),
        "right": ((1, 0, -1), (1, 0, 1), (1, 2, 1), (1, 2, -1)),
    }


SHORT_BOX = ((0.05, 0.0, -0.05), (0.65, 0.6, 0.55))
TALL_BOX = ((-0.65, 0.0, -0.6), (-0.05, 1.2, 0.0))
LIGHT_QUAD = ((-0.25, 1.99, -0.25), (0.25, 1.99, -0.25), (0.25, 1.99, 0.25), (-0.25, 1.99, 0.25))
LIGHT_RADIANCE = 15.0


def cornell_camera(width=64, height=64) -> Camera:
    return Camera((0.0, 1.0, 3.5), (0.0, 1.0, 0.0), (0.0, 1.0, 0.0), 40.0, width, height)


def _shape_table(n):
    return dict(
        bsdf=np.zeros(n, np.int32), tex=np.full(n, -1, np.int32),
        albedo_index=np.full(n, -1, np.int32), rough_index=np.full(n, -1, np.int32),
        alpha=np.full(n, 0.3, np.float32), f0=np.zeros((n, 3), np.float32),
        eta=np.full(n, 1.5, np.float32), emission=np.zeros((n, 3), np.float32),
        diffuse_weight=np.full(n, 0.8, np.float32))


# ----------------------------------------------------------------------------
# Cornell-style room, 36 triangles, 5 constant albedos
# ----------------------------------------------------------------------------

def cornell(seed: int = 2022, width: int = 64, height: int = 64) -> Scene:
    """36 triangles: 5 walls (10), two boxes (24), quad light (2).

    Shapes 0..4 carry the five RGB albedos (0 = floor+ceiling+back,
    1 = left, 2 = right, 3 = short box, 4 = tall box); shape 5 is the light
    (radiance 15, emitting toward -y, black BSDF).  Albedos ~ U[0.2,0.8]^3.
    """
    rng = np.random.default_rng(seed)
    albedo = rng.uniform(0.2, 0.8, size=(5, 3)).astype(np.float32)
    walls = _room_walls()
    tris, uvs, shp = [], [], []

    def add_quad(corners, shape):
        for t, uv in zip(_quad(*corners), _QUAD_UV):
            tris.append(t)
            uvs.append(uv)
            shp.append(shape)

    add_quad(walls["floor"], 0)
    add_quad(walls["ceiling"], 0)
    add_quad(walls["back"], 0)
    add_quad(walls["left"], 1)
    add_quad(walls["right"], 2)
    for f in _box_faces(*SHORT_BOX):
        add_quad(f, 3)
    for f in _box_faces(*TALL_BOX):
        add_quad(f, 4)
    add_quad(LIGHT_QUAD, 5)

    st = _shape_table(6)
    st["bsdf"][:5] = BSDF_DIFFUSE
    st["albedo_index"][:5] = np.arange(5)
    st["bsdf"][5] = BSDF_NONE
    st["emission"][5] = LIGHT_RADIANCE
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.asarray(uvs, np.float32),
                 tri_shape=np.asarray(shp, np.int32), albedo=albedo, textures=[],
                 roughness=np.zeros(0, np.float32), env=None,
                 cameras=[cornell_camera(width, height)], name="cornell36", **st)


def cornell_target_albedo(albedo: np.ndarray) -> np.ndarray:
    """Target albedos of the tiny gradient workload: +0.05, clamped to 0.95."""
    return np.minimum(albedo + 0.05, 0.95).astype(np.float32)


# ----------------------------------------------------------------------------
# value noise (texture content and sphere displacement)
# ----------------------------------------------------------------------------

def _smooth(t):
    return t * t * (3.0 - 2.0 * t)


def value_noise_2d(height, width, channels, cell, seed, lo=0.0, hi=1.0) -> np.ndarray:
    """Lattice value noise: random values every `cell` texels, smoothstep-blended."""
    rng = np.random.default_rng(seed)
    gh, gw = height // cell + 2, width // cell + 2
    lat = rng.uniform(lo, hi, size=(gh, gw, channels))
    y = (np.arange(height) + 0.5) / cell
    x = (np.arange(width) + 0.5) / cell
    y0 = np.floor(y).astype(np.int64)
    x0 = np.floor(x).astype(np.int64)
    ty = _smooth(y - y0)[:, None, None]
    tx = _smooth(x - x0)[None, :, None]
    a = lat[y0][:, x0]
    b = lat[y0][:, x0 + 1]
    c = lat[y0 + 1][:, x0]
    d = lat[y0 + 1][:, x0 + 1]
    out = (a * (1 - tx) + b * tx) * (1 - ty) + (c * (1 - tx) + d * tx) * ty
    return out.astype(np.float32)


def value_noise_3d(points: np.ndarray, freq: float, seed: int, size: int = 32) -> np.ndarray:
    """Periodic 3-D lattice value noise in [0,1] evaluated at `points` [N,3]."""
    rng = np.random.default_rng(seed)
    lat = rng.uniform(0.0, 1.0, size=(size, size, size))
    p = points * freq
    i0 = np.floor(p).astype(np.int64)
    t = _smooth(p - i0)
    out = np.zeros(points.shape[0])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1])
                     * (t[:, 2] if dz else 1 - t[:, 2]))
                ix = (i0[:, 0] + dx) % size
                iy = (i0[:, 1] + dy) % size
                iz = (i0[:, 2] + dz) % size
                out += w * lat[ix, iy, iz]
    return out


def rgba_texture(size: int, seed: int, lo: float, hi: float, cell: int = 16) -> np.ndarray:
    rgb = value_noise_2d(size, size, 3, cell, seed, lo, hi)
    a = np.ones((size, size, 1), np.float32)
    return np.ascontiguousarray(np.concatenate([rgb, a], axis=2), dtype=np.float32)


# ----------------------------------------------------------------------------
# Cornell room re-tessellated into 96 shapes (texture + roughness gradients)
# ----------------------------------------------------------------------------

ATLAS_RES = 2048
ATLAS_CELL = 204
ATLAS_GRID = 10


def _atlas_uv(shape_id, s, t):
    cx, cy = shape_id % ATLAS_GRID, shape_id // ATLAS_GRID
    u = (cx * ATLAS_CELL + 1.0 + s * (ATLAS_CELL - 2.0)) / ATLAS_RES
    v = (cy * ATLAS_CELL + 1.0 + t * (ATLAS_CELL - 2.0)) / ATLAS_RES
    return (u, v)


def cornell96(seed: int = 2022, width: int = 512, height: int = 512, tex_res: int = ATLAS_RES) -> Scene:
    """96 shapes: 5 walls x (4x4 tiles) = 80, 12 box faces, light as 2x2 tiles.

    Every non-light shape uses the blend BSDF (0.8 textured diffuse +
    0.2 GGX with F0 = 0.04, roughness = its own entry of `roughness`).
    Texture: one RGBA atlas, cell k of a 10x10 grid of 204^2 texels per shape.
    """
    rng = np.random.default_rng(seed)
    tris, uvs, shp = [], [], []

    def lerp3(a, b, t):
        return tuple(a[i] + (b[i] - a[i]) * t for i in range(3))

    def add_tiled(corners, n, first_shape):
        p0, p1, p2, p3 = [np.array(c, np.float64) for c in corners]
        sid = first_shape
        for j in range(n):
            for i in range(n):
                s0, s1, t0, t1 = i / n, (i + 1) / n, j / n, (j + 1) / n

                def P(s, t):
                    a = p0 + (p1 - p0) * s
                    b = p3 + (p2 - p3) * s
                    return a + (b - a) * t
                q = [P(s0, t0), P(s1, t0), P(s1, t1), P(s0, t1)]
                quv = [_atlas_uv(sid, 0, 0), _atlas_uv(sid, 1, 0), _atlas_uv(sid, 1, 1), _atlas_uv(sid, 0, 1)]
                for tri_idx in ((0, 1, 2), (0, 2, 3)):
                    tris.append(np.array([q[k] for k in tri_idx]))
                    uvs.append(np.array([quv[k] for k in tri_idx]))
                    shp.append(sid)
                sid += 1
        return sid

    walls = _room_walls()
    sid = 0
    for name in ("floor", "ceiling", "back", "left", "right"):
        sid = add_tiled(walls[name], 4, sid)
    for box in (SHORT_BOX, TALL_BOX):
        for f in _box_faces(*box):
            sid = add_tiled(f, 1, sid)
    light_first = sid
    sid = add_tiled(LIGHT_QUAD, 2, sid)
    assert sid == 96

    st = _shape_table(96)
    st["bsdf"][:] = BSDF_BLEND
    st["tex"][:] = 0
    st["rough_index"][:] = np.arange(96)
    st["f0"][:] = 0.04
    st["diffuse_weight"][:] = 0.8
    st["bsdf"][light_first:] = BSDF_NONE
    st["tex"][light_first:] = -1
    st["rough_index"][light_first:] = -1
    st["emission"][light_first:] = LIGHT_RADIANCE
    roughness = rng.uniform(0.1, 0.5, size=96).astype(np.float32)
    tex = rgba_texture(tex_res, seed + 11, 0.2, 0.8)
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.asarray(uvs, np.float32),
                 tri_shape=np.asarray(shp, np.int32), albedo=np.zeros((0, 3), np.float32),
                 textures=[tex], roughness=roughness, env=None,
                 cameras=[cornell_camera(width, height)], name="cornell96", **st)


def cornell96_target_texture(tex: np.ndarray, seed: int = 2022) -> np.ndarray:
    """Seeded perturbation: base + 0.1 (noise - 0.5), clamped to [0.05, 0.95]."""
    n = value_noise_2d(tex.shape[0], tex.shape[1], 3, 16, seed + 23)
    out = tex.copy()
    out[..., :3] = np.clip(tex[..., :3] + 0.1 * (n - 0.5), 0.05, 0.95)
    return np.ascontiguousarray(out, dtype=np.float32)


# ----------------------------------------------------------------------------
# icosphere scene under an environment map
# ----------------------------------------------------------------------------

def icosphere(level: int):
    """Unit icosphere by repeated 4:1 midpoint subdivision; outward winding."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces, np.int64)
    # make the winding outward
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, V[F[:, 0]]) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def sky_env(width=512, height=256, sun_elev_deg=35.0, sun_azim_deg=60.0,
            sun_radius_deg=0.5, sun_radiance=2.0e4, supersample=8) -> np.ndarray:
    """Equirectangular sky: row 0 looks along +y, column angle phi from +x toward +z.

    Above the horizon the colour blends from (0.8,0.8,0.8) at the horizon to
    (0.3,0.5,1.0) at the zenith; below it is 0.2 grey.  A sun disk of the
    given angular radius is added with per-texel coverage (supersampled).
    """
    y = (np.arange(height) + 0.5) / height
    theta = y * np.pi
    elev = np.pi / 2 - theta
    t = np.clip(elev / (np.pi / 2), 0.0, 1.0)[:, None]
    horizon = np.array([0.8, 0.8, 0.8])
    zenith = np.array([0.3, 0.5, 1.0])
    row = horizon * (1 - t) + zenith * t
    row = np.where((elev < 0)[:, None], 0.2, row)
    img = np.repeat(row[:, None, :], width, axis=1)
    se, sa = math.radians(sun_elev_deg), math.radians(sun_azim_deg)
    sun = np.array([math.cos(se) * math.cos(sa), math.sin(se), math.cos(se) * math.sin(sa)])
    cosr = math.cos(math.radians(sun_radius_deg))
    th_s = math.pi / 2 - se
    y_lo = max(int((th_s - 0.05) / math.pi * height), 0)
    y_hi = min(int((th_s + 0.05) / math.pi * height) + 1, height)
    ph_s = sa % (2 * math.pi)
    x_c = ph_s / (2 * math.pi) * width
    span = int(0.05 / (2 * math.pi) * width / max(math.sin(th_s), 0.1)) + 2
    for yy in range(y_lo, y_hi):
        for xx in range(int(x_c) - span, int(x_c) + span + 1):
            xw = xx % width
            sub = (np.arange(supersample) + 0.5) / supersample
            th = (yy + sub[:, None]) / height * np.pi
            ph = (xx + sub[None, :]) / width * 2 * np.pi
            d = np.stack([np.sin(th) * np.cos(ph), np.cos(th) * np.ones_like(ph), np.sin(th) * np.sin(ph)], -1)
            cov = np.mean(d @ sun >= cosr)
            if cov > 0:
                img[yy, xw] = img[yy, xw] * (1 - cov) + sun_radiance * cov
    out = np.concatenate([img, np.ones((height, width, 1))], axis=2)
    return np.ascontiguousarray(out, dtype=np.float32)


def spheres(seed: int = 2022, n_spheres: int = 32, level: int = 4, grid=(8, 4),
            ground_quads: int = 128, ground_size=(12.0, 6.0), tex_res: int = 1024,
            width: int = 1024, height: int = 1024, env_size=(512, 256)) -> Scene:
    """Noise-displaced icospheres on a jittered grid over a textured ground plane.

    Sphere i uses BSDF i mod 3 (textured diffuse, GGX conductor with alpha ~
    U[0.1,0.5] and F0 ~ U[0.5,1]^3, dielectric eta = 1.5).  The ground is a
    textured diffuse plane of `ground_quads`^2 quads.  Default sizes give
    32 x 5,120 + 32,768 = 196,608 triangles.
    """
    rng = np.random.default_rng(seed)
    V0, F = icosphere(level)
    gx, gz = grid
    sx, sz = ground_size
    tris, uvs, shp = [], [], []
    n_shapes = n_spheres + 1
    st = _shape_table(n_shapes)
    roughness = np.zeros(0, np.float32)
    rough_list = []
    cell_x, cell_z = sx / gx, sz / gz
    for i in range(n_spheres):
        cx_i, cz_i = i % gx, (i // gx) % gz
        r = rng.uniform(0.3, 0.8) * min(cell_x, cell_z) / 1.8
        cx = -sx / 2 + (cx_i + 0.5) * cell_x + rng.uniform(-0.15, 0.15) * cell_x
        cz = -sz / 2 + (cz_i + 0.5) * cell_z + rng.uniform(-0.15, 0.15) * cell_z
        disp = value_noise_3d(V0 + i * 7.31, 4.0, seed + 101)
        V = V0 * (r * (1.0 + 0.1 * disp))[:, None] + np.array([cx, r, cz])
        T = V[F]
        u = np.arctan2(V0[:, 2], V0[:, 0]) / (2 * np.pi) + 0.5
        v = np.arccos(np.clip(V0[:, 1], -1, 1)) / np.pi
        UV = np.stack([u, v], -1)[F]
        tris.append(T)
        uvs.append(UV)
        shp.append(np.full(F.shape[0], i, np.int32))
        kind = i % 3
        if kind == 0:
            st["bsdf"][i] = BSDF_DIFFUSE
            st["tex"][i] = 0
        elif kind == 1:
            st["bsdf"][i] = BSDF_CONDUCTOR
            st["rough_index"][i] = len(rough_list)
            rough_list.append(rng.uniform(0.1, 0.5))
            st["f0"][i] = rng.uniform(0.5, 1.0, size=3)
        else:
            st["bsdf"][i] = BSDF_DIELECTRIC
            st["eta"][i] = 1.5
    # ground plane (normal +y)
    n = ground_quads
    xs = np.linspace(-sx / 2, sx / 2, n + 1)
    zs = np.linspace(-sz / 2, sz / 2, n + 1)
    X, Z = np.meshgrid(xs, zs, indexing="xy")
    P = np.stack([X, np.zeros_like(X), Z], -1)
    Uc = np.stack([(X + sx / 2) / sx, (Z + sz / 2) / sz], -1)
    a, b = P[:-1, :-1], P[:-1, 1:]
    c, d = P[1:, 1:], P[1:, :-1]
    ua, ub, uc, ud = Uc[:-1, :-1], Uc[:-1, 1:], Uc[1:, 1:], Uc[1:, :-1]
    # winding so that (p1-p0) x (p2-p0) points to +y
    t1 = np.stack([a, d, c], 2).reshape(-1, 3, 3)
    t2 = np.stack([a, c, b], 2).reshape(-1, 3, 3)
    u1 = np.stack([ua, ud, uc], 2).reshape(-1, 3, 2)
    u2 = np.stack([ua, uc, ub], 2).reshape(-1, 3, 2)
    G = np.concatenate([t1, t2])
    GU = np.concatenate([u1, u2])
    tris.append(G)
    uvs.append(GU)
    shp.append(np.full(G.shape[0], n_spheres, np.int32))
    st["bsdf"][n_spheres] = BSDF_DIFFUSE
    st["tex"][n_spheres] = 0
    roughness = np.asarray(rough_list, np.float32)
    tex = rgba_texture(tex_res, seed + 13, 0.15, 0.85, cell=32)
    env = sky_env(*env_size)
    cam = Camera((0.0, 3.2, 8.5), (0.0, 0.35, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    return Scene(vertices=np.concatenate(tris).astype(np.float32),
                 uvs=np.concatenate(uvs).astype(np.float32),
                 tri_shape=np.concatenate(shp).astype(np.int32), albedo=np.zeros((0, 3), np.float32),
                 textures=[tex], roughness=roughness, env=env, cameras=[cam],
                 name=f"spheres{n_spheres}x{20 * 4 ** level}", **st)


def spheres_target_texture(tex: np.ndarray, seed: int = 2022) -> np.ndarray:
    n = value_noise_2d(tex.shape[0], tex.shape[1], 3, 32, seed + 29)
    out = tex.copy()
    out[..., :3] = np.clip(tex[..., :3] + 0.1 * (n - 0.5), 0.05, 0.95)
    return np.ascontiguousarray(out, dtype=np.float32)


# ----------------------------------------------------------------------------
# closed-form test scenes
# ----------------------------------------------------------------------------

def furnace(albedo: float = 0.5, emission: float = 1.0, width=16, height=16) -> Scene:
    """Closed inward-facing cube [-1,1]^3: every face diffuse albedo `a` AND emitting E.

    Emission is one-sided along the inward normal.  With BSDF sampling only,
    every path has radiance E * sum_{k<D} a^k exactly.
    """
    tris, uvs = [], []
    for f in _box_faces((-1, -1, -1), (1, 1, 1)):
        # reverse corner order -> inward normals
        q = f[::-1]
        for t, uv in zip(_quad(*q), _QUAD_UV):
            tris.append(t)
            uvs.append(uv)
    st = _shape_table(1)
    st["bsdf"][0] = BSDF_DIFFUSE
    st["albedo_index"][0] = 0
    st["emission"][0] = emission
    cam = Camera((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), (0.0, 1.0, 0.0), 60.0, width, height)
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.asarray(uvs, np.float32),
                 tri_shape=np.zeros(12, np.int32), albedo=np.full((1, 3), albedo, np.float32),
                 textures=[], roughness=np.zeros(0, np.float32), env=None, cameras=[cam],
                 name="furnace", **st)


def lit_plane(albedo: float = 0.6, env_radiance: float = 1.0, env_size=(64, 32),
              width=16, height=16) -> Scene:
    """Huge diffuse plane y=0 (normal +y) under a uniform environment of radiance L."""
    s = 1.0e4
    q = ((-s, 0, s), (s, 0, s), (s, 0, -s), (-s, 0, -s))
    tris = _quad(*q)
    st = _shape_table(1)
    st["bsdf"][0] = BSDF_DIFFUSE
    st["albedo_index"][0] = 0
    env = np.full((env_size[1], env_size[0], 4), env_radiance, np.float32)
    env[..., 3] = 1.0
    cam = Camera((0.0, 1.0, 0.0), (0.0, 1.0 - math.sin(math.radians(40)), -math.cos(math.radians(40))),
                 (0.0, 1.0, 0.0), 70.0, width, height)
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.asarray(_QUAD_UV, np.float32),
                 tri_shape=np.zeros(2, np.int32), albedo=np.full((1, 3), albedo, np.float32),
                 textures=[], roughness=np.zeros(0, np.float32), env=env, cameras=[cam],
                 name="lit_plane", **st)


def glass_sphere(eta: float = 1.5, env_radiance: float = 1.0, inside: bool = False, level: int = 3,
                 width=16, height=16) -> Scene:
    """A closed smooth-dielectric icosphere of radius 1 (outward winding) at the
    origin under a uniform environment of radiance L.

    With `inside`, the camera sits at the centre, inside the glass; otherwise it
    looks at the sphere from outside, so that the image shows the sphere and the
    sky around it.  Transport through a lossless interface keeps L / n^2, so a
    path that leaves into the sky carries L (camera outside) or eta^2 L (camera
    inside the glass).
    """
    V, F = icosphere(level)
    tris = V[F]
    st = _shape_table(1)
    st["bsdf"][0] = BSDF_DIELECTRIC
    st["eta"][0] = eta
    env = np.full((16, 32, 4), env_radiance, np.float32)
    env[..., 3] = 1.0
    if inside:
        cam = Camera((0.0, 0.0, 0.0), (0.3, 0.2, -1.0), (0.0, 1.0, 0.0), 90.0, width, height)
    else:
        cam = Camera((0.0, 0.4, 3.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.zeros((len(F), 3, 2), np.float32),
                 tri_shape=np.zeros(len(F), np.int32), albedo=np.zeros((0, 3), np.float32), textures=[],
                 roughness=np.zeros(0, np.float32), env=env, cameras=[cam], name="glass_sphere", **st)


def occluder_sky(center=(0.15, 0.1), depth=3.0, side=0.4, env_radiance=1.0, width=64, height=64,
                 vfov_deg=40.0) -> Scene:
    """A black square facing a pinhole camera under a uniform environment.

    Camera at the origin looking along -z; the square (shape 0, two triangles)
    spans center +- side/2 in x and y at z = -depth.  The image is the
    environment radiance outside the square's projection and 0 inside, so the
    summed image changes with the square's depth by a closed form (its projected
    area is (side/depth)^2 on the image plane at unit distance) and not at all
    with a move parallel to the image plane.
    """
    cx, cy = center
    h = 0.5 * side
    q = ((cx - h, cy - h, -depth), (cx + h, cy - h, -depth), (cx + h, cy + h, -depth), (cx - h, cy + h, -depth))
    tris = _quad(*q)
    st = _shape_table(1)
    st["bsdf"][0] = BSDF_NONE
    env = np.full((16, 32, 4), env_radiance, np.float32)
    env[..., 3] = 1.0
    cam = Camera((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), (0.0, 1.0, 0.0), vfov_deg, width, height)
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.asarray(_QUAD_UV, np.float32),
                 tri_shape=np.zeros(2, np.int32), albedo=np.zeros((0, 3), np.float32), textures=[],
                 roughness=np.zeros(0, np.float32), env=env, cameras=[cam], name="occluder_sky", **st)


def shadow_scene(light=(-1.2, 2.0, 0.0), light_half=0.25, occluder=(-0.6, 0.8, 0.0), occluder_half=0.3,
                 camera=((1.6, 0.5, 0.0), (-0.2, 0.0, 0.0)), vfov_deg=40.0, width=64, height=64,
                 radiance=20.0, floor_bsdf=BSDF_DIFFUSE, floor_alpha=0.3) -> Scene:
    """A floor, a square area light and a square occluder casting a shadow.

    Shapes: 0 floor (y = 0, |x|,|z| <= 2; diffuse with albedo row 0, or a GGX
    conductor of roughness floor_alpha and F0 (0.9, 0.7, 0.5), or a blend), 1 light
    (facing -y, radiance `radiance`, black BSDF), 2 occluder (horizontal, diffuse,
    albedo row 1).  Nothing else: rays that miss see black.
    """
    tris, uvs, shp = [], [], []

    def add(corners, shape):
        for t, uv in zip(_quad(*corners), _QUAD_UV):
            tris.append(t)
            uvs.append(uv)
            shp.append(shape)

    add(((-2, 0, 2), (2, 0, 2), (2, 0, -2), (-2, 0, -2)), 0)
    lx, ly, lz = light
    h = light_half
    add(((lx - h, ly, lz - h), (lx + h, ly, lz - h), (lx + h, ly, lz + h), (lx - h, ly, lz + h)), 1)
    ox, oy, oz = occluder
    h = occluder_half
    add(((ox - h, oy, oz + h), (ox + h, oy, oz + h), (ox + h, oy, oz - h), (ox - h, oy, oz - h)), 2)
    st = _shape_table(3)
    st["bsdf"][[0, 2]] = BSDF_DIFFUSE
    st["bsdf"][0] = floor_bsdf
    st["alpha"][0] = floor_alpha
    st["f0"][0] = (0.9, 0.7, 0.5) if floor_bsdf == BSDF_CONDUCTOR else (0.04, 0.04, 0.04)
    st["albedo_index"][0] = 0
    st["albedo_index"][2] = 1
    st["bsdf"][1] = BSDF_NONE
    st["emission"][1] = radiance
    albedo = np.array([[0.7, 0.6, 0.5], [0.3, 0.5, 0.4]], np.float32)
    cam = Camera(tuple(camera[0]), tuple(camera[1]), (0.0, 1.0, 0.0), vfov_deg, width, height)
    return Scene(vertices=np.asarray(tris, np.float32), uvs=np.asarray(uvs, np.float32),
                 tri_shape=np.asarray(shp, np.int32), albedo=albedo, textures=[],
                 roughness=np.zeros(0, np.float32), env=None, cameras=[cam], name="shadow", **st)


# ----------------------------------------------------------------------------
# user meshes
# ----------------------------------------------------------------------------

def load_obj(path_or_text: str):
    """Minimal Wavefront OBJ reader: `v`, `vt`, `f` (polygons fanned into
    triangles, negative indices allowed) and `o` / `g` groups.  Returns
    (vertices [T,3,3] f32, uvs [T,3,2] f32, group [T] i32, group names).  No
    materials, normals or other statements (they are ignored)."""
    import os
    text = open(path_or_text).read() if os.path.exists(path_or_text) else path_or_text
    pos, uv, tris, tuvs, grp, names = [], [], [], [], [], []
    current = -1
    for line in text.splitlines():
        parts = line.split("#", 1)[0].split()
        if not parts:
            continue
        key = parts[0]
        if key == "v":
            pos.append([float(x) for x in parts[1:4]])
        elif key == "vt":
            uv.append([float(x) for x in parts[1:3]] + [0.0] * (2 - len(parts[1:3])))
        elif key in ("o", "g"):
            names.append(" ".join(parts[1:]) or f"group{len(names)}")
            current = len(names) - 1
        elif key == "f":
            if current < 0:
                names.append("default")
                current = 0
            corners = []
            for c in parts[1:]:
                idx = c.split("/")
                vi = int(idx[0])
                vi = vi - 1 if vi > 0 else len(pos) + vi
                ti = None
                if len(idx) > 1 and idx[1]:
                    ti = int(idx[1])
                    ti = ti - 1 if ti > 0 else len(uv) + ti
                corners.append((vi, ti))
            for k in range(1, len(corners) - 1):
                tri = (corners[0], corners[k], corners[k + 1])
                tris.append([pos[v] for v, _ in tri])
                tuvs.append([uv[t] if t is not None else [0.0, 0.0] for _, t in tri])
                grp.append(current)
    if not tris:
        raise ValueError("no faces in the OBJ input")
    return (np.asarray(tris, np.float32), np.asarray(tuvs, np.float32), np.asarray(grp, np.int32), names)


def mesh_scene(vertices, uvs=None, tri_shape=None, bsdf=None, albedo=None, emission=None, alpha=None,
               env=None, cameras=(), name="mesh") -> Scene:
    """A scene from user triangles: vertices [T,3,3], optional uvs [T,3,2] and a
    shape id per triangle [T] (default: one shape).  Per shape: bsdf codes
    (default diffuse), constant RGB albedos (default 0.5), emission, GGX alpha."""
    v = np.ascontiguousarray(vertices, np.float32).reshape(-1, 3, 3)
    t = v.shape[0]
    ts = np.zeros(t, np.int32) if tri_shape is None else np.ascontiguousarray(tri_shape, np.int32)
    n = int(ts.max()) + 1
    st = _shape_table(n)
    st["bsdf"][:] = BSDF_DIFFUSE if bsdf is None else np.asarray(bsdf, np.int32)
    alb = np.full((n, 3), 0.5, np.float32) if albedo is None else np.asarray(albedo, np.float32).reshape(n, 3)
    st["albedo_index"][:] = np.arange(n)
    if emission is not None:
        st["emission"][:] = np.asarray(emission, np.float32).reshape(n, 3)
    if alpha is not None:
        st["alpha"][:] = np.asarray(alpha, np.float32)
    uv = np.zeros((t, 3, 2), np.float32) if uvs is None else np.ascontiguousarray(uvs, np.float32)
    return Scene(vertices=v, uvs=uv, tri_shape=ts, albedo=alb, textures=[], roughness=np.zeros(0, np.float32),
                 env=None if env is None else np.ascontiguousarray(env, np.float32), cameras=list(cameras),
                 name=name, **st)


# ----------------------------------------------------------------------------
# batched-launch workload: many cameras of uneven size over several scenes
# ----------------------------------------------------------------------------

@dataclass
class BatchCamera:
    scene: int
    camera: Camera
    spp: int


def batch_cameras(n_cameras=64, n_scenes=3, seed=2022, lo=128, hi=1024,
                  spp_choices=(4, 8, 16, 32, 64)) -> List[BatchCamera]:
    """Cameras with sizes log-uniform in [lo, hi] per side, assigned round-robin."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_cameras):
        w = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        h = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        spp = int(rng.choice(spp_choices))
        ang = rng.uniform(-0.6, 0.6)
        dist = rng.uniform(7.0, 10.0)
        cam = Camera((dist * math.sin(ang), rng.uniform(2.0, 4.0), dist * math.cos(ang)),
                     (0.0, 0.4, 0.0), (0.0, 1.0, 0.0), float(rng.uniform(35, 55)), w, h)
        out.append(BatchCamera(i % n_scenes, cam, spp))
    return out


def batch_scenes(seed=2022, sizes=("10k", "200k", "2M")) -> List[Scene]:
    out = []
    for s in sizes:
        if s == "10k":
            out.append(spheres(seed, n_spheres=2, level=4, grid=(2, 1), ground_quads=8,
                               ground_size=(4.0, 2.0), tex_res=256))
        elif s == "200k":
            out.append(spheres(seed))
        elif s == "2M":
            out.append(spheres(seed, n_spheres=24, level=6, grid=(6, 4)))
        else:
            raise ValueError(s)
    return out


# ----------------------------------------------------------------------------
# radiance-cache inputs: initial weights and synthetic records
# ----------------------------------------------------------------------------

MLP_N_PARAMS = 5 * 64 * 64 + 3 * 64


def mlp_init_weights(seed: int = 2022) -> np.ndarray:
    """Uniform +-sqrt(6/64) initial weights in the flat layout (layer l at l*4096 as
    [out][in], then the [3][64] head)."""
    rng = np.random.default_rng(seed)
    a = math.sqrt(6.0 / 64.0)
    return rng.uniform(-a, a, size=MLP_N_PARAMS).astype(np.float32)


def random_cache_records(n: int, seed: int, box_lo=(-1, 0, -1), box_hi=(1, 2, 1)):
    """Raw records (position in the box, unit direction, unit normal, roughness) and
    smooth synthetic RGB targets (a fixed function of the inputs, for training tests)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(box_lo, np.float64), np.asarray(box_hi, np.float64)
    p = lo + (hi - lo) * rng.random((n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    nn = rng.normal(size=(n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    a = rng.uniform(0.1, 1.0, size=(n, 1))
    raw = np.concatenate([p, d, nn, a], 1).astype(np.float32)
    x = (p - lo) / (hi - lo)
    t = np.stack([0.5 + 0.4 * np.sin(3 * x[:, 0] + d[:, 1]),
                  0.4 + 0.3 * np.cos(2 * x[:, 1] - nn[:, 2]),
                  0.3 + 0.2 * x[:, 2] * (1 + d[:, 0])], 1)
    return raw, t.astype(np.float32)
