"""Seeded synthetic scenes and cameras for the per-frame atlasing path.

This module only makes inputs: triangle meshes (float32 positions [V][3], uint32
CCW index triples [T][3]) and row-major float32 view-projection matrices
(clip = M . [p, 1]).  It holds none of the atlasing arithmetic, so both the CUDA
path and the CPU oracle can be fed from it without sharing any of the method.

The scenes stand in for the paper's Computer Graphics Archive scenes (Sec. 6,
Appendix B "Test Corpus"), which are not available here:

* ``grid_scene``      - a 64x64-vertex heightfield patch (7,938 triangles),
                        z = 0.2 sin(3x) cos(2y) + U(-0.02, 0.02).
* ``icosphere_scene`` - N icospheres at subdivision 5 (20,480 triangles each),
                        radially displaced by 4-octave lattice value noise, then
                        randomly rotated, scaled (0.5-2) and placed in a 50^3 box.
* ``instanced_grid_scene`` - many seeded copies of the heightfield patch.

Cameras are 45 degree vertical-FOV pinhole cameras (OpenGL conventions: the near
plane is z_clip = -w_clip, front faces are CCW on screen).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Scene:
    pos: np.ndarray  # float32 [V, 3]
    idx: np.ndarray  # uint32 [T, 3], CCW seen from outside / above

    @property
    def V(self) -> int:
        return int(self.pos.shape[0])

    @property
    def T(self) -> int:
        return int(self.idx.shape[0])


# --------------------------------------------------------------------------- cameras

def perspective(fovy_deg: float, aspect: float, near: float, far: float) -> np.ndarray:
    """OpenGL-style perspective matrix (float64), maps z_eye=-near to z_ndc=-1."""
    f = 1.0 / np.tan(np.radians(fovy_deg) * 0.5)
    P = np.zeros((4, 4), dtype=np.float64)
    P[0, 0] = f / aspect
    P[1, 1] = f
    P[2, 2] = (far + near) / (near - far)
    P[2, 3] = 2.0 * far * near / (near - far)
    P[3, 2] = -1.0
    return P


def look_at(eye, target, up) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    V = np.eye(4, dtype=np.float64)
    V[0, :3] = s
    V[1, :3] = u
    V[2, :3] = -f
    V[0, 3] = -s @ eye
    V[1, 3] = -u @ eye
    V[2, 3] = f @ eye
    return V


def view_proj(eye, target, up, width: int, height: int, fovy_deg: float = 45.0,
              near: float = 0.05, far: float = 100.0) -> np.ndarray:
    """Row-major float32 view-projection matrix, clip = M . [x, y, z, 1]."""
    M = perspective(fovy_deg, width / height, near, far) @ look_at(eye, target, up)
    return M.astype(np.float32)


def hemisphere_camera(seed: int, width: int, height: int, radius: float = 3.0) -> np.ndarray:
    """Seeded pose on the upper (z > 0) hemisphere of a radius, looking at the origin."""
    rng = np.random.default_rng([seed, 0xCA3E])
    az = rng.uniform(0.0, 2.0 * np.pi)
    el = np.radians(rng.uniform(25.0, 75.0))
    eye = radius * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    return view_proj(eye, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), width, height)


def box_camera(seed: int, width: int, height: int, half: float = 25.0) -> np.ndarray:
    """Seeded pose just inside one face of the [-half, half]^3 box, looking inwards."""
    rng = np.random.default_rng([seed, 0xB0C5])
    eye = rng.uniform(-0.6 * half, 0.6 * half, size=3)
    axis = int(rng.integers(0, 3))
    sign = 1.0 if rng.integers(0, 2) else -1.0
    eye[axis] = sign * 0.96 * half
    target = rng.uniform(-0.2 * half, 0.2 * half, size=3)
    d = target - eye
    up = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 * np.linalg.norm(d) else np.array([0.0, 1.0, 0.0])
    return view_proj(eye, target, up, width, height)


def spline_cameras(seed: int, n_frames: int, width: int, height: int, radius: float = 3.0):
    """n_frames view-projection matrices along a closed Catmull-Rom spline through
    seeded control points on the upper hemisphere, all looking at the origin."""
    rng = np.random.default_rng([seed, 0x5B1E])
    n_ctrl = 8
    az = np.sort(rng.uniform(0.0, 2.0 * np.pi, n_ctrl))
    el = np.radians(rng.uniform(25.0, 70.0, n_ctrl))
    rad = radius * rng.uniform(0.8, 1.2, n_ctrl)
    P = np.stack([rad * np.cos(el) * np.cos(az), rad * np.cos(el) * np.sin(az), rad * np.sin(el)], 1)
    out = []
    for f in range(n_frames):
        s = f * n_ctrl / n_frames
        i = int(np.floor(s))
        t = s - i
        p0, p1, p2, p3 = (P[(i + j - 1) % n_ctrl] for j in range(4))
        t2, t3 = t * t, t * t * t
        eye = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)
        eye[2] = max(eye[2], 0.3)
        out.append(view_proj(eye, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), width, height))
    return out


# --------------------------------------------------------------------------- meshes

def grid_scene(seed: int, n: int = 64) -> Scene:
    """n x n vertex heightfield on [-1, 1]^2: 2 (n-1)^2 CCW triangles seen from +z."""
    rng = np.random.default_rng([seed, 0x6121D])
    lin = np.linspace(-1.0, 1.0, n)
    y, x = np.meshgrid(lin, lin, indexing="ij")
    z = 0.2 * np.sin(3.0 * x) * np.cos(2.0 * y) + rng.uniform(-0.02, 0.02, size=x.shape)
    pos = np.stack([x, y, z], -1).reshape(-1, 3).astype(np.float32)
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    v00 = (i * n + j).ravel()
    v01 = v00 + 1
    v10 = v00 + n
    v11 = v10 + 1
    tri = np.empty((2 * v00.size, 3), dtype=np.uint32)
    tri[0::2] = np.stack([v00, v01, v11], 1)
    tri[1::2] = np.stack([v00, v11, v10], 1)
    return Scene(pos, tri)


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def icosphere(level: int = 5):
    """Unit icosphere: 10 * 4^level + 2 vertices, 20 * 4^level outward-CCW triangles.
    Children of a face are stored next to each other (spatially coherent order)."""
    v, f = _icosahedron()
    for _ in range(level):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
        key = np.minimum(e[:, 0], e[:, 1]) * (1 << 32) + np.maximum(e[:, 0], e[:, 1])
        ukey, inv = np.unique(key, return_inverse=True)
        a = ukey >> 32
        b = ukey & 0xFFFFFFFF
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], 0)
        F = f.shape[0]
        m01 = nv + inv[:F]
        m12 = nv + inv[F:2 * F]
        m20 = nv + inv[2 * F:]
        child = np.stack([np.stack([f[:, 0], m01, m20], 1),
                          np.stack([f[:, 1], m12, m01], 1),
                          np.stack([f[:, 2], m20, m12], 1),
                          np.stack([m01, m12, m20], 1)], 1)
        f = child.reshape(-1, 3)
    return v, f


def _hash3(ix, iy, iz, seed):
    """Integer lattice hash -> uniform [-1, 1) (splitmix64 finaliser on packed coords)."""
    h = (ix.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)
         ^ iy.astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F)
         ^ iz.astype(np.uint64) * np.uint64(0x165667B19E3779F9)
         ^ np.uint64((int(seed) * 0xD6E8FEB86659FD93) & 0xFFFFFFFFFFFFFFFF))
    h ^= h >> np.uint64(30)
    h *= np.uint64(0xBF58476D1CE4E5B9)
    h ^= h >> np.uint64(27)
    h *= np.uint64(0x94D049BB133111EB)
    h ^= h >> np.uint64(31)
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0


def value_noise(p: np.ndarray, seed: int) -> np.ndarray:
    """Trilinear lattice value noise with smoothstep weights, in [-1, 1]."""
    fl = np.floor(p)
    fr = p - fl
    w = fr * fr * (3.0 - 2.0 * fr)
    i = fl.astype(np.int64)
    out = np.zeros(p.shape[0])
    for dx in (0, 1):
        wx = w[:, 0] if dx else 1.0 - w[:, 0]
        for dy in (0, 1):
            wy = w[:, 1] if dy else 1.0 - w[:, 1]
            for dz in (0, 1):
                wz = w[:, 2] if dz else 1.0 - w[:, 2]
                out += wx * wy * wz * _hash3(i[:, 0] + dx, i[:, 1] + dy, i[:, 2] + dz, seed)
    return out


def fbm(p: np.ndarray, seed: int, octaves: int = 4, amplitude: float = 0.1,
        frequency: float = 2.0) -> np.ndarray:
    """Octave sum: frequency doubles and amplitude halves per octave."""
    out = np.zeros(p.shape[0])
    a, f = amplitude, frequency
    for o in range(octaves):
        out += a * value_noise(p * f, seed * 16 + o)
        a *= 0.5
        f *= 2.0
    return out


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def icosphere_scene(seed: int, n_spheres: int = 200, level: int = 5, half: float = 25.0) -> Scene:
    """n_spheres displaced icospheres baked into one world-space mesh."""
    rng = np.random.default_rng([seed, 0x1C05])
    v0, f0 = icosphere(level)
    nv, nf = v0.shape[0], f0.shape[0]
    pos = np.empty((n_spheres * nv, 3), dtype=np.float32)
    idx = np.empty((n_spheres * nf, 3), dtype=np.uint32)
    for s in range(n_spheres):
        disp = 1.0 + fbm(v0 * 1.5, seed * 1000 + s)
        p = v0 * disp[:, None]
        R = _random_rotation(rng)
        scale = rng.uniform(0.5, 2.0)
        trans = rng.uniform(-0.96 * half, 0.96 * half, size=3)
        pos[s * nv:(s + 1) * nv] = (scale * (p @ R.T) + trans).astype(np.float32)
        idx[s * nf:(s + 1) * nf] = (f0 + s * nv).astype(np.uint32)
    return Scene(pos, idx)


def instanced_grid_scene(seed: int, n_instances: int, n: int = 64, half: float = 6.0) -> Scene:
    """n_instances seeded copies of the heightfield patch (each its own noise),
    rotated about z, scaled 0.5-1.5 and spread over a [-half, half]^2 floor."""
    rng = np.random.default_rng([seed, 0x1257])
    base = grid_scene(seed, n)
    nv, nf = base.V, base.T
    pos = np.empty((n_instances * nv, 3), dtype=np.float32)
    idx = np.empty((n_instances * nf, 3), dtype=np.uint32)
    for s in range(n_instances):
        g = grid_scene(seed * 7919 + s + 1, n)
        a = rng.uniform(0.0, 2.0 * np.pi)
        c, sn = np.cos(a), np.sin(a)
        R = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
        scale = rng.uniform(0.5, 1.5)
        trans = np.array([rng.uniform(-half, half), rng.uniform(-half, half), rng.uniform(-0.3, 0.3)])
        pos[s * nv:(s + 1) * nv] = (scale * (g.pos.astype(np.float64) @ R.T) + trans).astype(np.float32)
        idx[s * nf:(s + 1) * nf] = base.idx + np.uint32(s * nv)
    return Scene(pos, idx)


# --------------------------------------------------------------------------- box sets

def lognormal_boxes(seed: int, n: int, mean_texels: float = 12.0, sigma: float = 1.0,
                    max_texels: float = 1024.0):
    """Footprints for the standalone packer: (fa, fb) uint32 in 1/256 texel with
    fb >= fa, log-normally distributed sides clipped to [0.25, max_texels] texels."""
    rng = np.random.default_rng([seed, 0xB0E5])
    s = np.exp(rng.normal(np.log(mean_texels), sigma, size=(n, 2)))
    s = np.clip(s, 0.25, max_texels)
    q = np.ceil(s * 256.0).astype(np.uint64)
    fa = np.minimum(q[:, 0], q[:, 1]).astype(np.uint32)
    fb = np.maximum(q[:, 0], q[:, 1]).astype(np.uint32)
    return fa, fb


# Named workloads -----------------------------------------------------------------

def heightfield_frame(seed: int = 1):
    """64x64-vertex heightfield, 480x270 view, ratio 1.0, 1024^2 atlas."""
    sc = grid_scene(seed)
    return sc, hemisphere_camera(seed, 480, 270), dict(width=480, height=270, ratio=1.0, atlas_log2=10)


def icosphere_frame(seed: int = 1, n_spheres: int = 200, ratio: float = 1.0):
    """200 displaced icospheres (4,096,000 tris), 1920x1080 view, 2048^2 atlas."""
    sc = icosphere_scene(seed, n_spheres)
    return sc, box_camera(seed, 1920, 1080), dict(width=1920, height=1080, ratio=ratio, atlas_log2=11)


def camera_path_frames(seed: int = 1, n_frames: int = 300):
    """The 64x64-vertex heightfield seen along a closed n_frames-camera spline path,
    1920x1080 views, ratio 1.0, 2048^2 atlas (one atlas per frame)."""
    sc = grid_scene(seed)
    cams = spline_cameras(seed, n_frames, 1920, 1080)
    return sc, cams, dict(width=1920, height=1080, ratio=1.0, atlas_log2=11)


BATCH_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080), (2560, 1440))
BATCH_ATLAS_LOG2 = (10, 11, 12)


def batch_views(seed: int = 1, n_views: int = 64, min_instances: int = 50, max_instances: int = 400):
    """n_views independent views: each an instanced heightfield floor with a seeded
    number of patches in [min_instances, max_instances], a resolution drawn from
    BATCH_RESOLUTIONS, an atlas side from BATCH_ATLAS_LOG2, ratio 1.0, and a camera
    on a hemisphere looking at the floor's centre."""
    rng = np.random.default_rng([seed, 0xBA7C4])
    views = []
    for v in range(n_views):
        n_inst = int(rng.integers(min_instances, max_instances + 1))
        W, H = BATCH_RESOLUTIONS[int(rng.integers(len(BATCH_RESOLUTIONS)))]
        log2 = BATCH_ATLAS_LOG2[int(rng.integers(len(BATCH_ATLAS_LOG2)))]
        sc = instanced_grid_scene(seed * 1009 + v, n_inst)
        M = hemisphere_camera(seed * 1009 + v, W, H, radius=10.0)
        views.append((sc, M, dict(width=W, height=H, ratio=1.0, atlas_log2=log2)))
    return views
