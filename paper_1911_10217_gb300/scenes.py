"""Seeded synthetic inputs: Cornell-boxes-in-a-room scenes and G-buffers.

This module only builds input arrays (triangles, radiance, occluder boxes,
shading points) and the grid parameters that go with them. It holds none of
the sampling or learning arithmetic; both the CUDA path and the CPU oracle
consume what it returns.

The paper's scenes ("Cornell Boxes in Salle de Bain", Section 4) are not
available, so these stand in for them: every emitter patch sits inside its
own walled cell and lights only that cell, which is the complex-occlusion
situation the method is built for (Section 4, teaser figure).

Array conventions (all float32, C-contiguous):
  tris      [N, 3, 3]  triangle vertices; emission is one-sided along the
                       winding normal (v1 - v0) x (v2 - v0)
  emission  [N, 3]     RGB radiance
  boxes     [K, 6]     axis-aligned occluders (xmin, ymin, zmin, xmax, ymax, zmax)
  pos, nrm  [3, P]     shading point positions / unit normals, SoA
  albedo    [P]        Lambertian albedo
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class GridConfig:
    table_size: int          # hash table slots H (power of two)
    cut_size: int            # M
    origin: tuple            # grid origin (3 floats)
    cell_size: float         # h
    normal_bins: int         # quantisation bins per octahedral axis
    jitter: bool
    q_init: float = 1e-3     # Q of a new cell's leaves (below the reward scale of these scenes)
    alpha: float = 0.03      # Eq. 1 learning rate
    eps: float = 0.02        # Eq. 2 floor
    threshold: float = 2.0   # split-collapse T
    split_iterations: int = 1  # split-collapse steps per cell and pass (1: the basic algorithm)
    levels: int = 1          # resolution levels (cell size * 2^l); > 1 with per-point footprints


@dataclasses.dataclass
class Scene:
    name: str
    tris: np.ndarray
    emission: np.ndarray
    boxes: np.ndarray
    pos: np.ndarray
    nrm: np.ndarray
    albedo: np.ndarray
    grid: GridConfig
    spp: int
    frames: int
    seed: int
    width: int = 0
    height: int = 0
    # dynamic lighting (blinking lights): per-light omega [rad/s], phase, mask
    blink_omega: np.ndarray | None = None
    blink_phase: np.ndarray | None = None
    blink_mask: np.ndarray | None = None
    # per-point footprint (world units) for multi-resolution grids, or None
    footprint: np.ndarray | None = None
    # inputs of one diffuse bounce from every point (path scenes), or None
    bounce: object = None

    @property
    def n_lights(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.pos.shape[1])

    def emission_at(self, frame: int, fps: float = 30.0) -> np.ndarray:
        """Radiance of every light at a frame: Le0 * (1 + 0.9 sin(w t + phi)) for
        blinking lights, Le0 for the rest (t = frame / fps seconds)."""
        if self.blink_mask is None:
            return self.emission
        t = frame / fps
        s = 1.0 + 0.9 * np.sin(self.blink_omega * t + self.blink_phase)
        scale = np.where(self.blink_mask, s, 1.0).astype(np.float32)
        return (self.emission * scale[:, None]).astype(np.float32)

    def emission_bound(self) -> np.ndarray:
        """Radiance bound over all frames (1.9 Le0 for blinking lights)."""
        if self.blink_mask is None:
            return self.emission
        scale = np.where(self.blink_mask, np.float32(1.9), np.float32(1.0)).astype(np.float32)
        return (self.emission * scale[:, None]).astype(np.float32)


def _box(lo, hi):
    return [lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]]


def _quad_patch(center, u_axis, v_axis, nu, nv, rng, jitter=0.0):
    """Triangulated nu x nv quad grid spanning center +- u_axis/2 +- v_axis/2.
    Winding makes the normal point along cross(u_axis, v_axis)."""
    center = np.asarray(center, np.float64)
    u_axis = np.asarray(u_axis, np.float64)
    v_axis = np.asarray(v_axis, np.float64)
    gu = np.linspace(-0.5, 0.5, nu + 1)
    gv = np.linspace(-0.5, 0.5, nv + 1)
    P = center + gu[:, None, None] * u_axis + gv[None, :, None] * v_axis
    if jitter > 0.0:
        du = np.linalg.norm(u_axis) / nu
        dv = np.linalg.norm(v_axis) / nv
        j = rng.uniform(-jitter, jitter, size=(nu + 1, nv + 1, 2))
        inner = np.zeros((nu + 1, nv + 1, 1))
        inner[1:-1, 1:-1] = 1.0
        P = P + inner * (j[..., :1] * du * u_axis / np.linalg.norm(u_axis)
                         + j[..., 1:] * dv * v_axis / np.linalg.norm(v_axis))
    a, b = P[:-1, :-1], P[1:, :-1]
    c, d = P[1:, 1:], P[:-1, 1:]
    t1 = np.stack([a, b, c], axis=2)            # [nu, nv, 3, 3]
    t2 = np.stack([a, c, d], axis=2)
    return np.stack([t1, t2], axis=2).reshape(-1, 3, 3)  # (i, k) quad -> two triangles


def _orthonormal(n):
    n = np.asarray(n, np.float64)
    n = n / np.linalg.norm(n)
    t = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 0.0, 1.0])
    u = np.cross(n, t)
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    return u, v


def _cone_dirs(axis, max_angle, count, rng):
    """Directions uniformly distributed in solid angle within max_angle of axis."""
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    u, v = _orthonormal(axis)
    cos_max = math.cos(max_angle)
    z = rng.uniform(cos_max, 1.0, size=count)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=count)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = (r * np.cos(phi))[:, None] * u + (r * np.sin(phi))[:, None] * v + z[:, None] * axis
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def tiny_scene(seed: int = 0, jitter: bool = False) -> Scene:
    """Unit-cube room split by full-height walls on x=0.5 and z=0.5 into four
    Cornell-style cells, one block per cell (8 boxes); a downward-facing
    0.2 x 0.2 patch of 64 triangles at y = 0.95 per cell (256 lights, RGB
    radiance U[0.5, 2]); 64 x 64 floor points (normal +y, albedo 0.7);
    8^3 grid, cut size 16, 4 samples per point, 8 learning iterations."""
    rng = np.random.default_rng(seed)
    w0, w1 = 0.495, 0.505
    boxes = [
        _box((w0, 0.0, 0.0), (w1, 1.0, 0.5)),
        _box((w0, 0.0, 0.5), (w1, 1.0, 1.0)),
        _box((0.0, 0.0, w0), (0.5, 1.0, w1)),
        _box((0.5, 0.0, w0), (1.0, 1.0, w1)),
    ]
    tris = []
    for cx in (0.25, 0.75):
        for cz in (0.25, 0.75):
            bx = cx + rng.uniform(-0.12, 0.12 - 0.15)
            bz = cz + rng.uniform(-0.12, 0.12 - 0.15)
            boxes.append(_box((bx, 0.0, bz), (bx + 0.15, 0.4, bz + 0.15)))
            # winding normal = (+x) cross (+z) = -y: the patch faces the floor
            tris.append(_quad_patch((cx, 0.95, cz), (0.2, 0, 0), (0, 0, 0.2), 8, 4, rng))
    tris = np.concatenate(tris).astype(np.float32)
    emission = rng.uniform(0.5, 2.0, size=(tris.shape[0], 3)).astype(np.float32)
    n = 64
    g = (np.arange(n) + 0.5) / n
    X, Z = np.meshgrid(g, g, indexing="xy")
    P = n * n
    pos = np.stack([X.ravel(), np.zeros(P), Z.ravel()]).astype(np.float32)
    nrm = np.stack([np.zeros(P), np.ones(P), np.zeros(P)]).astype(np.float32)
    albedo = np.full(P, 0.7, np.float32)
    grid = GridConfig(table_size=1024, cut_size=16, origin=(0.0, 0.0, 0.0),
                      cell_size=0.125, normal_bins=1, jitter=jitter)
    return Scene("tiny", tris, emission, np.asarray(boxes, np.float32), pos, nrm, albedo,
                 grid, spp=4, frames=8, seed=seed, width=n, height=n)


def _room_cells(rng, cells_per_side, n_boxes, wall_t=0.006):
    """Full-height walls on the interior cell boundaries of a unit room, split
    into one segment per cell edge, plus random blocks up to n_boxes."""
    c = cells_per_side
    pitch = 1.0 / c
    boxes = []
    for i in range(1, c):
        x = i * pitch
        for j in range(c):
            boxes.append(_box((x - wall_t, 0.0, j * pitch), (x + wall_t, 1.0, (j + 1) * pitch)))
            boxes.append(_box((j * pitch, 0.0, x - wall_t), ((j + 1) * pitch, 1.0, x + wall_t)))
    k = 0
    while len(boxes) < n_boxes:
        ci, cj = k % c, (k // c) % c
        k += 1
        sx, sy, sz = rng.uniform(0.08, 0.2) * pitch * 2, rng.uniform(0.05, 0.35), rng.uniform(0.08, 0.2) * pitch * 2
        x0 = ci * pitch + rng.uniform(0.1 * pitch, max(0.1 * pitch, 0.9 * pitch - sx))
        z0 = cj * pitch + rng.uniform(0.1 * pitch, max(0.1 * pitch, 0.9 * pitch - sz))
        boxes.append(_box((x0, 0.0, z0), (x0 + sx, sy, z0 + sz)))
    return np.asarray(boxes[:n_boxes], np.float32)


def _emitter_patches(rng, cells_per_side, n_patches, tris_per_patch):
    """Clustered mesh emitters: each patch a jittered triangulated quad in the
    upper part of one cell, facing down into the room within 40 degrees."""
    c = cells_per_side
    pitch = 1.0 / c
    nq = tris_per_patch // 2
    nu = int(2 ** math.floor(math.log2(math.sqrt(nq))))
    nv = nq // nu
    patches = []
    for p in range(n_patches):
        ci, cj = p % c, (p // c) % c
        center = (ci * pitch + rng.uniform(0.2, 0.8) * pitch,
                  rng.uniform(0.6, 0.95),
                  cj * pitch + rng.uniform(0.2, 0.8) * pitch)
        normal = _cone_dirs((0.0, -1.0, 0.0), math.radians(40.0), 1, rng)[0]
        u, v = _orthonormal(normal)
        size = rng.uniform(0.15, 0.3) * pitch
        # winding normal = cross(u_axis, v_axis); _orthonormal gives v = n x u,
        # so cross(u, v) = n and the patch faces along `normal`.
        patches.append(_quad_patch(center, u * size, v * size, nu, nv, rng, jitter=0.25))
    return np.concatenate(patches).astype(np.float32)


def _gbuffer_planes(rng, width, height, cells_per_side, n_planes=16, normal_jitter_deg=15.0):
    """width x height shading points on n_planes random plane patches (one
    rectangular block of pixels per plane), normals jittered within
    normal_jitter_deg of the plane normal, albedo U[0.2, 0.9]."""
    c = cells_per_side
    pitch = 1.0 / c
    gx = int(round(math.sqrt(n_planes)))
    gy = n_planes // gx
    bw, bh = width // gx, height // gy
    pos = np.zeros((3, height, width), np.float32)
    nrm = np.zeros((3, height, width), np.float32)
    ys, xs = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    for k in range(n_planes):
        px, py = k % gx, k // gx
        x0, x1 = px * bw, (px + 1) * bw if px < gx - 1 else width
        y0, y1 = py * bh, (py + 1) * bh if py < gy - 1 else height
        ci, cj = k % c, (k // c) % c
        normal = _cone_dirs((0.0, 1.0, 0.0), math.radians(30.0), 1, rng)[0]
        u, v = _orthonormal(normal)
        ext = 0.7 * pitch
        center = np.array([(ci + 0.5) * pitch, rng.uniform(0.0, 0.25), (cj + 0.5) * pitch])
        su = (xs[y0:y1, x0:x1] - x0 + 0.5) / (x1 - x0) - 0.5
        sv = (ys[y0:y1, x0:x1] - y0 + 0.5) / (y1 - y0) - 0.5
        P = center[:, None, None] + ext * (su[None] * u[:, None, None] + sv[None] * v[:, None, None])
        pos[:, y0:y1, x0:x1] = P
        npx = (x1 - x0) * (y1 - y0)
        dirs = _cone_dirs(normal, math.radians(normal_jitter_deg), npx, rng)
        nrm[:, y0:y1, x0:x1] = dirs.T.reshape(3, y1 - y0, x1 - x0)
    albedo = rng.uniform(0.2, 0.9, size=width * height).astype(np.float32)
    return pos.reshape(3, -1).copy(), nrm.reshape(3, -1).copy(), albedo


def frame_scene(seed: int = 1, width: int = 1920, height: int = 1080, n_patches: int = 64,
                tris_per_patch: int = 1024, n_boxes: int = 64, table_size: int = 1 << 20,
                cut_size: int = 32, frames: int = 32) -> Scene:
    """Frame-scale static scene: 64K emissive triangles in 64 clustered patches,
    64 occluder boxes forming 16 walled cells, a 1920 x 1080 G-buffer on 16
    random planes (normals jittered +-15 deg, albedo U[0.2, 0.9]); 2^20-entry
    hash grid, cut size 32, 1 sample per point per frame. The cell size
    scales with the resolution so that a cell keeps the same pixel count."""
    rng = np.random.default_rng(seed)
    c = 4
    boxes = _room_cells(rng, c, n_boxes)
    tris = _emitter_patches(rng, c, n_patches, tris_per_patch)
    emission = rng.uniform(0.5, 2.0, size=(tris.shape[0], 3)).astype(np.float32)
    pos, nrm, albedo = _gbuffer_planes(rng, width, height, c)
    # cells of ~43 x 43 pixels on the planes: ~100 samples per cell per frame
    grid = GridConfig(table_size=table_size, cut_size=cut_size, origin=(0.0, 0.0, 0.0),
                      cell_size=1.0 / 64.0 * (1920.0 / width), normal_bins=2, jitter=True)
    return Scene("frame", tris, emission, boxes, pos, nrm, albedo, grid, spp=1,
                 frames=frames, seed=seed, width=width, height=height)


def dynamic_scene(seed: int = 2, width: int = 3840, height: int = 2160, n_patches: int = 1024,
                  tris_per_patch: int = 1024, n_boxes: int = 64, table_size: int = 1 << 21,
                  cut_size: int = 64, frames: int = 120, blink_fraction: float = 0.1) -> Scene:
    """Dynamic lighting: 1M emissive triangles (1024 patches), 10% blinking as
    1 + 0.9 sin(w t + phi), w ~ U[0.5, 4] rad/s, phi ~ U[0, 2 pi); 3840 x 2160
    G-buffer; cut size 64; 2^21-entry grid; 120 frames."""
    rng = np.random.default_rng(seed)
    c = 4
    boxes = _room_cells(rng, c, n_boxes)
    tris = _emitter_patches(rng, c, n_patches, tris_per_patch)
    n = tris.shape[0]
    emission = rng.uniform(0.5, 2.0, size=(n, 3)).astype(np.float32)
    mask = rng.uniform(size=n) < blink_fraction
    omega = rng.uniform(0.5, 4.0, size=n).astype(np.float32)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n).astype(np.float32)
    pos, nrm, albedo = _gbuffer_planes(rng, width, height, c)
    grid = GridConfig(table_size=table_size, cut_size=cut_size, origin=(0.0, 0.0, 0.0),
                      cell_size=1.0 / 64.0 * (1920.0 / width), normal_bins=2, jitter=True)
    return Scene("dynamic", tris, emission, boxes, pos, nrm, albedo, grid, spp=1,
                 frames=frames, seed=seed, width=width, height=height,
                 blink_omega=omega, blink_phase=phase, blink_mask=mask)


def small_frame_scene(seed: int = 3, width: int = 96, height: int = 64, n_patches: int = 16,
                      tris_per_patch: int = 64, n_boxes: int = 32, table_size: int = 1 << 14,
                      cut_size: int = 32, spp: int = 2) -> Scene:
    """A reduced frame-scale scene (same recipe as frame_scene) small enough
    for the CPU oracle to finish every sample in about a second."""
    s = frame_scene(seed=seed, width=width, height=height, n_patches=n_patches,
                    tris_per_patch=tris_per_patch, n_boxes=n_boxes, table_size=table_size,
                    cut_size=cut_size, frames=4)
    s.name = "small_frame"
    s.spp = spp
    return s


def batched_scenes(seed: int = 4, n_scenes: int = 256, light_range=(1 << 10, 1 << 18),
                   point_range=(1 << 16, 1 << 21), cut_sizes=(16, 32, 64), scale: float = 1.0):
    """Uneven independent scenes: light counts and shading-point counts
    log-uniform over the given ranges, cut size uniform over cut_sizes.
    `scale` shrinks the point and light counts (for tests)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        nl = int(math.exp(rng.uniform(math.log(light_range[0]), math.log(light_range[1]))) * scale)
        npnt = int(math.exp(rng.uniform(math.log(point_range[0]), math.log(point_range[1]))) * scale)
        nl = max(nl, 16)
        npnt = max(npnt, 64)
        m = int(rng.choice(cut_sizes))
        n_patches = max(1, int(round(nl / 256)))
        tpp = max(2, (nl // n_patches) // 2 * 2)
        width = int(math.sqrt(npnt * 16 / 9)) // 4 * 4 or 4
        height = max(4, npnt // width // 4 * 4)
        table = 1 << max(10, int(math.ceil(math.log2(max(1, width * height) / 16))))
        s = frame_scene(seed=seed * 100003 + i, width=width, height=height, n_patches=n_patches,
                        tris_per_patch=tpp, n_boxes=32, table_size=table, cut_size=m, frames=1)
        s.name = f"batched{i}"
        out.append(s)
    return out


def _wall_boxes(axis, side, openings, t=0.02):
    """Boxes of one wall of the unit room with rectangular openings.

    axis: 0 -> wall plane x = side (u = z), 2 -> z = side (u = x),
    1 -> ceiling y = 1 (u = x, v = z). The wall lies outside the room
    (thickness t). openings: list of (u0, u1, v0, v1) in the wall's (u, v)
    coordinates (v = y for side walls), all in one band v0..v1 per row of
    openings; rows are given as separate lists of openings sharing v0, v1."""
    boxes = []

    def put(u0, u1, v0, v1):
        if u1 <= u0 or v1 <= v0:
            return
        if axis == 1:
            boxes.append(_box((u0, 1.0, v0), (u1, 1.0 + t, v1)))
        elif axis == 0:
            x0 = side - t if side <= 0.0 else side
            boxes.append(_box((x0, v0, u0), (x0 + t, v1, u1)))
        else:
            z0 = side - t if side <= 0.0 else side
            boxes.append(_box((u0, v0, z0), (u1, v1, z0 + t)))

    lo_u, hi_u = -t, 1.0 + t
    v_prev = 0.0 if axis != 1 else -t
    for row in openings:
        v0, v1 = row[0][2], row[0][3]
        put(lo_u, hi_u, v_prev, v0)             # solid band below the row
        u_prev = lo_u
        for (u0, u1, _, _) in sorted(row):
            put(u_prev, u0, v0, v1)             # pier between openings
            u_prev = u1
        put(u_prev, hi_u, v0, v1)
        v_prev = v1
    put(lo_u, hi_u, v_prev, 1.0 if axis != 1 else 1.0 + t)  # solid band above
    return boxes


def _sky_dome(center, radius, rings, segments, max_elev_deg=88.0):
    """Hemisphere of rings x segments quads (2 triangles each) from the horizon
    up to max_elev_deg, wound so that every normal points to the centre."""
    el = np.radians(np.linspace(0.0, max_elev_deg, rings + 1))
    az = np.linspace(0.0, 2.0 * math.pi, segments + 1)
    E, A = np.meshgrid(el, az, indexing="ij")
    P = np.stack([np.cos(E) * np.cos(A), np.sin(E), np.cos(E) * np.sin(A)], axis=-1) * radius
    P = P + np.asarray(center, np.float64)
    a, b = P[:-1, :-1], P[1:, :-1]
    c, d = P[1:, 1:], P[:-1, 1:]
    # (b - a) x (d - a) points outward for increasing elevation / azimuth;
    # the order (a, d, b) flips it inward
    t1 = np.stack([a, d, b], axis=2)
    t2 = np.stack([b, d, c], axis=2)
    return np.stack([t1, t2], axis=2).reshape(-1, 3, 3)


def sky_scene(seed: int = 5, width: int = 1920, height: int = 1080, rings: int = 32, segments: int = 32,
              table_size: int = 1 << 15, cut_size: int = 32, cell_size: float = 1.0 / 64.0, spp: int = 1,
              frames: int = 64, windows_per_wall: int = 4, sun: bool = False) -> Scene:
    """Interior lit only through small openings (the situation of the paper's
    "Arch interior" scene, Section 4, where a uniform sky is the only light):
    a closed unit room whose four walls each have a row of windows_per_wall
    small windows and whose ceiling has two skylights, a few blocks inside;
    outside, a sky dome of 2 * rings * segments inward-facing triangles with
    uniform radiance. With sun=True a small, very bright, distant quad (two
    triangles) stands in for a directional light. Shading points: a
    width x height grid over the floor (normal +y, albedo U[0.2, 0.9]).
    Cells of cell_size, one normal bin."""
    rng = np.random.default_rng(seed)
    boxes = []
    k = windows_per_wall
    for axis, side in ((0, 0.0), (0, 1.0), (2, 0.0), (2, 1.0)):
        sill = rng.uniform(0.35, 0.5)
        row = []
        for i in range(k):
            cu = (i + 0.5) / k + rng.uniform(-0.05, 0.05) / k
            w = rng.uniform(0.05, 0.09)
            row.append((cu - w / 2, cu + w / 2, sill, sill + rng.uniform(0.1, 0.16)))
        v0, v1 = min(r[2] for r in row), max(r[3] for r in row)
        row = [(u0, u1, v0, v1) for (u0, u1, _, _) in row]
        boxes += _wall_boxes(axis, side, [row])
    sky_row = [(0.25, 0.37, 0.3, 0.42), (0.6, 0.72, 0.3, 0.42)]
    boxes += _wall_boxes(1, 1.0, [sky_row])
    for _ in range(6):  # blocks inside the room
        sx, sy, sz = rng.uniform(0.06, 0.16), rng.uniform(0.15, 0.5), rng.uniform(0.06, 0.16)
        x0, z0 = rng.uniform(0.1, 0.9 - sx), rng.uniform(0.1, 0.9 - sz)
        boxes.append(_box((x0, 0.0, z0), (x0 + sx, sy, z0 + sz)))
    center = np.array([0.5, 0.0, 0.5])
    dome = _sky_dome(center, 20.0, rings, segments)
    sky_le = np.array([0.5, 0.65, 1.0])
    # "sun": a 0.6 x 0.6 quad at distance 18, elevation 50 deg, facing the room
    el, az = math.radians(50.0), math.radians(30.0)
    d = np.array([math.cos(el) * math.cos(az), math.sin(el), math.cos(el) * math.sin(az)])
    u, v = _orthonormal(-d)
    sun_tris = _quad_patch(center + 18.0 * d, u * 0.6, v * 0.6, 1, 1, rng)
    sun_le = np.array([2000.0, 1800.0, 1500.0])
    if not sun:
        sun_tris = sun_tris[:0]
    tris = np.concatenate([dome, sun_tris]).astype(np.float32)
    emission = np.concatenate([np.tile(sky_le, (dome.shape[0], 1)),
                               np.tile(sun_le, (sun_tris.shape[0], 1))]).astype(np.float32)
    gx = (np.arange(width) + 0.5) / width
    gz = (np.arange(height) + 0.5) / height
    X, Z = np.meshgrid(gx, gz, indexing="xy")
    P = width * height
    pos = np.stack([X.ravel(), np.zeros(P), Z.ravel()]).astype(np.float32)
    nrm = np.stack([np.zeros(P), np.ones(P), np.zeros(P)]).astype(np.float32)
    albedo = rng.uniform(0.2, 0.9, size=P).astype(np.float32)
    grid = GridConfig(table_size=table_size, cut_size=cut_size, origin=(0.0, 0.0, 0.0),
                      cell_size=cell_size, normal_bins=1, jitter=True)
    return Scene("sky", tris, emission, np.asarray(boxes, np.float32), pos, nrm, albedo, grid, spp=spp,
                 frames=frames, seed=seed, width=width, height=height)


def tiny_sky_scene(seed: int = 6, jitter: bool = False, sun: bool = True) -> Scene:
    """The sky scene small enough for the oracle: 64 x 64 floor points, a
    dome of 8 x 8 quads (128 triangles) plus (by default) the 2-triangle sun,
    cells of 1/8, cut size 16, 4 samples per point, 8 learning passes."""
    s = sky_scene(seed=seed, width=64, height=64, rings=8, segments=8, table_size=1024, cut_size=16,
                  cell_size=0.125, spp=4, frames=8, sun=sun)
    s.name = "tiny_sky"
    s.grid.jitter = jitter
    return s


# Path vertices: the bounce vertices themselves (one cosine-weighted diffuse
# bounce per shading point, its nearest surface, its footprint from the area
# pdf) are computed by the method -- the CUDA library's rll_bounce_vertices,
# or the oracle in tests. This generator only supplies the primary points and
# the bounce's inputs.
ROOM = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0], np.float32)  # the walled rooms' enclosure, min xyz, max xyz


@dataclasses.dataclass
class BounceSpec:
    """Inputs of one bounce from every primary point: the Philox key and
    frame of its directions, the paths N_t leaving one tile, the room it
    stays in, and the albedo of the surface each vertex lands on."""
    seed: int
    frame: int
    paths_per_tile: float
    room: np.ndarray
    albedo: np.ndarray


def path_scene(base: Scene, seed: int = 7, levels: int = 8, paths_per_tile: float = 100.0) -> Scene:
    """Primary points of `base` (footprint = the cell size, the finest level)
    with the inputs of one diffuse bounce each (scene.bounce); the grid gets
    `levels` resolution levels. The bounce vertices are appended by
    with_bounce_vertices once they are computed."""
    rng = np.random.default_rng(seed)
    s = dataclasses.replace(base)
    s.name = base.name + "_paths"
    s.footprint = np.full(base.n_points, np.float32(base.grid.cell_size), np.float32)
    s.grid = dataclasses.replace(base.grid, levels=levels)
    s.bounce = BounceSpec(seed=seed, frame=0, paths_per_tile=float(paths_per_tile), room=ROOM.copy(),
                          albedo=rng.uniform(0.2, 0.9, size=base.n_points).astype(np.float32))
    return s


def with_bounce_vertices(s: Scene, pos: np.ndarray, nrm: np.ndarray, footprint: np.ndarray) -> Scene:
    """The path scene's points followed by its bounce vertices (SoA [3][P]
    positions and normals, footprints [P])."""
    out = dataclasses.replace(s)
    out.pos = np.concatenate([s.pos, np.asarray(pos, np.float32)], axis=1)
    out.nrm = np.concatenate([s.nrm, np.asarray(nrm, np.float32)], axis=1)
    out.albedo = np.concatenate([s.albedo, s.bounce.albedo])
    out.footprint = np.concatenate([s.footprint, np.asarray(footprint, np.float32)])
    return out
