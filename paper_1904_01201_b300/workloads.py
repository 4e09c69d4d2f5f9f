"""Seeded synthetic workloads: procedural indoor scenes, agent poses, random walks.

This module holds scene *inputs* only (geometry, texture atlases, semantic tables,
camera poses). It contains none of the rendering arithmetic, so the CUDA path and
the CPU oracle can both consume its output without sharing any method code.

Every random number comes from a counter-based splitmix64 stream keyed by
(seed, stream name), so one seed gives byte-identical arrays on any machine
(apart from the libm sin/cos used for pose yaw and cylinder rims).

Scene recipes stand in for the Matterport3D / Gibson scans the paper renders
(Sec. 3 "Performance", Table 1, Table 2): multi-room houses with extruded walls,
floors, ceilings, door openings and box / cylinder furniture, subdivided to a
target triangle count, with planar UV charts packed into one RGBA8 atlas.
Agent conventions follow Sec. 4 "Agent embodiment" and "Sensory input": camera
1.5 m above the floor, 90 degree horizontal field of view, body radius 0.1 m,
actions move_forward 0.25 m and turn 10 degrees.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ----------------------------------------------------------------------------
# counter-based random numbers
# ----------------------------------------------------------------------------
_M64 = (1 << 64) - 1
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, name: str) -> int:
    h = seed & _M64
    for ch in name.encode():
        h = int(_mix64(np.array([(h ^ ch) & _M64], dtype=np.uint64))[0])
    return h


class Stream:
    """splitmix64 evaluated at counters key + i*gamma (i = 1, 2, ...)."""

    def __init__(self, seed: int, name: str):
        self.key = np.uint64(_key(seed, name))
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            ctr = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
            out = _mix64(self.key + ctr * _GAMMA)
        self.pos += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi)."""
        return lo + (self.u64(n) % np.uint64(hi - lo)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# scene container
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    """A static triangle mesh in the C-ABI layout (world is Y-up, metres).

    Front faces are counter-clockwise seen from the side their normal points to.
    """

    xyz: np.ndarray                      # [V,3] float32
    idx: np.ndarray                      # [T,3] uint32
    uv: Optional[np.ndarray] = None      # [V,2] float32
    vrgb: Optional[np.ndarray] = None    # [V,3] uint8
    atlas: Optional[np.ndarray] = None   # [Ht,Wt,4] uint8, row 0 is v = 0
    sem: Optional[np.ndarray] = None     # [T] uint32
    # free space for agent placement: rooms (x0, z0, x1, z1) and obstacle footprints
    rooms: List[Tuple[float, float, float, float]] = dataclasses.field(default_factory=list)
    boxes: List[Tuple[float, float, float, float]] = dataclasses.field(default_factory=list)
    circles: List[Tuple[float, float, float]] = dataclasses.field(default_factory=list)
    name: str = ""

    @property
    def n_tris(self) -> int:
        return int(self.idx.shape[0])

    @property
    def n_verts(self) -> int:
        return int(self.xyz.shape[0])

    def nbytes(self) -> int:
        n = self.xyz.nbytes + self.idx.nbytes
        for a in (self.uv, self.vrgb, self.atlas, self.sem):
            if a is not None:
                n += a.nbytes
        return n


@dataclasses.dataclass
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float = 0.01
    zfar: float = 10.0

    def as_array(self) -> np.ndarray:
        return np.array([self.fx, self.fy, self.cx, self.cy, self.znear, self.zfar], dtype=np.float32)


def pinhole_90(width: int, height: int, znear: float = 0.01, zfar: float = 10.0) -> Intrinsics:
    """90 degree horizontal field of view, square pixels (Sec. 4 "Sensory input")."""
    f = width / 2.0
    return Intrinsics(f, f, width / 2.0, height / 2.0, znear, zfar)


# ----------------------------------------------------------------------------
# mesh builder
# ----------------------------------------------------------------------------
class _Builder:
    def __init__(self):
        self.xyz: List[np.ndarray] = []
        self.tri: List[np.ndarray] = []
        self.local_st: List[np.ndarray] = []    # per-vertex chart coordinates (m)
        self.chart_of_vert: List[np.ndarray] = []
        self.chart_size: List[Tuple[float, float]] = []
        self.obj_of_tri: List[np.ndarray] = []
        self.nv = 0
        self.n_obj = 0

    def new_object(self) -> int:
        self.n_obj += 1
        return self.n_obj - 1

    def add(self, xyz, tri, st, chart_wh, normal, obj):
        xyz = np.asarray(xyz, dtype=np.float64)
        tri = np.asarray(tri, dtype=np.int64)
        # orient every triangle so that its normal agrees with the face normal
        a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
        n = np.cross(b - a, c - a)
        flip = (n @ np.asarray(normal, dtype=np.float64)) < 0
        tri = tri.copy()
        tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
        chart = len(self.chart_size)
        self.chart_size.append(chart_wh)
        self.xyz.append(xyz)
        self.tri.append(tri + self.nv)
        self.local_st.append(np.asarray(st, dtype=np.float64))
        self.chart_of_vert.append(np.full(len(xyz), chart, dtype=np.int64))
        self.obj_of_tri.append(np.full(len(tri), obj, dtype=np.int64))
        self.nv += len(xyz)

    def quad(self, o, a, b, s, normal, obj):
        """Rectangle o + [0,1]a + [0,1]b subdivided into cells of about s metres."""
        o, a, b = (np.asarray(v, dtype=np.float64) for v in (o, a, b))
        la, lb = float(np.linalg.norm(a)), float(np.linalg.norm(b))
        n = max(1, int(round(la / s)))
        m = max(1, int(round(lb / s)))
        i, j = np.meshgrid(np.arange(n + 1), np.arange(m + 1), indexing="xy")
        fi = (i / n).reshape(-1, 1)
        fj = (j / m).reshape(-1, 1)
        xyz = o + fi * a + fj * b
        st = np.concatenate([fi * la, fj * lb], axis=1)
        ci, cj = np.meshgrid(np.arange(n), np.arange(m), indexing="xy")
        v00 = (cj * (n + 1) + ci).reshape(-1)
        v10 = v00 + 1
        v01 = v00 + (n + 1)
        v11 = v01 + 1
        tri = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
        self.add(xyz, tri, st, (la, lb), normal, obj)

    def cylinder(self, cx, cz, r, h, k, s, obj):
        perim_seg = 2.0 * r * math.sin(math.pi / k)
        c = max(1, int(round(perim_seg / s)))
        m = max(1, int(round(h / s)))
        cols = k * c
        ang = 2.0 * math.pi * np.arange(k + 1) / k
        corners = np.stack([cx + r * np.cos(ang), cz + r * np.sin(ang)], 1)
        # side: polygon perimeter subdivided; seam column duplicated for the UV chart
        t = np.arange(cols + 1)
        e = np.minimum(t // c, k - 1)
        f = (t - e * c) / c
        f[-1] = 1.0
        px = corners[e, 0] + f * (corners[e + 1, 0] - corners[e, 0])
        pz = corners[e, 1] + f * (corners[e + 1, 1] - corners[e, 1])
        px[-1], pz[-1] = corners[0, 0], corners[0, 1]
        jj = np.arange(m + 1) / m
        X = np.repeat(px[None, :], m + 1, 0).reshape(-1)
        Z = np.repeat(pz[None, :], m + 1, 0).reshape(-1)
        Y = np.repeat(jj[:, None] * h, cols + 1, 1).reshape(-1)
        xyz = np.stack([X, Y, Z], 1)
        s_arc = (t * perim_seg / c)
        st = np.stack([np.repeat(s_arc[None, :], m + 1, 0).reshape(-1), Y], 1)
        ci, cj = np.meshgrid(np.arange(cols), np.arange(m), indexing="xy")
        v00 = (cj * (cols + 1) + ci).reshape(-1)
        v10, v01 = v00 + 1, v00 + cols + 1
        v11 = v01 + 1
        tri = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
        # outward normals differ per column: orient each quad individually
        centre = np.array([cx, 0.0, cz])
        self._add_radial(xyz, tri, st, (k * perim_seg, h), centre, obj)
        # top cap: k-gon subdivided into L rings, shared vertices
        L = max(1, int(round(r / s)))
        verts = [np.array([cx, h, cz])]
        ring_base = [0]
        for j in range(1, L + 1):
            ring_base.append(len(verts))
            for e_ in range(k):
                for tt in range(j):
                    fr = tt / j
                    p = corners[e_] + fr * (corners[e_ + 1] - corners[e_])
                    q = np.array([cx, cz]) + (j / L) * (p - np.array([cx, cz]))
                    verts.append(np.array([q[0], h, q[1]]))
        cap = np.array(verts)

        def vid(j, p):
            if j == 0:
                return 0
            return ring_base[j] + (p % (k * j))

        tris = []
        for j in range(1, L + 1):
            for e_ in range(k):
                for tt in range(j):
                    tris.append((vid(j, e_ * j + tt), vid(j, e_ * j + tt + 1), vid(j - 1, e_ * (j - 1) + tt)))
                for tt in range(j - 1):
                    tris.append((vid(j - 1, e_ * (j - 1) + tt), vid(j, e_ * j + tt + 1), vid(j - 1, e_ * (j - 1) + tt + 1)))
        st_cap = np.stack([cap[:, 0] - (cx - r), cap[:, 2] - (cz - r)], 1)
        self.add(cap, np.array(tris), st_cap, (2 * r, 2 * r), (0.0, 1.0, 0.0), obj)

    def _add_radial(self, xyz, tri, st, chart_wh, centre, obj):
        a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
        n = np.cross(b - a, c - a)
        out = (a + b + c) / 3.0 - centre
        out[:, 1] = 0.0
        flip = np.einsum("ij,ij->i", n, out) < 0
        tri = tri.copy()
        tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
        chart = len(self.chart_size)
        self.chart_size.append(chart_wh)
        self.xyz.append(xyz)
        self.tri.append(tri + self.nv)
        self.local_st.append(np.asarray(st, dtype=np.float64))
        self.chart_of_vert.append(np.full(len(xyz), chart, dtype=np.int64))
        self.obj_of_tri.append(np.full(len(tri), obj, dtype=np.int64))
        self.nv += len(xyz)

    def arrays(self):
        xyz = np.concatenate(self.xyz, 0)
        tri = np.concatenate(self.tri, 0)
        st = np.concatenate(self.local_st, 0)
        chart = np.concatenate(self.chart_of_vert, 0)
        obj = np.concatenate(self.obj_of_tri, 0)
        return xyz, tri, st, chart, obj


# ----------------------------------------------------------------------------
# layout primitives (a recipe is a list of surfaces; subdivision comes later)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class _Layout:
    quads: list          # (o, a, b, normal, obj)
    cylinders: list      # (cx, cz, r, h, k, obj)
    n_obj: int
    rooms: list
    boxes: list
    circles: list

    def area(self) -> float:
        tot = 0.0
        for o, a, b, _, _ in self.quads:
            tot += float(np.linalg.norm(a) * np.linalg.norm(b))
        for cx, cz, r, h, k, _ in self.cylinders:
            tot += 2 * math.pi * r * h + math.pi * r * r
        return tot


def _box_faces(quads, x0, z0, x1, z1, y0, y1, obj, outward=True, skip_bottom=True):
    """Axis-aligned box; outward normals for objects, inward for rooms."""
    sgn = 1.0 if outward else -1.0
    dx, dy, dz = x1 - x0, y1 - y0, z1 - z0
    # +X face
    quads.append(((x1, y0, z1), (0, 0, -dz), (0, dy, 0), (sgn, 0, 0), obj))
    quads.append(((x0, y0, z0), (0, 0, dz), (0, dy, 0), (-sgn, 0, 0), obj))
    quads.append(((x0, y0, z1), (dx, 0, 0), (0, dy, 0), (0, 0, sgn), obj))
    quads.append(((x1, y0, z0), (-dx, 0, 0), (0, dy, 0), (0, 0, -sgn), obj))
    quads.append(((x0, y1, z0), (dx, 0, 0), (0, 0, dz), (0, sgn, 0), obj))
    if not skip_bottom:
        quads.append(((x0, y0, z0), (dx, 0, 0), (0, 0, dz), (0, -sgn, 0), obj))


def _layout_room(seed: int) -> _Layout:
    """5 x 4 x 3 m box room with 20 axis-aligned box furniture pieces."""
    rs = Stream(seed, "room")
    quads: list = []
    W, D, Hh = 5.0, 4.0, 3.0
    obj = 0
    # floor (+Y), ceiling (-Y), four inward walls
    quads.append(((0, 0, D), (W, 0, 0), (0, 0, -D), (0, 1, 0), obj))
    quads.append(((0, Hh, 0), (W, 0, 0), (0, 0, D), (0, -1, 0), obj))
    quads.append(((0, 0, 0), (0, 0, D), (0, Hh, 0), (1, 0, 0), obj))
    quads.append(((W, 0, D), (0, 0, -D), (0, Hh, 0), (-1, 0, 0), obj))
    quads.append(((W, 0, 0), (-W, 0, 0), (0, Hh, 0), (0, 0, 1), obj))
    quads.append(((0, 0, D), (W, 0, 0), (0, Hh, 0), (0, 0, -1), obj))
    boxes = []
    for i in range(20):
        sx, sy, sz = rs.uniform(3, 0.3, 1.5)
        x0 = float(rs.uniform(1, 0.0, W - sx)[0])
        z0 = float(rs.uniform(1, 0.0, D - sz)[0])
        _box_faces(quads, x0, z0, x0 + sx, z0 + sz, 0.0, float(sy), obj=i + 1)
        boxes.append((x0, z0, x0 + float(sx), z0 + float(sz)))
    return _Layout(quads, [], 21, [(0.0, 0.0, W, D)], boxes, [])


def _split_rooms(rs: Stream, w: float, d: float, n_rooms: int):
    rects = [(0.0, 0.0, w, d)]
    while len(rects) < n_rooms:
        areas = [(r[2] - r[0]) * (r[3] - r[1]) for r in rects]
        i = int(np.argmax(areas))
        x0, z0, x1, z1 = rects.pop(i)
        f = float(rs.uniform(1, 0.35, 0.65)[0])
        if (x1 - x0) >= (z1 - z0):
            xm = x0 + f * (x1 - x0)
            rects += [(x0, z0, xm, z1), (xm, z0, x1, z1)]
        else:
            zm = z0 + f * (z1 - z0)
            rects += [(x0, z0, x1, zm), (x0, zm, x1, z1)]
    return rects


def _layout_house(seed: int, n_objects: int = 300) -> _Layout:
    """Multi-room floorplan (8-12 rooms) by recursive splits, extruded walls with
    door openings, floors, ceilings, and random boxes and cylinders."""
    rs = Stream(seed, "house")
    n_rooms = int(rs.integers(1, 8, 13)[0])
    area = n_rooms * float(rs.uniform(1, 14.0, 22.0)[0])
    aspect = float(rs.uniform(1, 0.75, 1.33)[0])
    w = math.sqrt(area * aspect)
    d = area / w
    Hh = float(rs.uniform(1, 2.5, 3.0)[0])
    t = 0.05                      # half wall thickness
    door_w, door_h = 0.9, 2.1
    rects = _split_rooms(rs, w, d, n_rooms)
    quads: list = []
    # door positions on shared walls, one per adjacent pair
    doors = {}                    # (axis, coord) -> list of (g0, g1)
    for i in range(len(rects)):
        for j in range(i + 1, len(rects)):
            a, b = rects[i], rects[j]
            walls = []
            # axis 0: wall on x = const, spanning z; axis 1: wall on z = const, spanning x
            for line in {a[2], a[0]} & {b[0], b[2]}:
                if (line == a[2] and line == b[0]) or (line == a[0] and line == b[2]):
                    walls.append((0, line, max(a[1], b[1]), min(a[3], b[3])))
            for line in {a[3], a[1]} & {b[1], b[3]}:
                if (line == a[3] and line == b[1]) or (line == a[1] and line == b[3]):
                    walls.append((1, line, max(a[0], b[0]), min(a[2], b[2])))
            for axis, line, s0, s1 in walls:
                if s1 - s0 < door_w + 2 * t + 0.3:
                    continue
                g0 = float(rs.uniform(1, s0 + t + 0.15, s1 - t - 0.15 - door_w)[0])
                doors.setdefault((axis, round(line, 9)), []).append((g0, g0 + door_w))
    obj = 0
    rooms_free = []
    for (x0, z0, x1, z1) in rects:
        ix0, iz0, ix1, iz1 = x0 + t, z0 + t, x1 - t, z1 - t
        rooms_free.append((ix0, iz0, ix1, iz1))
        dx, dz = ix1 - ix0, iz1 - iz0
        quads.append(((ix0, 0, iz1), (dx, 0, 0), (0, 0, -dz), (0, 1, 0), obj))
        quads.append(((ix0, Hh, iz0), (dx, 0, 0), (0, 0, dz), (0, -1, 0), obj))
        walls = [
            # (fixed axis, fixed coord, along-axis interval, inward normal)
            (0, x0, ix0, (iz0, iz1), (1, 0, 0)),
            (0, x1, ix1, (iz0, iz1), (-1, 0, 0)),
            (1, z0, iz0, (ix0, ix1), (0, 0, 1)),
            (1, z1, iz1, (ix0, ix1), (0, 0, -1)),
        ]
        for axis, line, pos, (p0, p1), nrm in walls:
            gaps = sorted(g for g in doors.get((axis, round(line, 9)), []) if g[0] >= p0 - 1e-9 and g[1] <= p1 + 1e-9)
            segs, cur = [], p0
            for g0, g1 in gaps:
                segs.append((cur, g0, 0.0, Hh))
                segs.append((g0, g1, door_h, Hh))
                cur = g1
            segs.append((cur, p1, 0.0, Hh))
            for (a0, a1, y0, y1) in segs:
                if a1 - a0 < 1e-6:
                    continue
                if axis == 0:
                    quads.append(((pos, y0, a0), (0, 0, a1 - a0), (0, y1 - y0, 0), nrm, obj))
                else:
                    quads.append(((a0, y0, pos), (a1 - a0, 0, 0), (0, y1 - y0, 0), nrm, obj))
            # door jambs and lintel underside, facing into the opening
            for g0, g1 in gaps:
                if axis == 0:
                    quads.append(((line, 0, g0), (pos - line, 0, 0), (0, door_h, 0), (0, 0, 1), obj))
                    quads.append(((line, 0, g1), (pos - line, 0, 0), (0, door_h, 0), (0, 0, -1), obj))
                    quads.append(((line, door_h, g0), (pos - line, 0, 0), (0, 0, g1 - g0), (0, -1, 0), obj))
                    quads.append(((line, 0, g0), (pos - line, 0, 0), (0, 0, g1 - g0), (0, 1, 0), obj))
                else:
                    quads.append(((g0, 0, line), (0, 0, pos - line), (0, door_h, 0), (1, 0, 0), obj))
                    quads.append(((g1, 0, line), (0, 0, pos - line), (0, door_h, 0), (-1, 0, 0), obj))
                    quads.append(((g0, door_h, line), (g1 - g0, 0, 0), (0, 0, pos - line), (0, -1, 0), obj))
                    quads.append(((g0, 0, line), (g1 - g0, 0, 0), (0, 0, pos - line), (0, 1, 0), obj))
        obj += 1
    # furniture: boxes and cylinders, rooms chosen proportionally to area
    ra = np.array([(r[2] - r[0]) * (r[3] - r[1]) for r in rooms_free])
    cum = np.cumsum(ra / ra.sum())
    cyls, boxes, circles = [], [], []
    for k in range(n_objects):
        ri = int(np.searchsorted(cum, float(rs.uniform(1)[0]), side="right"))
        ri = min(ri, len(rooms_free) - 1)
        x0, z0, x1, z1 = rooms_free[ri]
        if float(rs.uniform(1)[0]) < 0.6:
            sx, sz = rs.uniform(2, 0.2, 1.2)
            sy = float(rs.uniform(1, 0.3, 2.0)[0])
            sx, sz = min(sx, x1 - x0 - 0.1), min(sz, z1 - z0 - 0.1)
            bx = float(rs.uniform(1, x0, x1 - sx)[0])
            bz = float(rs.uniform(1, z0, z1 - sz)[0])
            _box_faces(quads, bx, bz, bx + sx, bz + sz, 0.0, sy, obj)
            boxes.append((bx, bz, bx + float(sx), bz + float(sz)))
        else:
            r = float(rs.uniform(1, 0.1, 0.45)[0])
            r = min(r, 0.45 * (x1 - x0), 0.45 * (z1 - z0))
            hc = float(rs.uniform(1, 0.3, 1.6)[0])
            nk = int(rs.integers(1, 16, 33)[0])
            cx = float(rs.uniform(1, x0 + r, x1 - r)[0])
            cz = float(rs.uniform(1, z0 + r, z1 - r)[0])
            cyls.append((cx, cz, r, hc, nk, obj))
            circles.append((cx, cz, r))
        obj += 1
    return _Layout(quads, cyls, obj, rooms_free, boxes, circles)


def _tri_count(lay: _Layout, s: float) -> int:
    n = 0
    for o, a, b, _, _ in lay.quads:
        n += 2 * max(1, int(round(np.linalg.norm(a) / s))) * max(1, int(round(np.linalg.norm(b) / s)))
    for cx, cz, r, h, k, _ in lay.cylinders:
        seg = 2.0 * r * math.sin(math.pi / k)
        n += 2 * k * max(1, int(round(seg / s))) * max(1, int(round(h / s)))
        n += k * max(1, int(round(r / s))) ** 2
    return n


def _cell_size(lay: _Layout, target: int) -> float:
    s = math.sqrt(2.0 * lay.area() / target)
    for _ in range(30):
        n = _tri_count(lay, s)
        if abs(n - target) <= 0.01 * target:
            break
        s *= math.sqrt(n / target) ** (0.8)
    return s


def _pack_atlas(chart_wh: Sequence[Tuple[float, float]], aw: int, ah: int, pad: int = 2):
    """Shelf packing of planar charts at one texel density; returns (origin, rho)."""
    wh = np.array(chart_wh, dtype=np.float64)
    rho = math.sqrt(0.85 * aw * ah / max(1e-12, float((wh[:, 0] * wh[:, 1]).sum())))
    order = np.argsort(-wh[:, 1], kind="stable")
    for _ in range(200):
        cw = np.ceil(wh[:, 0] * rho).astype(np.int64) + 2 * pad + 1
        ch = np.ceil(wh[:, 1] * rho).astype(np.int64) + 2 * pad + 1
        origin = np.zeros((len(wh), 2), dtype=np.int64)
        x = y = shelf_h = 0
        ok = True
        for c in order:
            if cw[c] > aw:
                ok = False
                break
            if x + cw[c] > aw:
                y += shelf_h
                x, shelf_h = 0, 0
            origin[c] = (x, y)
            x += cw[c]
            shelf_h = max(shelf_h, int(ch[c]))
            if y + shelf_h > ah:
                ok = False
                break
        if ok:
            return origin, rho, pad
        rho *= 0.93
    raise RuntimeError("atlas packing failed")


def _atlas_noise(seed: int, aw: int, ah: int, kind: str) -> np.ndarray:
    st = Stream(seed, "atlas")
    n = aw * ah
    words = st.u64((n + 1) // 2)
    b = words.view(np.uint8).reshape(-1, 8)[:, :6].reshape(-1, 3)[:n]   # 3 bytes / texel
    tex = np.empty((ah, aw, 4), dtype=np.uint8)
    tex[..., :3] = b.reshape(ah, aw, 3)
    tex[..., 3] = 255
    if kind == "smooth":
        g = 16
        gw, gh = aw // g + 2, ah // g + 2
        coarse = Stream(seed, "atlas-smooth").u64(gw * gh * 3).view(np.uint8)[::8][: gw * gh * 3]
        coarse = coarse.reshape(gh, gw, 3).astype(np.float32)
        ys = np.arange(ah, dtype=np.float32) / g
        xs = np.arange(aw, dtype=np.float32) / g
        y0 = ys.astype(np.int64)
        x0 = xs.astype(np.int64)
        fy = (ys - y0)[:, None, None]
        fx = (xs - x0)[None, :, None]
        c = (coarse[y0][:, x0] * (1 - fx) * (1 - fy) + coarse[y0][:, x0 + 1] * fx * (1 - fy)
             + coarse[y0 + 1][:, x0] * (1 - fx) * fy + coarse[y0 + 1][:, x0 + 1] * fx * fy)
        tex[..., :3] = np.clip(0.85 * c + 0.15 * tex[..., :3].astype(np.float32), 0, 255).astype(np.uint8)
    return tex


def _build(lay: _Layout, target_tris: int, seed: int, atlas_size: Optional[int], vertex_colours: bool,
           semantic: bool, atlas_kind: str = "uniform", name: str = "") -> Scene:
    s = _cell_size(lay, target_tris)
    b = _Builder()
    for o, a, bb, nrm, obj in lay.quads:
        b.quad(o, a, bb, s, nrm, obj)
    for cx, cz, r, h, k, obj in lay.cylinders:
        b.cylinder(cx, cz, r, h, k, s, obj)
    xyz, tri, st, chart, obj = b.arrays()
    scene = Scene(xyz=xyz.astype(np.float32), idx=tri.astype(np.uint32), name=name)
    if atlas_size:
        origin, rho, pad = _pack_atlas(b.chart_size, atlas_size, atlas_size)
        u = (origin[chart, 0] + pad + st[:, 0] * rho) / atlas_size
        v = (origin[chart, 1] + pad + st[:, 1] * rho) / atlas_size
        scene.uv = np.stack([u, v], 1).astype(np.float32)
        scene.atlas = _atlas_noise(seed, atlas_size, atlas_size, atlas_kind)
    if vertex_colours:
        raw = Stream(seed, "vrgb3").u64(len(xyz) * 3)
        scene.vrgb = (raw & np.uint64(0xFF)).astype(np.uint8).reshape(-1, 3)
    if semantic:
        ids = (Stream(seed, "semantic").u64(lay.n_obj) >> np.uint64(33)).astype(np.uint32)
        scene.sem = ids[obj].astype(np.uint32)
    scene.rooms, scene.boxes, scene.circles = lay.rooms, lay.boxes, lay.circles
    return scene


# ----------------------------------------------------------------------------
# public recipes
# ----------------------------------------------------------------------------
def make_room(seed: int = 0, target_tris: int = 10_000) -> Scene:
    """Small room: 5x4x3 m, 20 boxes, ~10k triangles, random per-vertex RGB."""
    return _build(_layout_room(seed), target_tris, seed, None, True, False, name=f"room{seed}")


def make_house(seed: int = 0, target_tris: int = 1_000_000, atlas_size: int = 4096,
               semantic: bool = False, atlas_kind: str = "uniform", n_objects: int = 300) -> Scene:
    """Multi-room house (8-12 rooms, 300 boxes/cylinders) with one RGBA8 atlas."""
    return _build(_layout_house(seed, n_objects), target_tris, seed, atlas_size, False, semantic,
                  atlas_kind, name=f"house{seed}-{target_tris}")


def make_semantic_mesh(seed: int = 0, target_tris: int = 3_000_000, n_objects: int = 300) -> Scene:
    """The semantic mesh of make_house(seed): the same layout tessellated to
    `target_tris` triangles, no colour, a per-object semantic id per triangle
    (Table 2 footnote: semantic sensors read separate, denser meshes)."""
    return _build(_layout_house(seed, n_objects), target_tris, seed, None, False, True,
                  name=f"house{seed}-sem-{target_tris}")


def _free(scene: Scene, x: float, z: float, clear: float) -> bool:
    inside = any(r[0] + clear <= x <= r[2] - clear and r[1] + clear <= z <= r[3] - clear for r in scene.rooms)
    if not inside:
        return False
    for (x0, z0, x1, z1) in scene.boxes:
        if x0 - clear <= x <= x1 + clear and z0 - clear <= z <= z1 + clear:
            return False
    for (cx, cz, r) in scene.circles:
        if (x - cx) ** 2 + (z - cz) ** 2 <= (r + clear) ** 2:
            return False
    return True


AGENT_RADIUS = 0.1       # Sec. 4: cylinder of 0.2 m diameter
CAMERA_HEIGHT = 1.5      # Sec. 4: sensor 1.5 m above the agent base
FORWARD_STEP = 0.25      # Sec. 4: move_forward displacement
TURN_DEG = 10.0          # Sec. 4: turn_left / turn_right angle


def yaw_quat(theta: np.ndarray) -> np.ndarray:
    """Unit quaternions (w, x, y, z) for rotations by theta about +Y."""
    theta = np.asarray(theta, dtype=np.float64)
    q = np.zeros(theta.shape + (4,), dtype=np.float64)
    q[..., 0] = np.cos(theta / 2)
    q[..., 2] = np.sin(theta / 2)
    return q


def random_poses(scene: Scene, n: int, seed: int = 0) -> np.ndarray:
    """[n,7] float32 poses (x, y, z, qw, qx, qy, qz) on free floor, yaw uniform."""
    rs = Stream(seed, "poses-" + scene.name)
    out = np.zeros((n, 7), dtype=np.float64)
    ra = np.array([(r[2] - r[0]) * (r[3] - r[1]) for r in scene.rooms])
    cum = np.cumsum(ra / ra.sum())
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > 10000 * max(1, n):
            raise RuntimeError("no free space for poses")
        ri = min(int(np.searchsorted(cum, float(rs.uniform(1)[0]), side="right")), len(scene.rooms) - 1)
        x0, z0, x1, z1 = scene.rooms[ri]
        x = float(rs.uniform(1, x0, x1)[0])
        z = float(rs.uniform(1, z0, z1)[0])
        th = float(rs.uniform(1, 0.0, 2 * math.pi)[0])
        if not _free(scene, x, z, 2 * AGENT_RADIUS):
            continue
        out[k, :3] = (x, CAMERA_HEIGHT, z)
        out[k, 3:] = yaw_quat(np.array(th))
        k += 1
    return out.astype(np.float32)


def navmap(scene: Scene, cell: float = 0.05, clear: float = AGENT_RADIUS):
    """Top-down navigability grid of a scene: (x0, z0, cell, grid [nz, nx] u8),
    grid cell (i, k) covering [x0 + i cell, x0 + (i+1) cell) x [z0 + k cell, ...)
    is 1 iff its centre is free floor with `clear` metres to every wall and
    obstacle footprint (the agent cylinder of Sec. 4 fits there)."""
    r = np.array(scene.rooms, dtype=np.float64).reshape(-1, 4)
    x0, z0 = float(np.floor(r[:, 0].min())), float(np.floor(r[:, 1].min()))
    nx = int(math.ceil((r[:, 2].max() - x0) / cell)) + 1
    nz = int(math.ceil((r[:, 3].max() - z0) / cell)) + 1
    xc = x0 + (np.arange(nx) + 0.5) * cell
    zc = z0 + (np.arange(nz) + 0.5) * cell
    X, Z = np.meshgrid(xc, zc)
    free = np.zeros(X.shape, dtype=bool)
    for (a, b, c, d) in scene.rooms:
        free |= (X >= a + clear) & (X <= c - clear) & (Z >= b + clear) & (Z <= d - clear)
    for (a, b, c, d) in scene.boxes:
        free &= ~((X >= a - clear) & (X <= c + clear) & (Z >= b - clear) & (Z <= d + clear))
    for (cx, cz, rr) in scene.circles:
        free &= (X - cx) ** 2 + (Z - cz) ** 2 > (rr + clear) ** 2
    return np.float32(x0), np.float32(z0), np.float32(cell), free.astype(np.uint8)


def navigable_poses(scene: Scene, nav, n: int, seed: int = 0) -> np.ndarray:
    """[n,7] float32 poses at camera height on navigable cells of `nav`, yaw uniform."""
    x0, z0, cell, grid = nav
    rs = Stream(seed, "navposes-" + scene.name)
    ks, iis = np.nonzero(grid)
    pick = rs.integers(n, 0, len(ks))
    out = np.zeros((n, 7), dtype=np.float64)
    out[:, 0] = float(x0) + (iis[pick] + 0.5) * float(cell)
    out[:, 1] = CAMERA_HEIGHT
    out[:, 2] = float(z0) + (ks[pick] + 0.5) * float(cell)
    out[:, 3:] = yaw_quat(rs.uniform(n, 0.0, 2 * math.pi))
    return out.astype(np.float32)


class RandomWalk:
    """Agents stepping with move_forward 0.25 m / turn_left 10 deg / turn_right 10 deg,
    chosen uniformly; forward moves that leave free space are refused (no sliding)."""

    def __init__(self, scene: Scene, n_agents: int, seed: int = 0):
        self.scene = scene
        p = random_poses(scene, n_agents, seed)
        self.pos = p[:, :3].astype(np.float64)
        self.yaw = 2.0 * np.arctan2(p[:, 5].astype(np.float64), p[:, 3].astype(np.float64))
        self.rs = Stream(seed, "walk-" + scene.name)

    def step(self, agent: int) -> np.ndarray:
        a = int(self.rs.integers(1, 0, 3)[0])
        if a == 0:
            fwd = np.array([-math.sin(self.yaw[agent]), 0.0, -math.cos(self.yaw[agent])])
            nxt = self.pos[agent] + FORWARD_STEP * fwd
            if _free(self.scene, nxt[0], nxt[2], AGENT_RADIUS):
                self.pos[agent] = nxt
        elif a == 1:
            self.yaw[agent] += math.radians(TURN_DEG)
        else:
            self.yaw[agent] -= math.radians(TURN_DEG)
        return self.pose(agent)

    def pose(self, agent: int) -> np.ndarray:
        out = np.zeros(7, dtype=np.float64)
        out[:3] = self.pos[agent]
        out[3:] = yaw_quat(np.array(self.yaw[agent]))
        return out.astype(np.float32)


def dirichlet_split(total: int, parts: int, alpha: float, seed: int) -> np.ndarray:
    """Integer split of `total` items into `parts` (at least 1 each), proportions ~ Dirichlet(alpha).
    Gamma(1/2) variates are drawn as Z^2 / 2 (alpha must be 0.5 or 1)."""
    rs = Stream(seed, "dirichlet")
    if alpha == 0.5:
        g = rs.normal(parts) ** 2 / 2.0
    elif alpha == 1.0:
        g = -np.log1p(-rs.uniform(parts))
    else:
        raise ValueError("alpha must be 0.5 or 1.0")
    p = g / g.sum()
    rest = total - parts
    raw = p * rest
    base = np.floor(raw).astype(np.int64)
    rem = rest - int(base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:rem]] += 1
    return base + 1


def batching_scenes(seed: int = 0, n_scenes: int = 8, lo: float = 2e5, hi: float = 2e6,
                    atlas_size: int = 2048) -> List[Scene]:
    """Scenes with log-uniform triangle counts in [lo, hi], each with its own atlas."""
    rs = Stream(seed, "batching")
    counts = np.exp(rs.uniform(n_scenes, math.log(lo), math.log(hi))).astype(np.int64)
    return [make_house(seed * 1000 + i + 1, int(c), atlas_size) for i, c in enumerate(counts)]
