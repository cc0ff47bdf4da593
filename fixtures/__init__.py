"""Seeded synthetic inputs for the geometry-aware local-MLP renderer.

This module only *generates inputs*: occupancy grids shaped like indoor
captures, voxel-to-field labellings, per-field MLP weights and cameras.  It
holds none of the rendering arithmetic (ray generation, marching, field
lookup, positional encoding, MLP evaluation, compositing, gradients); both the
FP64 CPU oracle and the CUDA library consume what it produces.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` with
``seed = 1000 * workload_id + role`` (role 0 scene, 1 teacher weights,
2 student weights, 3 cameras, 4 ray batch, 5 noise), so any input can be
rebuilt from its workload id alone.

Conventions shared with the library's C ABI (the library documents them in
``include/roam.h``):

* grid bits: ``uint32[Gz][Gy][Gx/32]``, bit ``b`` of word ``w`` in a row is the
  voxel ``x = 32*w + b``; voxel ``(x,y,z)`` covers
  ``[origin + i*vox, origin + (i+1)*vox)`` on each axis;
* ``field_of_rank[r]`` is the field of the r-th occupied voxel in linear order
  ``(z*Gy + y)*Gx + x`` (x fastest);
* per-field affine ``(scale[3], offset[3])`` maps world points of the field's
  box onto ``[-1, 1]^3`` as ``scale*p + offset``;
* weights per field, FP32, in the layer order of the tiny MLP: W1[W][63], b1[W],
  then (H-1) x (Wk[W][W], bk[W]), Wh[1+W][W], bh[1+W] (row 0 is the density
  logit, rows 1..W the feature), Wc[W][W+27], bc[W], Wo[3][W], bo[3];
* camera: model (0 equirectangular, 1 perspective), width, height,
  horizontal field of view (radians, perspective only), camera-to-world
  rotation R (row-major 3x3) and centre o.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

ROLE_SCENE, ROLE_TEACHER, ROLE_STUDENT, ROLE_CAMERAS, ROLE_RAYS, ROLE_NOISE, ROLE_WIDTHS = range(7)

PE_POS_DIM = 63   # 3 + 2*3*10
PE_DIR_DIM = 27   # 3 + 2*3*4


def rng_for(workload: int, role: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * workload + role))


# ---------------------------------------------------------------------------
# occupancy grids
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    dims: Tuple[int, int, int]          # (Gx, Gy, Gz)
    origin: Tuple[float, float, float]
    vox: float
    occ: np.ndarray                     # bool [Gz][Gy][Gx]
    rooms: List[Tuple[Tuple[int, int, int], Tuple[int, int, int]]]  # interior boxes (lo, hi) voxels

    @property
    def bits(self) -> np.ndarray:
        return pack_bits(self.occ)

    @property
    def n_occupied(self) -> int:
        return int(self.occ.sum())


def pack_bits(occ: np.ndarray) -> np.ndarray:
    """bool [Gz][Gy][Gx] -> uint32 [Gz][Gy][Gx/32], x-fastest, LSB first."""
    gz, gy, gx = occ.shape
    if gx % 32:
        raise ValueError("Gx must be a multiple of 32")
    b = occ.reshape(gz, gy, gx // 32, 32).astype(np.uint64)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (b * weights).sum(axis=-1).astype(np.uint32)


def _box_sd(lo, hi, cx, cy, cz):
    """Signed distance (voxel units) from voxel centres to an axis-aligned box."""
    qx = np.maximum(lo[0] - cx, cx - hi[0])
    qy = np.maximum(lo[1] - cy, cy - hi[1])
    qz = np.maximum(lo[2] - cz, cz - hi[2])
    ox = np.maximum(qx, 0.0)
    oy = np.maximum(qy, 0.0)
    oz = np.maximum(qz, 0.0)
    outside = np.sqrt(ox * ox + oy * oy + oz * oz)
    inside = np.minimum(np.maximum(np.maximum(qx, qy), qz), 0.0)
    return outside + inside


def _rasterise(dims, solids, carves, sharpness, noise_sd, rng):
    """Probability field p = max_b peak_b * logistic(-k * sd_b) (+ noise), then
    the occupancy bits are p > 0.97 (the paper's occupied threshold)."""
    gx, gy, gz = dims
    p = np.zeros((gz, gy, gx), dtype=np.float32)
    for (lo, hi, peak) in solids:
        m = 2
        x0, y0, z0 = (max(0, lo[i] - m) for i in range(3))
        x1, y1, z1 = min(gx, hi[0] + m), min(gy, hi[1] + m), min(gz, hi[2] + m)
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            continue
        cz, cy, cx = np.meshgrid(np.arange(z0, z1) + 0.5, np.arange(y0, y1) + 0.5,
                                 np.arange(x0, x1) + 0.5, indexing="ij")
        sd = _box_sd(lo, hi, cx, cy, cz)
        pb = peak / (1.0 + np.exp(sharpness * sd))
        sub = p[z0:z1, y0:y1, x0:x1]
        np.maximum(sub, pb.astype(np.float32), out=sub)
    for (lo, hi) in carves:
        p[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 0.0
    if noise_sd > 0:
        p = p + rng.normal(0.0, noise_sd, size=p.shape).astype(np.float32)
    return p > 0.97


def room_scene(workload: int = 1, G: int = 32, vox: float = 0.1) -> Scene:
    """One room with walls, floor, ceiling and 6 furniture boxes in a G^3 grid
    (about 5% of voxels occupied); world y points down (floor at high y)."""
    rng = rng_for(workload, ROLE_SCENE)
    m = max(2, (3 * G) // 16)
    lo = np.array([m, m + 2, m])
    hi = np.array([G - m, G - m, G - m])
    solids = []
    peak = lambda: float(rng.uniform(0.985, 1.0))
    # floor (high y), ceiling (low y), 4 walls, 1 voxel thick
    solids.append(((lo[0], hi[1] - 1, lo[2]), (hi[0], hi[1], hi[2]), peak()))
    solids.append(((lo[0], lo[1], lo[2]), (hi[0], lo[1] + 1, hi[2]), peak()))
    solids.append(((lo[0], lo[1], lo[2]), (lo[0] + 1, hi[1], hi[2]), peak()))
    solids.append(((hi[0] - 1, lo[1], lo[2]), (hi[0], hi[1], hi[2]), peak()))
    solids.append(((lo[0], lo[1], lo[2]), (hi[0], hi[1], lo[2] + 1), peak()))
    solids.append(((lo[0], lo[1], hi[2] - 1), (hi[0], hi[1], hi[2]), peak()))
    inner_lo = lo + 1
    inner_hi = hi - 1
    for _ in range(6):
        sx, sz = rng.integers(2, max(3, G // 8) + 1, size=2)
        sy = int(rng.integers(2, max(3, G // 6) + 1))
        x0 = int(rng.integers(inner_lo[0], inner_hi[0] - sx + 1))
        z0 = int(rng.integers(inner_lo[2], inner_hi[2] - sz + 1))
        solids.append(((x0, inner_hi[1] - sy, z0), (x0 + sx, inner_hi[1], z0 + sz), peak()))
    occ = _rasterise((G, G, G), solids, [], sharpness=10.0, noise_sd=0.004, rng=rng)
    rooms = [(tuple(int(v) for v in inner_lo), tuple(int(v) for v in inner_hi))]
    return Scene((G, G, G), (0.0, 0.0, 0.0), vox, occ, rooms)


def floor_scene(workload: int, G: int, rooms_x: int, rooms_z: int, vox: float,
                wall: int = 2, height_frac: float = 0.3, boxes_per_room: int = 6) -> Scene:
    """A floor of rooms_x * rooms_z rooms (slab floor/ceiling, walls with
    doors, random furniture) inside a G^3 grid, probabilities with a sharp
    logistic at the surfaces, thresholded at 0.97."""
    rng = rng_for(workload, ROLE_SCENE)
    m = G // 16
    x_lo, x_hi = m, G - m
    z_lo, z_hi = m, G - m
    h = int(G * height_frac)
    y_lo = (G - h) // 2
    y_hi = y_lo + h
    solids, carves, rooms = [], [], []
    pk = 1.0
    solids.append(((x_lo, y_hi - wall, z_lo), (x_hi, y_hi, z_hi), pk))       # floor
    solids.append(((x_lo, y_lo, z_lo), (x_hi, y_lo + wall, z_hi), pk))       # ceiling
    xs = np.linspace(x_lo, x_hi, rooms_x + 1).round().astype(int)
    zs = np.linspace(z_lo, z_hi, rooms_z + 1).round().astype(int)
    # walls at room boundaries (exterior and interior)
    for i, xb in enumerate(xs):
        x0 = xb if i == 0 else (xb - wall if i == len(xs) - 1 else xb - wall // 2)
        solids.append(((x0, y_lo, z_lo), (x0 + wall, y_hi, z_hi), pk))
    for k, zb in enumerate(zs):
        z0 = zb if k == 0 else (zb - wall if k == len(zs) - 1 else zb - wall // 2)
        solids.append(((x_lo, y_lo, z0), (x_hi, y_hi, z0 + wall), pk))
    door_h = int(h * 0.6)
    door_w = max(4, G // 24)
    for i in range(1, rooms_x):           # doors through interior x-walls
        for k in range(rooms_z):
            zc = int(rng.integers(zs[k] + wall + door_w, zs[k + 1] - wall - door_w))
            xb = xs[i]
            carves.append(((xb - wall, y_hi - wall - door_h, zc - door_w // 2),
                           (xb + wall, y_hi - wall, zc + door_w // 2)))
    for k in range(1, rooms_z):           # doors through interior z-walls
        for i in range(rooms_x):
            xc = int(rng.integers(xs[i] + wall + door_w, xs[i + 1] - wall - door_w))
            zb = zs[k]
            carves.append(((xc - door_w // 2, y_hi - wall - door_h, zb - wall),
                           (xc + door_w // 2, y_hi - wall, zb + wall)))
    for i in range(rooms_x):
        for k in range(rooms_z):
            ilo = (xs[i] + wall, y_lo + wall, zs[k] + wall)
            ihi = (xs[i + 1] - wall, y_hi - wall, zs[k + 1] - wall)
            rooms.append((tuple(int(v) for v in ilo), tuple(int(v) for v in ihi)))
            for _ in range(boxes_per_room):
                sx = int(rng.integers(G // 48 + 2, G // 16 + 3))
                sz = int(rng.integers(G // 48 + 2, G // 16 + 3))
                sy = int(rng.integers(G // 48 + 2, h // 3))
                x0 = int(rng.integers(ilo[0], ihi[0] - sx))
                z0 = int(rng.integers(ilo[2], ihi[2] - sz))
                hang = rng.uniform() < 0.2          # some boxes hang from the ceiling
                y0 = ilo[1] if hang else ihi[1] - sy
                solids.append(((x0, y0, z0), (x0 + sx, y0 + sy, z0 + sz), pk))
    occ = _rasterise((G, G, G), solids, carves, sharpness=10.0, noise_sd=0.0, rng=rng)
    return Scene((G, G, G), (0.0, 0.0, 0.0), vox, occ, rooms)


# ---------------------------------------------------------------------------
# voxel -> field partitions (inputs to the renderer)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Partition:
    boxes: np.ndarray          # int32 [F][2][3]: half-open [lo, hi) in voxel coords (x,y,z)
    field_of_rank: np.ndarray  # uint16 [n_occupied]

    @property
    def n_fields(self) -> int:
        return int(self.boxes.shape[0])


def _occupied_xyz(occ: np.ndarray) -> np.ndarray:
    z, y, x = np.nonzero(occ)            # C order == linear order (x fastest)
    return np.stack([x, y, z], axis=1).astype(np.int32)


def _labels_from_boxes(xyz: np.ndarray, boxes: np.ndarray) -> np.ndarray:
    lab = np.full(xyz.shape[0], -1, dtype=np.int64)
    for f, (lo, hi) in enumerate(boxes):
        inside = np.all((xyz >= lo) & (xyz < hi), axis=1)
        lab[inside] = f
    if (lab < 0).any():
        raise RuntimeError("partition boxes do not cover every occupied voxel")
    return lab.astype(np.uint16)


def uniform_partition(scene: Scene, splits=(2, 2, 2)) -> Partition:
    """Equal-size cells (the uniform decomposition variant); cell order is
    x fastest, then y, then z."""
    gx, gy, gz = scene.dims
    boxes = []
    for k in range(splits[2]):
        for j in range(splits[1]):
            for i in range(splits[0]):
                lo = (gx * i // splits[0], gy * j // splits[1], gz * k // splits[2])
                hi = (gx * (i + 1) // splits[0], gy * (j + 1) // splits[1], gz * (k + 1) // splits[2])
                boxes.append((lo, hi))
    boxes = np.array(boxes, dtype=np.int32)
    return Partition(boxes, _labels_from_boxes(_occupied_xyz(scene.occ), boxes))


def kd_partition(scene: Scene, n_fields: int) -> Partition:
    """Recursive split of the grid box along its longest axis at the median
    occupied-voxel coordinate until n_fields leaves (a power of two) remain, so
    that leaves hold similar numbers of occupied voxels but cover different
    volumes.  Leaves are numbered in depth-first (low side first) order."""
    if n_fields & (n_fields - 1):
        raise ValueError("kd partition needs a power-of-two field count")
    xyz = _occupied_xyz(scene.occ)
    depth = int(round(math.log2(n_fields)))
    leaves = []

    def rec(idx, lo, hi, d):
        if d == 0:
            leaves.append((lo.copy(), hi.copy(), idx))
            return
        ext = hi - lo
        # longest axis first; fall back to another axis when occupied voxels
        # pile up on one plane (a floor slab) and the median split is lopsided
        best = None
        for axis in sorted(range(3), key=lambda a: (-ext[a], a)):
            if ext[axis] < 2:
                continue
            if idx.size >= 2:
                vals = np.sort(xyz[idx, axis])
                med = int(vals[idx.size // 2])
                cands = [med, med + 1]
            else:
                cands = [int((lo[axis] + hi[axis]) // 2)]
            for s in cands:
                s = min(max(s, int(lo[axis]) + 1), int(hi[axis]) - 1)
                nl = int(np.count_nonzero(xyz[idx, axis] < s)) if idx.size else 0
                imb = abs(2 * nl - idx.size)
                if best is None or imb < best[0]:
                    best = (imb, axis, s)
            if best[0] <= idx.size // 2:
                break
        if best is None:
            raise RuntimeError("kd split ran out of voxels")
        _, axis, s = best
        left = idx[xyz[idx, axis] < s]
        right = idx[xyz[idx, axis] >= s]
        hl = hi.copy(); hl[axis] = s
        lr = lo.copy(); lr[axis] = s
        rec(left, lo, hl, d - 1)
        rec(right, lr, hi, d - 1)

    rec(np.arange(xyz.shape[0]), np.zeros(3, dtype=np.int64), np.array(scene.dims, dtype=np.int64), depth)
    boxes = np.array([(lo, hi) for (lo, hi, _) in leaves], dtype=np.int32)
    # each occupied voxel lies in the leaf whose subset it reached (the boxes
    # tile the grid, so this is also the containing box)
    lab = np.full(xyz.shape[0], -1, dtype=np.int64)
    for f, (_, _, idx) in enumerate(leaves):
        lab[idx] = f
    if (lab < 0).any():
        raise RuntimeError("kd leaves do not cover every occupied voxel")
    return Partition(boxes, lab.astype(np.uint16))


def field_affine(scene: Scene, part: Partition) -> np.ndarray:
    """float32 [F][6] = (scale xyz, offset xyz) mapping each field's world box
    onto [-1, 1]^3."""
    o = np.array(scene.origin, dtype=np.float64)
    lo = o + part.boxes[:, 0, :].astype(np.float64) * scene.vox
    hi = o + part.boxes[:, 1, :].astype(np.float64) * scene.vox
    scale = 2.0 / (hi - lo)
    offset = -1.0 - lo * scale
    return np.concatenate([scale, offset], axis=1).astype(np.float32)


# ---------------------------------------------------------------------------
# per-field MLP weights
# ---------------------------------------------------------------------------

def layer_shapes(W: int, H: int, pos_dim: int = PE_POS_DIM, dir_dim: int = PE_DIR_DIM):
    """(out, in) of each fully-connected layer, in storage order."""
    shapes = [(W, pos_dim)]
    shapes += [(W, W)] * (H - 1)
    shapes += [(1 + W, W), (W, W + dir_dim), (3, W)]
    return shapes


def n_params(W: int, H: int) -> int:
    return sum(o * i + o for o, i in layer_shapes(W, H))


def xavier_weights(workload: int, role: int, n_fields: int, W: int, H: int,
                   bias_scale: float = 0.0) -> np.ndarray:
    """float32 [F][P]: Xavier-uniform matrices, biases zero (or uniform in
    +-bias_scale when asked, to exercise the bias paths)."""
    rng = rng_for(workload, role)
    P = n_params(W, H)
    out = np.empty((n_fields, P), dtype=np.float32)
    for f in range(n_fields):
        parts = []
        for (o, i) in layer_shapes(W, H):
            a = math.sqrt(6.0 / (o + i))
            parts.append(rng.uniform(-a, a, size=o * i))
            parts.append(rng.uniform(-bias_scale, bias_scale, size=o) if bias_scale else np.zeros(o))
        out[f] = np.concatenate(parts).astype(np.float32)
    return out


def mixed_widths(workload: int, n_fields: int, choices=(32, 64, 128)) -> np.ndarray:
    """int32 [F]: an MLP width per field, drawn uniformly from `choices`."""
    rng = rng_for(workload, ROLE_WIDTHS)
    return np.asarray(choices, dtype=np.int32)[rng.integers(0, len(choices), n_fields)]


def xavier_weights_mixed(workload: int, role: int, widths: np.ndarray, H: int, bias_scale: float = 0.0) -> np.ndarray:
    """float32 1-D: the fields' parameters one after another, field f in the
    layout of width widths[f] (Xavier-uniform matrices as xavier_weights)."""
    rng = rng_for(workload, role)
    parts = []
    for W in widths:
        for (o, i) in layer_shapes(int(W), H):
            a = math.sqrt(6.0 / (o + i))
            parts.append(rng.uniform(-a, a, size=o * i))
            parts.append(rng.uniform(-bias_scale, bias_scale, size=o) if bias_scale else np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def density_scale(delta: float, median_alpha: float = 0.3) -> float:
    """Density multiplier so that a sample with density logit 0 (the median
    for symmetric random weights: softplus(0) = ln 2) has opacity
    median_alpha over one step of length delta."""
    return -math.log(1.0 - median_alpha) / (delta * math.log(2.0))


# ---------------------------------------------------------------------------
# cameras and ray batches
# ---------------------------------------------------------------------------

EQUIRECT, PERSPECTIVE = 0, 1


@dataclasses.dataclass
class Camera:
    model: int
    width: int
    height: int
    fov_h: float
    R: np.ndarray   # float64 [3][3] camera-to-world
    o: np.ndarray   # float64 [3]

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


def yaw_pitch(yaw: float, pitch: float = 0.0) -> np.ndarray:
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    return Ry @ Rx


def random_free_position(scene: Scene, rng: np.random.Generator, room: Optional[int] = None) -> np.ndarray:
    """World position at the centre of a free voxel inside a room's inner half."""
    for _ in range(10000):
        r = int(rng.integers(len(scene.rooms))) if room is None else room
        lo, hi = (np.array(v) for v in scene.rooms[r])
        q0 = lo + (hi - lo) // 4
        q1 = np.maximum(q0 + 1, hi - (hi - lo) // 4)
        v = np.array([rng.integers(q0[i], q1[i]) for i in range(3)])
        x, y, z = v
        nb = scene.occ[max(z - 1, 0):z + 2, max(y - 1, 0):y + 2, max(x - 1, 0):x + 2]
        if not nb.any():
            return np.array(scene.origin) + (v + 0.5) * scene.vox
    raise RuntimeError("no free voxel found")


def make_cameras(scene: Scene, workload: int, specs) -> List[Camera]:
    """specs: list of (model, width, height, fov_h); one seeded pose each."""
    rng = rng_for(workload, ROLE_CAMERAS)
    cams = []
    for (model, w, h, fov) in specs:
        o = random_free_position(scene, rng)
        R = yaw_pitch(float(rng.uniform(0, 2 * math.pi)), float(rng.uniform(-0.15, 0.15)))
        cams.append(Camera(model, w, h, fov, R, o))
    return cams


def ray_batch(workload: int, cams: List[Camera], n_rays: int) -> np.ndarray:
    """uint32 [n_rays][2] of (view, pixel) drawn uniformly over all pixels."""
    rng = rng_for(workload, ROLE_RAYS)
    sizes = np.array([c.n_pixels for c in cams], dtype=np.int64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    g = rng.integers(0, starts[-1], size=n_rays)
    view = np.searchsorted(starts, g, side="right") - 1
    pix = g - starts[view]
    return np.stack([view, pix], axis=1).astype(np.uint32)


def camera_array(cams: List[Camera]) -> np.ndarray:
    """float64 [n][16] = (model, width, height, fov_h, R[9], o[3]) for the
    oracle; the library takes its own struct built from the same fields."""
    out = np.zeros((len(cams), 16), dtype=np.float64)
    for i, c in enumerate(cams):
        out[i, 0:4] = (c.model, c.width, c.height, c.fov_h)
        out[i, 4:13] = np.asarray(c.R, dtype=np.float64).reshape(9)
        out[i, 13:16] = c.o
    return out


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    part: Partition
    affine: np.ndarray
    W: int
    H: int
    weights: np.ndarray
    sigma_scale: float
    delta: float
    n_max: int
    cams: List[Camera]
    t_stop: float = 1e-4
    widths: Optional[np.ndarray] = None     # per-field MLP widths (W == 0, weights 1-D) when mixed


def room32(W: int = 32, H: int = 2) -> Workload:
    """32^3 room, 8 fields on a uniform 2x2x2 split, W=32/H=2 MLPs
    (6,212 parameters each), one 128x64 equirectangular view, <=64 samples."""
    scene = room_scene(1, 32, 0.1)
    part = uniform_partition(scene, (2, 2, 2))
    delta = scene.vox / 4
    w = xavier_weights(1, ROLE_TEACHER, part.n_fields, W, H)
    cams = make_cameras(scene, 1, [(EQUIRECT, 128, 64, 0.0)])
    return Workload("room32_u8_w32h2_equirect128x64", scene, part, field_affine(scene, part), W, H, w,
                    density_scale(delta), delta, 64, cams)


def floor256(views: str = "both", n_fields: int = 512, W: int = 64, H: int = 3, role: int = ROLE_TEACHER) -> Workload:
    """256^3 eight-room floor, 512 kd fields, W=64/H=3 MLPs (22,724
    parameters each), 1024x512 equirectangular and 1920x1080 perspective
    (90 degree horizontal FOV) views, <=128 samples per ray."""
    scene = floor_scene(2, 256, 4, 2, 0.04)
    part = kd_partition(scene, n_fields)
    delta = scene.vox / 4
    w = xavier_weights(2, role, part.n_fields, W, H)
    specs = []
    if views in ("both", "equirect"):
        specs.append((EQUIRECT, 1024, 512, 0.0))
    if views in ("both", "perspective"):
        specs.append((PERSPECTIVE, 1920, 1080, math.pi / 2))
    cams = make_cameras(scene, 2, specs)
    return Workload(f"floor256_kd{n_fields}_w{W}h{H}", scene, part, field_affine(scene, part), W, H, w,
                    density_scale(delta), delta, 128, cams)


def floor512(n_fields: int = 4096, W: int = 128, H: int = 4, role: int = ROLE_TEACHER) -> Workload:
    """512^3 twenty-room floor (5 x 4 rooms, about 2% of voxels occupied),
    4096 kd fields, W=128/H=4 MLPs (94,724 parameters each), one 2048x1024
    equirectangular view, <=192 samples per ray."""
    scene = floor_scene(5, 512, 5, 4, 0.03, height_frac=0.25, boxes_per_room=3)
    part = kd_partition(scene, n_fields)
    delta = scene.vox / 4
    w = xavier_weights(5, role, part.n_fields, W, H)
    cams = make_cameras(scene, 5, [(EQUIRECT, 2048, 1024, 0.0)])
    return Workload(f"floor512_kd{n_fields}_w{W}h{H}", scene, part, field_affine(scene, part), W, H, w,
                    density_scale(delta), delta, 192, cams)


def multiview_specs():
    """32 views: 24 equirectangular panoramas in four sizes from 512x256 to
    2048x1024, and 8 perspective 1280x720 views at 90 degrees horizontal FOV,
    interleaved."""
    eq = [(512, 256), (1024, 512), (1536, 768), (2048, 1024)]
    specs = []
    for i in range(32):
        if i % 4 == 3:
            specs.append((PERSPECTIVE, 1280, 720, math.pi / 2))
        else:
            w, h = eq[(i - i // 4) % 4]
            specs.append((EQUIRECT, w, h, 0.0))
    return specs


def floor384(n_fields: int = 2048, H: int = 3, role: int = ROLE_TEACHER, specs=None) -> Workload:
    """384^3 twelve-room floor (4 x 3 rooms), 2048 kd fields whose MLP widths
    are drawn from 32/64/128 per field, H=3, the 32 mixed views of
    multiview_specs, <=128 samples per ray."""
    scene = floor_scene(4, 384, 4, 3, 0.03, height_frac=0.28, boxes_per_room=4)
    part = kd_partition(scene, n_fields)
    delta = scene.vox / 4
    widths = mixed_widths(4, part.n_fields)
    w = xavier_weights_mixed(4, role, widths, H)
    cams = make_cameras(scene, 4, specs if specs is not None else multiview_specs())
    return Workload(f"floor384_kd{n_fields}_mixedw_h{H}", scene, part, field_affine(scene, part), 0, H, w,
                    density_scale(delta), delta, 128, cams, widths=widths)


def roaming_path(scene: Scene, workload: int, n_frames: int, width: int = 1280, height: int = 720,
                 fov_h: float = math.pi / 2, step: float = 0.02) -> List[Camera]:
    """A walk through one room: start at a seeded free voxel, move `step`
    per frame along a seeded heading at eye height, turning slowly, and turn
    back at occupied voxels; one perspective camera per frame."""
    rng = rng_for(workload, ROLE_CAMERAS)
    o = random_free_position(scene, rng)
    yaw = float(rng.uniform(0, 2 * math.pi))
    cams = []
    for _ in range(n_frames):
        R = yaw_pitch(yaw, 0.0)
        fwd = R[:, 2]
        nxt = o + step * fwd
        c = np.floor((nxt - np.asarray(scene.origin)) / scene.vox).astype(int)
        inside = np.all(c >= 0) and np.all(c < np.asarray(scene.dims))
        if not inside or scene.occ[c[2], c[1], c[0]]:
            yaw += math.pi * 0.75
        else:
            o = nxt
        yaw += 0.01
        cams.append(Camera(PERSPECTIVE, width, height, fov_h, yaw_pitch(yaw, 0.0), o.copy()))
    return cams


def teacher_layer_shapes(W: int = 256, C: int = 128, pos_dim: int = PE_POS_DIM, dir_dim: int = PE_DIR_DIM):
    """(out, in) of every layer of the global 360NeRF, in storage order:
    layers 1-4, layer 5 on [layer 4; F(x)], layers 6-8, density head,
    feature head, layer 10 on [feature; F(d)], layer 11."""
    return ([(W, pos_dim)] + [(W, W)] * 3 + [(W, W + pos_dim)] + [(W, W)] * 3 + [(1, W), (W, W),
            (C, W + dir_dim), (3, C)])


def teacher_weights(workload: int, role: int = ROLE_TEACHER, bias_scale: float = 0.0) -> np.ndarray:
    """float32 [P] Xavier-uniform weights of the global 360NeRF (seeded)."""
    rng = rng_for(workload, role)
    parts = []
    for (o, i) in teacher_layer_shapes():
        a = math.sqrt(6.0 / (o + i))
        parts.append(rng.uniform(-a, a, size=o * i))
        parts.append(rng.uniform(-bias_scale, bias_scale, size=o) if bias_scale else np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def scene_affine(scene: Scene) -> np.ndarray:
    """float32 [6]: the whole grid box onto [-1, 1]^3 (scale xyz, offset xyz)."""
    o = np.array(scene.origin, dtype=np.float64)
    ext = np.array(scene.dims, dtype=np.float64) * scene.vox
    scale = 2.0 / ext
    return np.concatenate([scale, -1.0 - o * scale]).astype(np.float32)


def distill_points(scene: Scene, part: Partition, workload: int, per_field: int, step: int = 0):
    """Distillation samples: per field, `per_field` points uniform in
    uniformly drawn occupied voxels of the field, with uniform directions.
    Returns (p float32 [n, 3], d float32 [n, 3], field int32 [n])."""
    rng = rng_for(workload * 1000 + step, ROLE_RAYS)
    xyz = _occupied_xyz(scene.occ)
    lab = part.field_of_rank.astype(np.int64)
    order = np.argsort(lab, kind="stable")
    starts = np.searchsorted(lab[order], np.arange(part.n_fields + 1))
    ps, ds, fs = [], [], []
    for f in range(part.n_fields):
        cand = order[starts[f]:starts[f + 1]]
        if cand.size == 0:
            continue
        pick = cand[rng.integers(0, cand.size, per_field)]
        pts = (xyz[pick] + rng.uniform(0, 1, (per_field, 3))) * scene.vox + np.asarray(scene.origin)
        dd = rng.normal(size=(per_field, 3))
        dd /= np.linalg.norm(dd, axis=1, keepdims=True)
        ps.append(pts); ds.append(dd); fs.append(np.full(per_field, f))
    return (np.concatenate(ps).astype(np.float32), np.concatenate(ds).astype(np.float32),
            np.concatenate(fs).astype(np.int32))
