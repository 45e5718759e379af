"""Seeded synthetic inputs shaped like the paper's RGB-D workloads.

This module only draws inputs. It holds none of the rasterizer's arithmetic (no
projection, compositing, loss or gradient). Both the CUDA path and the oracle take
their inputs from it. The paper evaluates on TUM RGB-D (Sec. IV-A: 640 x 480 Kinect
frames); that dataset is not available here, so these scenes stand in for it:

* ``cube_scene``: Gaussians in a 2 m cube 1-3 m in front of the camera (the 160 x 120
  single-view case).
* ``room_scene``: Gaussians on the walls, floor and three boxes of a 5 x 4 x 3 m room,
  with a piecewise-smooth texture (the 640 x 480 tracking, 1200 x 680 mapping,
  batched-hypothesis and long-sequence cases).
* ``raycast_room``: an RGB-D "sensor" frame of the same room, made by intersecting
  pixel rays with the room's rectangles (plain geometry, not splatting). The benchmark
  uses it as its target frame; ``raycast_room_torch`` is the same in torch, for the
  long sequence's 200 frames on the GPU.
* ``spline_trajectory``: the long sequence's camera path around the room.

All floating-point attributes are returned as float32. That is what the GPU consumes;
the oracle receives the same values widened to float64.  Quaternions are (w, x, y, z);
poses are world->camera ``[qw, qx, qy, qz, tx, ty, tz]`` (float64).
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial.transform import Rotation

ROOM = (5.0, 3.0, 4.0)  # x extent, y (height) extent, z extent in metres


@dataclasses.dataclass
class Cam:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclasses.dataclass
class Gaussians:
    means: np.ndarray       # n x 3 float32
    quats: np.ndarray       # n x 4 float32, (w, x, y, z), not normalised
    log_scales: np.ndarray  # n x 3 float32
    logits: np.ndarray      # n float32
    rgb: np.ndarray         # n x 3 float32

    @property
    def n(self) -> int:
        return self.means.shape[0]

    def arrays(self):
        return self.means, self.quats, self.log_scales, self.logits, self.rgb


def _quat_wxyz(rot: Rotation) -> np.ndarray:
    x, y, z, w = rot.as_quat()
    return np.array([w, x, y, z], dtype=np.float64)


def pose_from_rt(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Pack a world->camera rotation matrix and translation as [qw, qx, qy, qz, t]."""
    q = _quat_wxyz(Rotation.from_matrix(np.asarray(R, dtype=np.float64)))
    if q[0] < 0:
        q = -q
    return np.concatenate([q, np.asarray(t, dtype=np.float64)])


def pose_rt(pose) -> tuple[np.ndarray, np.ndarray]:
    pose = np.asarray(pose, dtype=np.float64)
    w, x, y, z = pose[:4]
    return Rotation.from_quat([x, y, z, w]).as_matrix(), pose[4:7].copy()


def identity_pose() -> np.ndarray:
    return np.array([1.0, 0, 0, 0, 0, 0, 0])


def look_at(center, forward, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera pose of a camera at `center` looking along `forward` (x right,
    y down, z forward in the camera frame; world y is up)."""
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    xr = np.cross(f, np.asarray(up, dtype=np.float64))
    xr /= np.linalg.norm(xr)
    yd = np.cross(f, xr)
    R = np.stack([xr, yd, f])
    t = -R @ np.asarray(center, dtype=np.float64)
    return pose_from_rt(R, t)


def perturb_pose(pose, rng: np.random.Generator, rot_deg: float, trans_m: float) -> np.ndarray:
    """Rotate by exactly `rot_deg` about a uniform random axis (applied on the left) and
    shift the translation by exactly `trans_m` along a uniform random direction."""
    R, t = pose_rt(pose)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    dR = Rotation.from_rotvec(axis * np.deg2rad(rot_deg)).as_matrix()
    return pose_from_rt(dR @ R, t + trans_m * d)


def jitter_pose(pose, rng: np.random.Generator, rot_sigma_deg: float, trans_sigma_m: float) -> np.ndarray:
    """Rotation vector ~ N(0, sigma) per axis (left), translation += N(0, sigma) per axis."""
    R, t = pose_rt(pose)
    dR = Rotation.from_rotvec(rng.normal(0.0, np.deg2rad(rot_sigma_deg), size=3)).as_matrix()
    return pose_from_rt(dR @ R, t + rng.normal(0.0, trans_sigma_m, size=3))


def _random_quats(rng, n):
    return rng.normal(size=(n, 4)).astype(np.float32)


# ----------------------------------------------------------------------------- cube scene

def cube_scene(n: int = 2000, seed: int = 0) -> tuple[Gaussians, Cam]:
    """Means uniform in [-1,1]^2 x [1,3] (camera frame at the identity pose), log-scales
    N(-3.5, 0.3) per axis, random quaternions, logits N(0, 1), rgb U(0, 1); a 160 x 120
    pinhole camera with fx = fy = 140 and the principal point at the image centre."""
    rng = np.random.default_rng(seed)
    means = rng.uniform([-1.0, -1.0, 1.0], [1.0, 1.0, 3.0], size=(n, 3)).astype(np.float32)
    log_scales = rng.normal(-3.5, 0.3, size=(n, 3)).astype(np.float32)
    quats = _random_quats(rng, n)
    logits = rng.normal(0.0, 1.0, size=n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    cam = Cam(140.0, 140.0, 79.5, 59.5, 160, 120)
    return Gaussians(means, quats, log_scales, logits, rgb), cam


# ----------------------------------------------------------------------------- room scene

@dataclasses.dataclass
class _Rect:
    origin: np.ndarray
    u: np.ndarray      # unit vector along the first side
    v: np.ndarray      # unit vector along the second side
    su: float
    sv: float
    normal: np.ndarray  # facing into the room
    base: np.ndarray    # base colour
    phase: float


def _box_rects(lo, hi, base, phase):
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    ex, ey, ez = np.eye(3)
    sx, sy, sz = hi - lo
    return [
        _Rect(np.array([lo[0], hi[1], lo[2]]), ex, ez, sx, sz, ey, base, phase),             # top
        _Rect(np.array([lo[0], lo[1], lo[2]]), ex, ey, sx, sy, -ez, base * 0.9, phase + 1),  # front (z=lo)
        _Rect(np.array([lo[0], lo[1], hi[2]]), ex, ey, sx, sy, ez, base * 0.8, phase + 2),   # back (z=hi)
        _Rect(np.array([lo[0], lo[1], lo[2]]), ez, ey, sz, sy, -ex, base * 0.85, phase + 3), # left (x=lo)
        _Rect(np.array([hi[0], lo[1], lo[2]]), ez, ey, sz, sy, ex, base * 0.95, phase + 4),  # right (x=hi)
    ]


def room_rects(seed: int = 0) -> list:
    """The room's textured rectangles: four walls and the floor of a 5 x 3 x 4 m room
    (no ceiling) plus three axis-aligned boxes at seeded floor positions."""
    rng = np.random.default_rng(seed + 7919)
    X, Y, Z = ROOM
    ex, ey, ez = np.eye(3)
    rects = [
        _Rect(np.zeros(3), ez, ey, Z, Y, ex, np.array([0.75, 0.55, 0.45]), 0.3),               # wall x = 0
        _Rect(np.array([X, 0, 0]), ez, ey, Z, Y, -ex, np.array([0.45, 0.6, 0.75]), 1.1),       # wall x = X
        _Rect(np.zeros(3), ex, ey, X, Y, ez, np.array([0.6, 0.7, 0.5]), 2.3),                  # wall z = 0
        _Rect(np.array([0, 0, Z]), ex, ey, X, Y, -ez, np.array([0.8, 0.75, 0.6]), 3.7),        # wall z = Z
        _Rect(np.zeros(3), ex, ez, X, Z, ey, np.array([0.5, 0.45, 0.4]), 4.9),                 # floor y = 0
    ]
    sizes = [(0.8, 0.6, 0.5), (0.5, 1.0, 0.5), (1.2, 0.4, 0.7)]
    for k, (sx, sy, sz) in enumerate(sizes):
        x0 = rng.uniform(0.3, X - 0.3 - sx)
        z0 = rng.uniform(1.8, Z - 0.3 - sz) if k < 2 else rng.uniform(0.3, Z - 0.3 - sz)
        base = rng.uniform(0.25, 0.9, size=3)
        rects += _box_rects((x0, 0.0, z0), (x0 + sx, sy, z0 + sz), base, 6.0 + k)
    return rects


def _texture(rect: _Rect, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Piecewise-smooth colour at in-plane coordinates (a, b) metres: base colour, a
    low-frequency sine pattern (amplitude 0.15) and 0.5 m checker blocks, clipped."""
    s = 0.15 * np.sin(2.0 * np.pi * a / 1.7 + rect.phase) * np.sin(2.0 * np.pi * b / 1.3 + 0.5 * rect.phase)
    chk = ((np.floor(a / 0.5) + np.floor(b / 0.5)) % 2) * 0.12 - 0.06
    c = rect.base[None, :] + (s + chk)[:, None]
    return np.clip(c, 0.0, 1.0)


def morton_codes(points: np.ndarray, cell: float) -> np.ndarray:
    """Morton (Z-order) codes of points quantised to `cell`-sized cubes (21 bits per axis)."""
    q = np.clip(np.floor((points - points.min(axis=0)) / cell), 0, (1 << 21) - 1).astype(np.uint64)

    def spread(x):
        x = x & np.uint64(0x1FFFFF)
        x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
        return x

    return spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))


def room_scene(n: int, seed: int = 0, log_scale_mu: float = -4.0, log_scale_sigma: float = 0.4,
               logit_mu: float = 2.0, logit_sigma: float = 1.0, jitter_m: float = 0.005,
               ordered: bool = True) -> Gaussians:
    """`n` Gaussians with means sampled area-uniformly on the room's surfaces plus
    N(0, 5 mm) jitter along the normal, log-scales N(-4, 0.4), random quaternions,
    logits N(2, 1) and the room texture as colour; listed along a Morton curve of their
    means (ordered=False keeps the sampling order)."""
    rng = np.random.default_rng(seed)
    rects = room_rects(seed)
    areas = np.array([r.su * r.sv for r in rects])
    which = rng.choice(len(rects), size=n, p=areas / areas.sum())
    a = rng.uniform(0.0, 1.0, size=n)
    b = rng.uniform(0.0, 1.0, size=n)
    jit = rng.normal(0.0, jitter_m, size=n)
    means = np.zeros((n, 3))
    rgb = np.zeros((n, 3))
    for k, r in enumerate(rects):
        sel = which == k
        aa, bb = a[sel] * r.su, b[sel] * r.sv
        means[sel] = r.origin + aa[:, None] * r.u + bb[:, None] * r.v + jit[sel, None] * r.normal
        rgb[sel] = _texture(r, aa, bb)
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, size=(n, 3))
    quats = _random_quats(rng, n)
    logits = rng.normal(logit_mu, logit_sigma, size=n)
    if ordered:
        # a map built frame by frame lists neighbouring Gaussians together; so does this
        # one, along a Morton curve of the means (1 cm cells)
        order = np.argsort(morton_codes(means, 0.01), kind="stable")
        means, rgb, log_scales, quats, logits = means[order], rgb[order], log_scales[order], quats[order], logits[order]
    return Gaussians(means.astype(np.float32), quats, log_scales.astype(np.float32),
                     logits.astype(np.float32), rgb.astype(np.float32))


def raycast_room(pose, cam: Cam, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """RGB (3 x H x W) and depth (H x W, camera-frame z; 0 where no surface) of the room
    seen from `pose`, by intersecting every pixel-centre ray with the rectangles."""
    R, t = pose_rt(pose)
    H, W = cam.height, cam.width
    v, u = np.mgrid[0:H, 0:W].astype(np.float64)
    dc = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u)], axis=-1).reshape(-1, 3)
    dw = dc @ R           # rows: R^T d
    ow = -R.T @ t
    best = np.full(dw.shape[0], np.inf)
    col = np.zeros((dw.shape[0], 3))
    for r in room_rects(seed):
        den = dw @ r.normal
        with np.errstate(divide="ignore", invalid="ignore"):
            s = ((r.origin - ow) @ r.normal) / den
        hit = ow[None, :] + s[:, None] * dw - r.origin
        aa, bb = hit @ r.u, hit @ r.v
        ok = (np.abs(den) > 1e-12) & (s > 1e-6) & (aa >= 0) & (aa <= r.su) & (bb >= 0) & (bb <= r.sv) & (s < best)
        best[ok] = s[ok]
        if ok.any():
            col[ok] = _texture(r, aa[ok], bb[ok])
    depth = np.where(np.isfinite(best), best, 0.0)   # ray z-component is 1, so s is the camera depth
    rgb = col.T.reshape(3, H, W)
    return rgb.astype(np.float32), depth.reshape(H, W).astype(np.float32)


def raycast_room_torch(pose, cam: Cam, seed: int = 0, device="cpu"):
    """raycast_room in float64 torch on `device` (a GPU makes a long sequence's frames in
    milliseconds each): the same rays, rectangles and texture; returns float32 tensors
    rgb (3 x H x W) and depth (H x W)."""
    import torch
    f64 = dict(dtype=torch.float64, device=device)
    R, t = pose_rt(pose)
    H, W = cam.height, cam.width
    v, u = torch.meshgrid(torch.arange(H, **f64), torch.arange(W, **f64), indexing="ij")
    dc = torch.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, torch.ones_like(u)], -1).reshape(-1, 3)
    Rt = torch.as_tensor(R, **f64)
    dw = dc @ Rt
    ow = -Rt.T @ torch.as_tensor(t, **f64)
    best = torch.full((dw.shape[0],), float("inf"), **f64)
    col = torch.zeros(dw.shape[0], 3, **f64)
    for r in room_rects(seed):
        nrm, org = torch.as_tensor(r.normal, **f64), torch.as_tensor(r.origin, **f64)
        ru, rv = torch.as_tensor(r.u, **f64), torch.as_tensor(r.v, **f64)
        den = dw @ nrm
        s = ((org - ow) @ nrm) / den
        hit = ow[None, :] + s[:, None] * dw - org
        aa, bb = hit @ ru, hit @ rv
        ok = (den.abs() > 1e-12) & (s > 1e-6) & (aa >= 0) & (aa <= r.su) & (bb >= 0) & (bb <= r.sv) & (s < best)
        best = torch.where(ok, s, best)
        sn = 0.15 * torch.sin(2.0 * np.pi * aa / 1.7 + r.phase) * torch.sin(2.0 * np.pi * bb / 1.3 + 0.5 * r.phase)
        chk = torch.remainder(torch.floor(aa / 0.5) + torch.floor(bb / 0.5), 2) * 0.12 - 0.06
        c = (torch.as_tensor(r.base, **f64)[None, :] + (sn + chk)[:, None]).clamp(0.0, 1.0)
        col = torch.where(ok[:, None], c, col)
    depth = torch.where(torch.isfinite(best), best, torch.zeros_like(best))
    return col.T.reshape(3, H, W).float().contiguous(), depth.reshape(H, W).float().contiguous()


def prior_from_depth(depth: np.ndarray, rng: np.random.Generator, sigma: float, hole_frac: float) -> np.ndarray:
    """Depth prior = depth x (1 + N(0, sigma)) with a random `hole_frac` of pixels set to 0."""
    noise = rng.normal(0.0, sigma, size=depth.shape)
    holes = rng.uniform(size=depth.shape) < hole_frac
    return np.where(holes, 0.0, depth * (1.0 + noise)).astype(np.float32)


# ----------------------------------------------------------------------------- workloads

TUM_CAM = Cam(525.0, 525.0, 319.5, 239.5, 640, 480)
WIDE_CAM = Cam(600.0, 600.0, 599.5, 339.5, 1200, 680)
QVGA_CAM = Cam(262.5, 262.5, 159.5, 119.5, 320, 240)


def tracking_gt_pose() -> np.ndarray:
    """Ground-truth camera of the 640 x 480 tracking case: at (2.5, 1.5, 0.8) looking at the +z wall."""
    return look_at((2.5, 1.5, 0.8), (0.0, 0.0, 1.0))


def mapping_keyframes(n_views: int = 8) -> list:
    """Keyframes on a 1 m circle at height 1.5 m around the room centre, looking outward,
    with 360 / n_views degrees of yaw between them."""
    X, _, Z = ROOM
    c = np.array([X / 2, 1.5, Z / 2])
    poses = []
    for k in range(n_views):
        yaw = 2.0 * np.pi * k / n_views
        d = np.array([np.sin(yaw), 0.0, np.cos(yaw)])
        poses.append(look_at(c + 1.0 * d, d))
    return poses


def spline_trajectory(n_frames: int, seed: int = 0, n_ctrl: int = 8) -> list:
    """Camera poses along a closed Catmull-Rom spline through `n_ctrl` seeded control
    points that loop once around the room centre (ordered by azimuth, radius 0.7-1.5 m,
    height 0.9-2.1 m, so at least 0.5 m from every wall), each camera looking outward from
    the centre, nearly level: the heading turns about 360 / n_frames degrees per frame."""
    rng = np.random.default_rng(seed + 104729)
    X, Y, Z = ROOM
    centre = np.array([X / 2, 1.5, Z / 2])
    az = np.sort(rng.uniform(0.0, 2 * np.pi, n_ctrl))
    az = (az + np.linspace(0.0, 2 * np.pi, n_ctrl, endpoint=False)) / 2.0  # spread the azimuths
    rad = rng.uniform(0.7, 1.5, n_ctrl)
    ctrl = np.stack([centre[0] + rad * np.sin(az), rng.uniform(0.9, 2.1, n_ctrl), centre[2] + rad * np.cos(az)], 1)
    poses = []
    for f in range(n_frames):
        s = f * n_ctrl / n_frames
        i = int(np.floor(s))
        u = s - i
        p0, p1, p2, p3 = (ctrl[(i + k - 1) % n_ctrl] for k in range(4))
        pos = 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)
        look = pos - centre
        look[1] *= 0.2
        poses.append(look_at(pos, look))
    return poses


def batched_keyframes(n_frames: int = 32, n_hyp: int = 16, seed: int = 0):
    """Keyframes of uneven resolution (uniform over 320 x 240, 640 x 480, 1200 x 680, focal
    length scaled with width) at seeded positions inside the room, each with `n_hyp` pose
    hypotheses: rotation vector N(0, 2 deg) and translation N(0, 4 cm) per axis.  Returns the
    per-view cameras and hypothesis poses, the keyframe of each view, and the keyframes'
    ground-truth poses and cameras."""
    rng = np.random.default_rng(seed + 15485863)
    cams_choice = [QVGA_CAM, TUM_CAM, WIDE_CAM]
    X, Y, Z = ROOM
    cams, poses, frame_of, gts, frame_cams = [], [], [], [], []
    for f in range(n_frames):
        cam = cams_choice[rng.integers(0, 3)]
        pos = np.array([rng.uniform(1.0, X - 1.0), rng.uniform(1.0, Y - 1.0), rng.uniform(1.0, Z - 1.0)])
        yaw = rng.uniform(0.0, 2.0 * np.pi)
        gt = look_at(pos, (np.sin(yaw), rng.uniform(-0.2, 0.2), np.cos(yaw)))
        gts.append(gt)
        frame_cams.append(cam)
        for _ in range(n_hyp):
            cams.append(cam)
            poses.append(jitter_pose(gt, rng, 2.0, 0.04))
            frame_of.append(f)
    return cams, poses, np.array(frame_of), gts, frame_cams
