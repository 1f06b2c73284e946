"""The five synthetic workloads (seeded stroke-built canvases and their cameras).

Seeds are 170402724 + config id. Each recipe draws its stamp table from one
SplitMix64 stream in a fixed order. Lengths are in canvas units: the cube side
for config 0, metres for configs 1-4. Extinction sigma is per canvas unit.

  c0  depth 8, unit cube, 1,000 spheres, r U[2,20] finest cells, sigma U[0.5,20];
      one 256x256 camera, 60 deg, outside the cube, looking at the centre; black background.
  c1  depth 16, 1 km cube, 100,000 spheres, r log-U[1 finest cell, 50 m];
      70 % sigma U[0.5,20]/m, 30 % sigma log-U[200,2000]/m (near-opaque);
      one 1920x1080 camera, 60 deg, inside the cube, looking at the centre, from the point of a 4 m grid
      nearest (230, 110, -310) m that is 1 m clear of every sphere (the nominal point is inside paint).
  c2  depth 24, 40 km canvas (finest 2.4 mm): 10,000 background spheres r log-U[100 m, 1 km]
      (c1 extinction recipe, kept 10 m clear of the rooms) plus 200,000 fine spheres r log-U[2.4 mm, 10 cm]
      in four 1 m room boxes, extinction from an optical thickness 2 r sigma log-U[0.002, 0.2];
      stereo pair 2160x2160 per eye, 90 deg, eye separation 64 mm, head inside room 0.
  c3  depth 27, 40 km canvas (finest 0.3 mm): recipe of c2 with 1,000,000 fine spheres r log-U[0.3 mm, 10 cm];
      8 stereo pairs (4 rooms x scales 1 and 0.01). With ten cells per brush radius each fine sphere adds
      about 3,000 leaves at depth 27: about 3.1e9 leaves and 4.6e8 records, so leaf numbers pass 2^31
      (the pool format stores them modulo 2^31).
  c4  the c3 canvas; 64 views, square side log-U[256, 2160], camera scale log-U[1 mm, 10 km].
"""
import math

import numpy as np

from . import Rng, log_uniform, stamp_canvas, look_at_camera, cameras_array

SEED_BASE = 170402724

CONFIGS = {
    0: dict(name="c0_depth8_unit_cube_256sq", depth=8, extent=1.0),
    1: dict(name="c1_depth16_1km_1080p", depth=16, extent=1000.0),
    2: dict(name="c2_depth24_40km_stereo2160", depth=24, extent=40000.0),
    3: dict(name="c3_depth27_40km_1M_fine_stamps_8stereo2160", depth=27, extent=40000.0),
    4: dict(name="c4_depth27_40km_1M_fine_stamps_64views", depth=27, extent=40000.0),
}

ROOM_SIZE = 1.0
SKY = (0.25, 0.35, 0.5, 1.0)


def _c0_stamps(rng, n=1000):
    E = 1.0
    U = rng.uniform(n * 8).reshape(n, 8)
    centers = -0.5 * E + U[:, 0:3] * E
    radii = (2.0 + 18.0 * U[:, 3]) * (E / 256.0)
    rgba = np.empty((n, 4), dtype=np.float32)
    rgba[:, 0:3] = U[:, 4:7]
    rgba[:, 3] = 0.5 + 19.5 * U[:, 7]
    return centers, radii, rgba


def _c1_sigma(U_flag, U_val):
    opaque = U_flag < 0.3
    return np.where(opaque, log_uniform(200.0, 2000.0, U_val), 0.5 + 19.5 * U_val)


def _c1_stamps(rng, n=100_000):
    E, D = 1000.0, 16
    U = rng.uniform(n * 9).reshape(n, 9)
    centers = -0.5 * E + U[:, 0:3] * E
    radii = log_uniform(E / 2.0 ** D, 50.0, U[:, 3])
    rgba = np.empty((n, 4), dtype=np.float32)
    rgba[:, 0:3] = U[:, 4:7]
    rgba[:, 3] = _c1_sigma(U[:, 7], U[:, 8])
    return centers, radii, rgba


def _rooms(rng, n_rooms=4):
    """Room boxes [p, p + 1 m]^3 with p uniform in the central 2 km."""
    U = rng.uniform(n_rooms * 3).reshape(n_rooms, 3)
    return -1000.0 + U * (2000.0 - ROOM_SIZE)


def _box_dist(p, lo, hi):
    d = np.maximum(np.maximum(lo - p, 0.0), p - hi)
    return math.sqrt(float(np.sum(d * d)))


def _deep_stamps(rng, E, D, n_bg, n_fine, r_fine_min):
    rooms = _rooms(rng)
    # background spheres, redrawn while within 10 m of a room
    bc, br, bq = [], [], []
    while len(br) < n_bg:
        u = rng.uniform(9)
        c = -0.5 * E + u[0:3] * E
        r = float(log_uniform(100.0, 1000.0, u[3:4])[0])
        if any(_box_dist(c, p, p + ROOM_SIZE) < r + 10.0 for p in rooms):
            continue
        bc.append(c)
        br.append(r)
        bq.append([u[4], u[5], u[6], float(_c1_sigma(u[7:8], u[8:9])[0])])
    # fine spheres, an equal share per room, extinction from optical thickness
    per = n_fine // len(rooms)
    fc, fr, fq = [], [], []
    for p in rooms:
        U = rng.uniform(per * 8).reshape(per, 8)
        fc.append(p + U[:, 0:3] * ROOM_SIZE)
        r = log_uniform(r_fine_min, 0.1, U[:, 3])
        fr.append(r)
        q = np.empty((per, 4))
        q[:, 0:3] = U[:, 4:7]
        q[:, 3] = log_uniform(0.002, 0.2, U[:, 7]) / (2.0 * r)
        fq.append(q)
    centers = np.concatenate([np.array(bc).reshape(-1, 3)] + fc)
    radii = np.concatenate([np.array(br)] + fr)
    rgba = np.concatenate([np.array(bq).reshape(-1, 4)] + fq).astype(np.float32)
    return centers, radii, rgba, rooms


def config_stamps(cid, n_fine=None):
    """The stamp table of a config: (depth, extent, centres [n,3], radii [n], rgba [n,4] FP32, rooms or None)."""
    cfg = CONFIGS[cid]
    rng = Rng(SEED_BASE + cid)
    E, D = cfg["extent"], cfg["depth"]
    rooms = None
    if cid == 0:
        c, r, q = _c0_stamps(rng)
    elif cid == 1:
        c, r, q = _c1_stamps(rng)
    elif cid == 2:
        c, r, q, rooms = _deep_stamps(rng, E, D, 10_000, n_fine or 200_000, E / 2.0 ** D)
    elif cid in (3, 4):
        rng = Rng(SEED_BASE + 3)
        c, r, q, rooms = _deep_stamps(rng, E, D, 10_000, n_fine or 1_000_000, E / 2.0 ** D)
    else:
        raise KeyError(cid)
    return D, E, np.ascontiguousarray(c, dtype=np.float64), np.ascontiguousarray(r, dtype=np.float64), \
        np.ascontiguousarray(q, dtype=np.float32), rooms


def build_config(cid, n_fine=None):
    """Build the canvas of a config. n_fine overrides the fine stamp count (c2-c4) for reduced variants."""
    cfg = CONFIGS[cid]
    D, E, c, r, q, rooms = config_stamps(cid, n_fine)
    cv = stamp_canvas(D, E, c, r, q)
    cv.info["config"] = cfg["name"]
    if rooms is not None:
        cv.info["rooms"] = rooms
    return cv


def _rooms_only(cid):
    rng = Rng(SEED_BASE + (3 if cid in (3, 4) else cid))
    return _rooms(rng)


def _stereo_pair(head, yaw, pitch, scale, side, offset, bg):
    f = np.array([math.cos(pitch) * math.sin(yaw), math.sin(pitch), math.cos(pitch) * math.cos(yaw)])
    r = np.cross(f, [0.0, 1.0, 0.0])
    r /= np.linalg.norm(r)
    ipd = 0.064 * scale
    cams = []
    for k, s in enumerate((-0.5, 0.5)):
        eye = head + s * ipd * r
        cams.append(look_at_camera(eye, eye + f, [0.0, 1.0, 0.0], 1.0, side, side, offset + k * side * side, bg))
    return cams


def _clear_eye(eye, centers, radii, spacing=4.0, reach=60.0, clearance=1.0):
    """The point of a grid (spacing, within reach of eye per axis) nearest eye that is at least clearance away
    from every stamp sphere, so that the view does not start inside paint (ties: first in grid order)."""
    g = np.arange(-reach, reach + spacing / 2, spacing)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    P = eye + np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    order = np.argsort(np.linalg.norm(P - eye, axis=1), kind="stable")
    for p in P[order]:
        if np.min(np.linalg.norm(centers - p, axis=1) - radii) > clearance:
            return p
    raise ValueError("no clear eye position near the nominal one")


def config_cameras(cid, res_scale=1.0):
    """Camera records of a config. res_scale shrinks every image side (parity-test variants)."""
    def px(n):
        return max(1, int(round(n * res_scale)))

    if cid == 0:
        d = np.array([1.0, 0.7, 1.9])
        eye = 2.5 * d / np.linalg.norm(d)
        return cameras_array([look_at_camera(eye, [0, 0, 0], [0, 1, 0], math.tan(math.radians(30)), px(256), px(256))])
    if cid == 1:
        eye = _clear_eye(np.array([0.23, 0.11, -0.31]) * 1000.0, *config_stamps(1)[2:4])
        return cameras_array([look_at_camera(eye, [0, 0, 0], [0, 1, 0], math.tan(math.radians(30)),
                                             px(1920), px(1080), 0, SKY)])
    rng = Rng(SEED_BASE + 1000 + cid)
    rooms = _rooms_only(cid)
    if cid == 2:
        u = rng.uniform(5)
        head = rooms[0] + 0.5 * ROOM_SIZE + (u[0:3] - 0.5) * 0.2
        return cameras_array(_stereo_pair(head, 2 * math.pi * u[3], (u[4] - 0.5) * 0.6, 1.0, px(2160), 0, SKY))
    if cid == 3:
        cams = []
        off = 0
        for ri in range(4):
            for scale in (1.0, 0.01):
                u = rng.uniform(5)
                head = rooms[ri] + 0.5 * ROOM_SIZE + (u[0:3] - 0.5) * 0.2 * scale
                pair = _stereo_pair(head, 2 * math.pi * u[3], (u[4] - 0.5) * 0.6, scale, px(2160), off, SKY)
                off += 2 * px(2160) ** 2
                cams += pair
        return cameras_array(cams)
    if cid == 4:
        cams = []
        off = 0
        for v in range(64):
            u = rng.uniform(7)
            side = px(float(log_uniform(256.0, 2160.0, u[0:1])[0]))
            scale = float(log_uniform(1e-3, 1e4, u[1:2])[0])
            ri = v % 4
            # head placed at distance 0.2 x scale from the room centre, looking back at it
            dirv = u[2:5] - 0.5
            dirv /= np.linalg.norm(dirv)
            head = rooms[ri] + 0.5 * ROOM_SIZE + dirv * 0.2 * scale
            yaw = math.atan2(-dirv[0], -dirv[2]) + (u[5] - 0.5) * 0.4
            pitch = math.asin(max(-0.9, min(0.9, -dirv[1]))) + (u[6] - 0.5) * 0.2
            f = np.array([math.cos(pitch) * math.sin(yaw), math.sin(pitch), math.cos(pitch) * math.cos(yaw)])
            cams.append(look_at_camera(head, head + f, [0.0, 1.0, 0.0], 1.0, side, side, off, SKY))
            off += side * side
        return cameras_array(cams)
    raise KeyError(cid)
