"""Camera cases shared by the oracle pin and the GPU parity test of the camera model."""
import numpy as np

import synth


def gram_schmidt(forward, up, right):
    """The camera model's orthonormalisation, restated here in numpy: forward is normalised first,
    up loses its forward component, right loses its forward and up components (include/canvox.h)."""
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    u = np.asarray(up, dtype=np.float64)
    u = u - (u @ f) * f
    u = u / np.linalg.norm(u)
    r = np.asarray(right, dtype=np.float64)
    r = r - (r @ f) * f - (r @ u) * u
    r = r / np.linalg.norm(r)
    return f, u, r


def skewed_cameras(extent=1.0, offset=0):
    """Cameras whose right/up/forward are not orthonormal: a scaled forward, an up with a forward
    component, a right that is skewed towards forward and up and has the wrong length; one of them
    with a 'right' that points left (the frame keeps its sign: a mirrored image)."""
    cams, ortho = [], []
    rng = np.random.default_rng(404)
    specs = [([1.7, 0.4, -1.1], [0.02, -0.03, 0.01], 3.7, 0.9, (2.2, 0.7, -0.4), 21, 13),
             ([-0.3, 1.9, 0.8], [0.05, 0.0, -0.04], 0.21, -1.3, (0.6, -0.35, 0.8), 17, 17),
             ([0.1, 0.05, -0.2], [0.3, 0.1, 0.4], 1.0, 0.5, (-1.4, 0.2, 0.3), 12, 9)]   # eye inside, right -> left
    for eye, tgt, fs, uf, (rs, rf, ru), w, h in specs:
        eye = np.array(eye) * extent
        f0 = np.array(tgt) * extent - eye
        f0 /= np.linalg.norm(f0)
        r0 = np.cross(f0, [0.0, 1.0, 0.0] + 0.1 * rng.normal(size=3))
        r0 /= np.linalg.norm(r0)
        u0 = np.cross(r0, f0)
        fwd = fs * f0
        up = 0.6 * u0 + uf * f0
        right = rs * r0 + rf * f0 + ru * u0
        bg = (0.1, 0.2, 0.3, 1.0)
        cams.append(synth.camera(eye, right, up, fwd, 0.55, w, h, offset, bg))
        f, u, r = gram_schmidt(fwd, up, right)
        ortho.append(synth.camera(eye, r, u, f, 0.55, w, h, offset, bg))
        offset += w * h
    return synth.cameras_array(cams), synth.cameras_array(ortho)
