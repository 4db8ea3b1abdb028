"""Seeded synthetic frame pairs shaped like the paper's workloads.

The paper measures on MPI-Sintel (1024x436) and KITTI frames; neither dataset is available,
so these generators stand in for them with the same shapes and a known ground-truth flow.
This module holds none of the method's arithmetic: texture synthesis and warping use
scipy's Gaussian filter and linear interpolation routines.  Random numbers come from
numpy's counter-based Philox generator keyed by the seed.

Conventions: images are float32 in [0, 1], shape (H, W) (grayscale) or (3, H, W) (RGB);
flows are float32 (H, W, 2) with (u, v) along (x, y), such that I1(x + U(x)) ~ I0(x).
"""
import math

import numpy as np
from scipy import ndimage

__all__ = ["rng", "translation_pair", "layered_pair", "workload_pairs", "mixed_resolutions"]


def rng(seed):
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _sample(tex, ys, xs):
    """Linear interpolation of `tex` at float coordinates (rows ys, cols xs), edge clamped."""
    return ndimage.map_coordinates(tex, [ys, xs], order=1, mode="nearest")


def _octave_noise(g, h, w, sigmas=(1, 2, 4, 8, 16)):
    """Multi-octave blurred white noise: octaves normalised to unit deviation, weighted by
    sigma^0.5, summed and rescaled to [0, 1]."""
    acc = np.zeros((h, w))
    for s in sigmas:
        o = ndimage.gaussian_filter(g.standard_normal((h, w)), s, mode="reflect", truncate=4.0)
        acc += math.sqrt(s) * o / (o.std() + 1e-12)
    lo, hi = acc.min(), acc.max()
    return (acc - lo) / (hi - lo + 1e-12)


def translation_pair(seed, width=128, height=96, t=(2.3, -1.7), sigma=2.0):
    """White noise blurred with a Gaussian (sigma, truncated at 4 sigma, reflected border),
    rescaled to [0, 1]; frame 1 is frame 0 shifted by t with linear interpolation,
    I1(x) = I0(x - t) (edge clamped).  Ground truth: the constant flow t."""
    g = rng(seed)
    I0 = ndimage.gaussian_filter(g.standard_normal((height, width)), sigma, mode="reflect", truncate=4.0)
    I0 = (I0 - I0.min()) / (I0.max() - I0.min())
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    I1 = _sample(I0, ys - t[1], xs - t[0])
    gt = np.empty((height, width, 2), np.float32)
    gt[..., 0], gt[..., 1] = t[0], t[1]
    return I0.astype(np.float32), I1.astype(np.float32), gt


def layered_pair(seed, width=1024, height=436, n_ellipses=20, max_disp=40.0, channels=1, rotation_deg=0.0,
                 horizontal=False):
    """Layered scene: a multi-octave noise background under `n_ellipses` textured ellipses.

    Motion: background affine about the image centre (|A - I| <= 0.02, translation up to
    max_disp / 4) plus one translation per ellipse (up to max_disp); later ellipses occlude
    earlier ones; an optional global rotation about the centre is composed on top.
    Frame 1 renders every layer at its moved position (painter's order); regions that the
    motion uncovers show the background texture that frame 0 hid, i.e. fresh noise of the
    same spectrum.  Sizes scale with width / 1024.  Ground truth: the motion of the layer
    visible in frame 0.  channels = 3 draws an independent texture per channel over the
    shared geometry.  horizontal = True: a rectified stereo pair, every motion horizontal (the
    vertical components of the affine map, the background translation and the ellipse
    translations are zeroed after the same draws; no rotation), so gt[..., 1] == 0.
    Returns (I0, I1, gt)."""
    g = rng(seed)
    scale = width / 1024.0
    cx, cy = 0.5 * (width - 1), 0.5 * (height - 1)
    E = g.uniform(-0.02, 0.02, size=(2, 2))
    A = np.eye(2) + E
    r_bg, a_bg = (max_disp / 4.0) * math.sqrt(g.uniform()), g.uniform(0, 2 * math.pi)
    t_bg = np.array([r_bg * math.cos(a_bg), r_bg * math.sin(a_bg)])
    if horizontal:
        if rotation_deg:
            raise ValueError("a stereo pair has no rotation")
        E[1] = 0.0
        A = np.eye(2) + E
        t_bg[1] = 0.0
    ell = []
    for _ in range(n_ellipses):
        ax = g.uniform(20, 150) * scale
        bx = g.uniform(20, 150) * scale
        ang = g.uniform(0, math.pi)
        ex, ey = g.uniform(0, width), g.uniform(0, height)
        r, a = max_disp * math.sqrt(g.uniform()), g.uniform(0, 2 * math.pi)
        ell.append((ex, ey, ax, bx, ang, r * math.cos(a), 0.0 if horizontal else r * math.sin(a)))
    th = math.radians(rotation_deg)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Rinv = R.T

    def inside(k, X, Y):
        ex, ey, ax, bx, ang, _, _ = ell[k]
        dx, dy = X - ex, Y - ey
        c, s = math.cos(ang), math.sin(ang)
        p, q = c * dx + s * dy, -s * dx + c * dy
        return (p / ax) ** 2 + (q / bx) ** 2 <= 1.0

    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    # frame-0 layer labels and ground truth (before the global rotation)
    lab0 = np.full((height, width), -1, np.int32)
    for k in range(n_ellipses):
        lab0[inside(k, xs, ys)] = k
    fu = E[0, 0] * (xs - cx) + E[0, 1] * (ys - cy) + t_bg[0]
    fv = E[1, 0] * (xs - cx) + E[1, 1] * (ys - cy) + t_bg[1]
    for k in range(n_ellipses):
        m = lab0 == k
        fu[m], fv[m] = ell[k][5], ell[k][6]
    # compose the global rotation: x -> R (x + f(x) - c) + c
    tx, ty = xs + fu - cx, ys + fv - cy
    gt = np.stack([R[0, 0] * tx + R[0, 1] * ty + cx - xs, R[1, 0] * tx + R[1, 1] * ty + cy - ys], -1)
    # frame-1 sample coordinates in the unrotated scene
    qx = Rinv[0, 0] * (xs - cx) + Rinv[0, 1] * (ys - cy) + cx
    qy = Rinv[1, 0] * (xs - cx) + Rinv[1, 1] * (ys - cy) + cy
    lab1 = np.full((height, width), -1, np.int32)
    for k in range(n_ellipses):
        lab1[inside(k, qx - ell[k][5], qy - ell[k][6])] = k
    Ainv = np.linalg.inv(A)
    bx_ = Ainv[0, 0] * (qx - cx - t_bg[0]) + Ainv[0, 1] * (qy - cy - t_bg[1]) + cx
    by_ = Ainv[1, 0] * (qx - cx - t_bg[0]) + Ainv[1, 1] * (qy - cy - t_bg[1]) + cy
    margin = int(math.ceil(0.02 * 2 * max(width, height) + max_disp / 4.0 + 8 + abs(th) * max(width, height)))
    I0 = np.empty((channels, height, width))
    I1 = np.empty((channels, height, width))
    for c in range(channels):
        bg = _octave_noise(g, height + 2 * margin, width + 2 * margin)
        I0[c] = bg[margin:margin + height, margin:margin + width]
        I1[c] = _sample(bg, by_ + margin, bx_ + margin)
        for k in range(n_ellipses):
            ex, ey, ax, bxx, _, ux, uy = ell[k]
            rad = max(ax, bxx) + 2
            x0, y0 = int(math.floor(ex - rad)), int(math.floor(ey - rad))
            x1, y1 = int(math.ceil(ex + rad)), int(math.ceil(ey + rad))
            tex = _octave_noise(g, y1 - y0 + 1, x1 - x0 + 1)
            m0 = lab0 == k
            if m0.any():
                I0[c][m0] = _sample(tex, ys[m0] - y0, xs[m0] - x0)
            m1 = lab1 == k
            if m1.any():
                I1[c][m1] = _sample(tex, qy[m1] - uy - y0, qx[m1] - ux - x0)
    I0 = np.clip(I0, 0.0, 1.0).astype(np.float32)
    I1 = np.clip(I1, 0.0, 1.0).astype(np.float32)
    if channels == 1:
        I0, I1 = I0[0], I1[0]
    return I0, I1, gt.astype(np.float32)


MIXED_SIZES = ((320, 240), (640, 480), (1024, 436), (1280, 720), (1920, 1080))


def mixed_resolutions(seed, n):
    """n (width, height) pairs drawn uniformly from the mixed-resolution set."""
    g = rng(seed)
    return [MIXED_SIZES[int(i)] for i in g.integers(0, len(MIXED_SIZES), size=n)]


_WORKLOADS = {"translate128x96": (0, 1), "layered1024x436": (1000, 1), "mixed": (2000, 64),
              "layered512x256": (3000, 8), "rgb3840x2160": (4000, 4), "stereo320x240": (5000, 4),
              "stereo1440x960": (6000, 8)}


def workload_pair(name, i, n=None, base_seed=None):
    """Pair i of workload_pairs(name, n, base_seed), generated alone (for parallel generation)."""
    b, dn = _WORKLOADS[name]
    base_seed = b if base_seed is None else base_seed
    n = dn if n is None else n
    s = base_seed + i
    if name == "translate128x96":
        return translation_pair(s)
    if name == "layered1024x436":
        return layered_pair(s)
    if name == "mixed":
        w, h = mixed_resolutions(base_seed, n)[i]
        return layered_pair(s, width=w, height=h, max_disp=0.04 * w)
    if name == "layered512x256":
        return layered_pair(s, width=512, height=256, max_disp=20.0)
    if name == "rgb3840x2160":
        return layered_pair(s, width=3840, height=2160, max_disp=100.0, channels=3, rotation_deg=2.0)
    if name == "stereo320x240":
        return layered_pair(s, width=320, height=240, n_ellipses=8, max_disp=12.0, horizontal=True)
    if name == "stereo1440x960":
        return layered_pair(s, width=1440, height=960, max_disp=96.0, horizontal=True)
    raise KeyError(name)


def workload_pairs(name, n=None, base_seed=None):
    """Seeded pairs of the named workload; seed of pair i = base_seed + i.

    'translate128x96'      : translation_pair, 128x96, t = (2.3, -1.7)
    'layered1024x436'      : layered_pair 1024x436, 20 ellipses, displacements up to 40 px
    'mixed'                : layered_pair at mixed resolutions, displacements 4 % of width
    'layered512x256'       : layered_pair 512x256 (displacements scaled with width)
    'rgb3840x2160'         : layered_pair RGB 3840x2160, 2 degree rotation, up to 200 px total
    'stereo320x240'        : horizontal layered_pair 320x240, 8 ellipses, disparities up to 12 px
    'stereo1440x960'       : horizontal layered_pair 1440x960, disparities up to 96 px (the size
                             and disparity range of half-resolution Middlebury pairs)
    """
    n = _WORKLOADS[name][1] if n is None else n
    return [workload_pair(name, i, n, base_seed) for i in range(n)]
