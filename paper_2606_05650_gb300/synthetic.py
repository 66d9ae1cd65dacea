"""Seeded synthetic frames shaped like the paper's workloads.

The datasets the paper evaluates on (HiFi4G, N3DV, 8i, CMU Panoptic, static
scenes) are not available, so every frame here is generated from a seed:
positions on moving/deforming parametric surfaces, attributes with the
distributions of 3D Gaussian-splat parameters (Sec. 1.1: scale, rotation,
opacity, spherical-harmonic colour; 56 channels at SH degree 3) or of
point-cloud colour (Sec. 5.4).

This module only draws inputs.  It holds none of the codec's arithmetic and
is shared by the CUDA tests, the oracle tests and the benchmark.
"""
from __future__ import annotations

import numpy as np

# channel layout of a 3DGS frame: 3 log-scale, 4 quaternion, 1 opacity logit,
# 3 SH DC, 45 SH AC  (degree 3)
GS_CHANNELS = 56
GS_GROUP_NAMES = ("scale", "rotation", "opacity", "sh_dc", "sh_ac")
GS_BASE_STEPS = np.array([0.05, 0.02, 0.1, 0.05, 0.02], dtype=np.float64)


def gs_channel_groups(C: int = GS_CHANNELS) -> np.ndarray:
    """Group id per channel for the 56-channel layout (5 groups)."""
    if C != GS_CHANNELS:
        raise ValueError("the 3DGS layout has 56 channels")
    g = np.empty(C, dtype=np.uint8)
    g[0:3] = 0
    g[3:7] = 1
    g[7] = 2
    g[8:11] = 3
    g[11:56] = 4
    return g


def gs_attributes(rng: np.random.Generator, n: int) -> np.ndarray:
    """N x 56 float32 attributes with the 3DGS distributions."""
    a = rng.standard_normal((n, GS_CHANNELS), dtype=np.float32)
    a[:, 0:3] = a[:, 0:3] * np.float32(0.5) - np.float32(4.0)      # log-scale N(-4, 0.5)
    q = a[:, 3:7]
    q /= np.maximum(np.sqrt((q * q).sum(1, keepdims=True)), np.float32(1e-12))  # unit quaternion
    a[:, 7] *= np.float32(2.0)                                      # opacity logit N(0, 2)
    a[:, 8:11] *= np.float32(0.5)                                   # SH DC N(0, 0.5)
    a[:, 11:56] *= np.float32(0.05)                                 # SH AC N(0, 0.05)
    return a


def gs_attributes_correlated_sh(rng: np.random.Generator, n: int) -> np.ndarray:
    """N x 56 attributes whose SH colours are correlated like real 3DGS ones:
    each SH function's RGB share a luminance-like component (colour weights
    near grey), AC energy falls with the SH degree, and the AC functions are
    mixed by a fixed random matrix (cross-function correlation).  Other
    channels as in gs_attributes.  For measuring the colour decorrelation."""
    a = gs_attributes(rng, n)
    mix_rng = np.random.default_rng(12345)  # the same mixing for every frame
    mix = mix_rng.normal(0, 1, (15, 15)) * 0.35 + np.eye(15)
    degree = np.array([1] * 3 + [2] * 5 + [3] * 7)
    sig = (0.08 / degree).astype(np.float32)
    lum = (rng.standard_normal((n, 15), dtype=np.float32) * sig) @ mix.T.astype(np.float32)
    w = np.array([0.95, 1.0, 0.9], dtype=np.float32)
    for col in range(3):
        a[:, 11 + 15 * col:26 + 15 * col] = lum * w[col] + rng.standard_normal((n, 15), dtype=np.float32) * \
            (0.15 * sig)
    dc = rng.standard_normal((n, 1), dtype=np.float32) * np.float32(0.5)
    a[:, 8:11] = dc * w + rng.standard_normal((n, 3), dtype=np.float32) * np.float32(0.05)
    return a


def _sphere(rng, n, centre, radius):
    v = rng.normal(size=(n, 3))
    v /= np.maximum(np.linalg.norm(v, axis=1, keepdims=True), 1e-12)
    return centre + radius * v


def _torus(rng, n, centre, R, r, axis_rot):
    u = rng.uniform(0, 2 * np.pi, n)
    w = rng.uniform(0, 2 * np.pi, n)
    p = np.stack([(R + r * np.cos(w)) * np.cos(u), (R + r * np.cos(w)) * np.sin(u), r * np.sin(w)], 1)
    return centre + p @ axis_rot.T


def _random_rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def static_gs_frame(seed: int, n: int = 10_000):
    """Single static 3DGS frame: 70% on the surfaces of 3 random spheres/tori,
    30% uniform in the unit cube; 56 attributes."""
    rng = np.random.default_rng(seed)
    n_surf = int(round(0.7 * n))
    counts = rng.multinomial(n_surf, [1 / 3] * 3)
    parts = []
    for k in range(3):
        centre = rng.uniform(0.25, 0.75, 3)
        if rng.uniform() < 0.5:
            parts.append(_sphere(rng, counts[k], centre, rng.uniform(0.08, 0.22)))
        else:
            R = rng.uniform(0.1, 0.2)
            parts.append(_torus(rng, counts[k], centre, R, rng.uniform(0.02, 0.6 * R), _random_rotation(rng)))
    parts.append(rng.uniform(0.0, 1.0, size=(n - n_surf, 3)))
    pos = np.concatenate(parts, 0).astype(np.float32)
    pos = pos[rng.permutation(n)]
    return pos, gs_attributes(rng, n)


class DynamicScene:
    """Four parametric surfaces (sphere, torus, cylinder, plane patch) with
    rigid motion, a smooth sinusoidal warp and per-frame jitter N(0, 1e-3)."""

    def __init__(self, seed: int):
        rng = np.random.default_rng(seed)
        self.seed = seed
        self.centres = rng.uniform(0.3, 0.7, size=(4, 3))
        self.vel = rng.normal(0, 0.002, size=(4, 3))
        self.rot = [_random_rotation(rng) for _ in range(4)]
        self.omega = rng.normal(0, 0.01, size=4)
        self.warp_k = rng.uniform(4, 12, size=(4, 3))
        self.warp_a = rng.uniform(0.005, 0.02, size=4)
        self.weights = np.array([0.3, 0.3, 0.2, 0.2])

    def _surface(self, rng, s, n, t):
        if s == 0:
            v = rng.normal(size=(n, 3))
            p = 0.15 * v / np.maximum(np.linalg.norm(v, axis=1, keepdims=True), 1e-12)
        elif s == 1:
            u = rng.uniform(0, 2 * np.pi, n)
            w = rng.uniform(0, 2 * np.pi, n)
            p = np.stack([(0.14 + 0.05 * np.cos(w)) * np.cos(u), (0.14 + 0.05 * np.cos(w)) * np.sin(u), 0.05 * np.sin(w)], 1)
        elif s == 2:
            u = rng.uniform(0, 2 * np.pi, n)
            h = rng.uniform(-0.15, 0.15, n)
            p = np.stack([0.07 * np.cos(u), 0.07 * np.sin(u), h], 1)
        else:
            p = np.stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), np.zeros(n)], 1)
        ang = self.omega[s] * t
        c, sn = np.cos(ang), np.sin(ang)
        spin = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
        p = p @ (self.rot[s] @ spin).T
        p = p + self.warp_a[s] * np.sin(self.warp_k[s] * p[:, [1, 2, 0]] + 0.2 * t)
        return p + self.centres[s] + self.vel[s] * t

    def frame(self, t: int, n: int | None = None, n_base: int = 250_000):
        """Frame t: N = n, or n_base +- 10% drawn per frame."""
        rng = np.random.default_rng(self.seed * 1000 + t)
        if n is None:
            n = int(rng.integers(int(0.9 * n_base), int(1.1 * n_base) + 1))
        counts = rng.multinomial(n, self.weights)
        pos = np.concatenate([self._surface(rng, s, counts[s], t) for s in range(4)], 0)
        pos += rng.normal(0, 1e-3, size=pos.shape)
        pos = pos.astype(np.float32)[rng.permutation(n)]
        return pos, gs_attributes(rng, n)


def capsule_humanoids_frame(seed: int, t: int, n: int = 1_000_000):
    """Dynamic point cloud: 2 articulated humanoid-like capsule assemblies,
    RGB from smooth colour fields plus N(0, 4) noise, converted to BT.601
    full-range YCbCr scaled to [0, 1].  Returns (pos, attr[N,3])."""
    rng = np.random.default_rng(seed * 1000 + t)
    # capsule = segment (a, b) with radius r; a figure has 10 capsules
    bones = np.array([
        [0.0, 0.0, 0.9, 0.0, 0.0, 1.45, 0.12],    # torso
        [0.0, 0.0, 1.5, 0.0, 0.0, 1.7, 0.09],     # head
        [0.0, -0.2, 1.4, 0.0, -0.45, 1.1, 0.04],  # upper arm L
        [0.0, -0.45, 1.1, 0.0, -0.55, 0.8, 0.035],
        [0.0, 0.2, 1.4, 0.0, 0.45, 1.1, 0.04],    # upper arm R
        [0.0, 0.45, 1.1, 0.0, 0.55, 0.8, 0.035],
        [0.0, -0.1, 0.9, 0.0, -0.12, 0.45, 0.06],  # thigh L
        [0.0, -0.12, 0.45, 0.0, -0.12, 0.02, 0.05],
        [0.0, 0.1, 0.9, 0.0, 0.12, 0.45, 0.06],
        [0.0, 0.12, 0.45, 0.0, 0.12, 0.02, 0.05],
    ])
    pts = []
    per = rng.multinomial(n, np.full(20, 1 / 20))
    k = 0
    for fig in range(2):
        off = np.array([0.0, -0.5 + 1.0 * fig, 0.0])
        swing = 0.3 * np.sin(0.2 * t + fig)
        for bi, b in enumerate(bones):
            a, e, r = b[0:3].copy(), b[3:6].copy(), b[6]
            if bi >= 2:  # articulate limbs by a swing about the y axis around the joint
                piv = a.copy()
                ang = swing * (1 if bi % 2 == 0 else -1)
                c, s = np.cos(ang), np.sin(ang)
                R = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
                e = piv + R @ (e - piv)
            m = per[k]
            k += 1
            u = rng.uniform(0, 1, m)
            axis = e - a
            L = np.linalg.norm(axis) + 1e-12
            d = axis / L
            tmp = np.array([1.0, 0, 0]) if abs(d[0]) < 0.9 else np.array([0, 1.0, 0])
            e1 = np.cross(d, tmp)
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(d, e1)
            th = rng.uniform(0, 2 * np.pi, m)
            p = a + np.outer(u, axis) + r * (np.outer(np.cos(th), e1) + np.outer(np.sin(th), e2))
            pts.append(p + off)
    pos = np.concatenate(pts, 0)
    pos = (pos - pos.min(0)) / max(float((pos.max(0) - pos.min(0)).max()), 1e-9)
    f = 2 * np.pi
    rgb = np.stack([
        128 + 90 * np.sin(f * 1.3 * pos[:, 0] + 0.5) * np.cos(f * 0.7 * pos[:, 2]),
        128 + 90 * np.sin(f * 0.9 * pos[:, 1] + 1.1),
        128 + 90 * np.cos(f * 1.1 * pos[:, 2] + 0.3 * t),
    ], 1) + rng.normal(0, 4.0, size=(n, 3))
    rgb = np.clip(np.round(rgb), 0, 255)
    R, G, B = rgb[:, 0], rgb[:, 1], rgb[:, 2]
    Y = 0.299 * R + 0.587 * G + 0.114 * B
    Cb = 128 - 0.168736 * R - 0.331264 * G + 0.5 * B
    Cr = 128 + 0.5 * R - 0.418688 * G - 0.081312 * B
    attr = (np.stack([Y, Cb, Cr], 1) / 255.0).astype(np.float32)
    perm = rng.permutation(n)
    return pos.astype(np.float32)[perm], attr[perm]


def ladder_sizes(seed: int, frames: int = 64, lo: int = 50_000, hi: int = 2_000_000):
    """Gaussian counts log-uniform in [lo, hi] and depths 16/17/18 round robin."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), frames)).astype(np.int64)
    J = np.array([16 + (f % 3) for f in range(frames)], dtype=np.int32)
    return n, J


LADDER_RUNG_SCALES = np.array([1.0, 2.0, 4.0, 8.0, 16.0])


def look_at_view(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """3 x 4 world-to-camera [R | t] (FP64) of a pinhole camera at `eye`
    looking at `target`: camera z forward, x right, y down (image rows)."""
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return np.concatenate([R, (-R @ eye)[:, None]], 1)


def orbit_views(k: int, centre=(0.5, 0.5, 0.5), radius: float = 1.6, elevation: float = 0.35):
    """k test views on a circle around `centre` (the stand-in for a scene's
    held-out camera poses)."""
    c = np.asarray(centre, dtype=np.float64)
    out = []
    for i in range(k):
        a = 2 * np.pi * (i + 0.25) / k
        eye = c + radius * np.array([np.cos(a) * np.cos(elevation), np.sin(a) * np.cos(elevation), np.sin(elevation)])
        out.append(look_at_view(eye, c))
    return out
