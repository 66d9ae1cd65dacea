"""Rate-distortion selection over a bandwidth ladder (the R-D sweep of the
paper's evaluation, Sec. 5, done per frame on the encoder's own numbers).

Each frame is coded at several rungs (quantisation steps); for every rung the
encoder returns the stream size and the sum of squared coefficient errors per
channel (gsnfs_encode_batch_rd), which equals the squared error of the decoded
attributes against the voxel means because RAHT is orthonormal.  From those:

* psnr(): PSNR with peak 1 over all channels (or a channel subset) of a frame;
* rendered_psnr(): PSNR of rendered views of the decoded frame against the
  same views of the original Gaussians (the quality measure of Sec. 5.1),
  for any renderer (gsnfs.render on the GPU);
* upper_hull(): the rungs on the upper convex hull of (bytes, PSNR), i.e. the
  rungs no mixture of two other rungs beats;
* select(): per frame, the hull rung with the highest PSNR whose stream fits a
  byte budget (the smallest rung when none fits).
"""
from __future__ import annotations

import numpy as np


def psnr(sq_err_sum, n_voxels, channels=None, peak=1.0):
    """PSNR (dB) of each (frame, rung) from squared-error sums [F, R, C] and voxel counts [F]."""
    e = np.asarray(sq_err_sum, dtype=np.float64)
    if channels is not None:
        e = e[:, :, channels]
    n = np.asarray(n_voxels, dtype=np.float64).reshape(-1, 1)
    mse = e.sum(2) / np.maximum(n * e.shape[2], 1.0)
    with np.errstate(divide="ignore"):
        return 10.0 * np.log10(peak * peak / np.maximum(mse, 1e-300))


def upper_hull(rate, quality):
    """Indices of the points on the upper convex hull of (rate, quality),
    ascending in rate; among equal rates the best quality is kept."""
    r = np.asarray(rate, dtype=np.float64)
    qv = np.asarray(quality, dtype=np.float64)
    order = sorted(range(r.size), key=lambda i: (r[i], -qv[i]))
    pts = []
    for i in order:
        if pts and r[pts[-1]] == r[i]:
            continue  # same rate, lower quality
        if pts and qv[i] <= qv[pts[-1]]:
            continue  # more bytes for no gain: never on the upper hull
        while len(pts) >= 2:
            a, b = pts[-2], pts[-1]
            # drop b if it lies on or below the segment a -> i
            cross = (r[b] - r[a]) * (qv[i] - qv[a]) - (qv[b] - qv[a]) * (r[i] - r[a])
            if cross >= 0:
                pts.pop()
            else:
                break
        pts.append(i)
    return pts


def select(rate, quality, budget):
    """Per frame (rows of rate / quality [F, R]): the hull rung of highest
    quality with rate <= budget[f] (or the smallest-rate rung if none fits)."""
    rate = np.asarray(rate, dtype=np.float64)
    quality = np.asarray(quality, dtype=np.float64)
    budget = np.broadcast_to(np.asarray(budget, dtype=np.float64), (rate.shape[0],))
    out = np.zeros(rate.shape[0], dtype=np.int64)
    for f in range(rate.shape[0]):
        hull = upper_hull(rate[f], quality[f])
        fit = [i for i in hull if rate[f, i] <= budget[f]]
        out[f] = max(fit, key=lambda i: quality[f, i]) if fit else int(np.argmin(rate[f]))
    return out


def image_psnr(img, ref, peak=1.0):
    """PSNR (dB) of an image against a reference, both clamped to [0, peak]
    (numpy arrays or torch tensors of the same shape)."""
    if hasattr(img, "detach"):
        a = img.detach().clamp(0, peak).double()
        b = ref.detach().clamp(0, peak).double()
        mse = float(((a - b) ** 2).mean())
    else:
        a = np.clip(np.asarray(img, dtype=np.float64), 0, peak)
        b = np.clip(np.asarray(ref, dtype=np.float64), 0, peak)
        mse = float(((a - b) ** 2).mean())
    return float(10.0 * np.log10(peak * peak / max(mse, 1e-300)))


def rendered_psnr(render, original, decoded, views, peak=1.0):
    """Mean over views of image_psnr(render(*decoded, view), render(*original, view));
    original and decoded are (positions, attributes) pairs, render(pos, attr, view) -> image."""
    vals = [image_psnr(render(decoded[0], decoded[1], v), render(original[0], original[1], v), peak) for v in views]
    return float(np.mean(vals))
