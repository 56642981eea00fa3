"""Random coefficient fields: correlated log-normal permeability and
rasterised fracture segments on the unit square.

All arrays are (ny, nx) float64, row j holds cells (i, j) for i = 0..nx-1,
cell (i, j) covers [i h, (i+1) h] x [j h, (j+1) h] with h = 1/nx.
"""

import numpy as np


def correlated_lognormal(rng, nx, ny, corr_len, geo_mean, log_std=1.0):
    """k = geo_mean * exp(log_std * g), g a stationary Gaussian field.

    g is white noise convolved (periodically, by FFT) with a Gaussian kernel
    of standard deviation corr_len/2 cells, which gives the covariance
    exp(-r^2 / corr_len^2); it is then shifted and scaled to sample mean 0 and
    sample standard deviation 1.
    """
    w = rng.standard_normal((ny, nx))
    s = corr_len / 2.0
    dx = np.minimum(np.arange(nx), nx - np.arange(nx)).astype(np.float64)
    dy = np.minimum(np.arange(ny), ny - np.arange(ny)).astype(np.float64)
    ker = np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * s * s))
    g = np.fft.irfft2(np.fft.rfft2(w) * np.fft.rfft2(ker), s=(ny, nx))
    g = (g - g.mean()) / g.std()
    return geo_mean * np.exp(log_std * g)


def random_segments(rng, n_min=20, n_max=200, len_min=0.05, len_max=0.5):
    """Draw S ~ U{n_min..n_max} segments: centre U[0,1]^2, length
    U[len_min, len_max], angle U[0, pi). Returns an (S, 4) array of
    (x0, y0, x1, y1) end points, not yet clipped to the domain."""
    S = int(rng.integers(n_min, n_max + 1))
    cx = rng.uniform(0.0, 1.0, S)
    cy = rng.uniform(0.0, 1.0, S)
    ln = rng.uniform(len_min, len_max, S)
    th = rng.uniform(0.0, np.pi, S)
    hx = 0.5 * ln * np.cos(th)
    hy = 0.5 * ln * np.sin(th)
    return np.stack([cx - hx, cy - hy, cx + hx, cy + hy], axis=1)


def _clip_unit_square(x0, y0, x1, y1):
    """Liang-Barsky clip of one segment to [0,1]^2; None if nothing is left."""
    dx, dy = x1 - x0, y1 - y0
    t0, t1 = 0.0, 1.0
    for p, q in ((-dx, x0), (dx, 1.0 - x0), (-dy, y0), (dy, 1.0 - y0)):
        if p == 0.0:
            if q < 0.0:
                return None
            continue
        t = q / p
        if p < 0.0:
            t0 = max(t0, t)
        else:
            t1 = min(t1, t)
        if t0 > t1:
            return None
    return (x0 + t0 * dx, y0 + t0 * dy, x0 + t1 * dx, y0 + t1 * dy)


def segment_lengths(segments, nx, ny):
    """Exact length (in domain units) of the union of segment pieces inside
    each cell: the segments are clipped to the unit square, split at every
    grid line they cross, and each piece is credited to the cell holding its
    midpoint. Overlapping segments add up."""
    h = 1.0 / nx
    out = np.zeros((ny, nx))
    for seg in segments:
        c = _clip_unit_square(*map(float, seg))
        if c is None:
            continue
        x0, y0, x1, y1 = c
        dx, dy = x1 - x0, y1 - y0
        length = np.hypot(dx, dy)
        if length == 0.0:
            continue
        ts = [0.0, 1.0]
        if dx != 0.0:
            lo, hi = sorted((x0, x1))
            lines = np.arange(np.ceil(lo / h), np.floor(hi / h) + 1) * h
            ts.extend(((lines - x0) / dx).tolist())
        if dy != 0.0:
            lo, hi = sorted((y0, y1))
            lines = np.arange(np.ceil(lo / h), np.floor(hi / h) + 1) * h
            ts.extend(((lines - y0) / dy).tolist())
        t = np.unique(np.clip(np.asarray(ts), 0.0, 1.0))
        tm = 0.5 * (t[:-1] + t[1:])
        piece = (t[1:] - t[:-1]) * length
        ci = np.clip(np.floor((x0 + tm * dx) / h).astype(np.int64), 0, nx - 1)
        cj = np.clip(np.floor((y0 + tm * dy) / h).astype(np.int64), 0, ny - 1)
        np.add.at(out, (cj, ci), piece)
    return out
