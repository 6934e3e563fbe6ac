"""Seeded synthetic scalar fields on a regular 3D grid.

This module only *generates inputs*; it holds none of the simplification
method's arithmetic. Both the CUDA path and the CPU oracle take their inputs
from here, so a parity test always compares the two on the same bytes.

Every field is returned as a C-contiguous ``float32`` array of shape
``(Lz, Ly, Lx)``; flattening it gives the vertex order used everywhere in this
project, ``id = x + Lx * (y + Ly * z)``.  Values are computed in float64 and
cast to float32 once at the end.  Grid coordinates are ``x_i = i / (L - 1)``
in the unit cube.  Values are normalised to ``[0, 1]`` (the paper's
experiments normalise every dataset to that interval, Section 5).

The paper's own datasets (Aneurysm, Bonsai, Foot, Dark Sky, ...) are not
available; the generators below stand in for their shape (3D, up to 256^3)
and structure (smooth features plus many small noise pairs, filaments rich in
saddle-saddle pairs).
"""
from __future__ import annotations

import numpy as np


def _coords(shape):
    lz, ly, lx = shape
    z = np.linspace(0.0, 1.0, lz) if lz > 1 else np.zeros(1)
    y = np.linspace(0.0, 1.0, ly) if ly > 1 else np.zeros(1)
    x = np.linspace(0.0, 1.0, lx) if lx > 1 else np.zeros(1)
    return z[:, None, None], y[None, :, None], x[None, None, :]


def _normalise(f):
    lo, hi = float(f.min()), float(f.max())
    if hi > lo:
        f = (f - lo) / (hi - lo)
    else:
        f = np.zeros_like(f)
    return np.ascontiguousarray(f.astype(np.float32))


def gaussian_mixture(shape=(32, 32, 32), n_bumps=8, seed=0, noise_frac=0.05,
                     sigma=(0.05, 0.15), amp=(0.5, 1.0)):
    """Sum of isotropic Gaussians plus i.i.d. uniform noise.

    Draw order from ``numpy.random.default_rng(seed)``: centres (n x 3,
    U[0,1]), sigmas (U[sigma]), amplitudes (U[amp]), then the noise in C order
    (z, y, x), U[0, noise_frac * R) with R the range of the smooth part.
    With the defaults this is the 32^3, 8-bump, 5 %-noise plain-solver case.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_bumps, 3))
    sigmas = rng.uniform(sigma[0], sigma[1], size=n_bumps)
    amps = rng.uniform(amp[0], amp[1], size=n_bumps)
    z, y, x = _coords(shape)
    f = np.zeros(shape, dtype=np.float64)
    for c, s, a in zip(centres, sigmas, amps):
        d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        f += a * np.exp(-d2 / (2.0 * s * s))
    r = float(f.max() - f.min())
    if noise_frac > 0:
        f = f + rng.uniform(0.0, noise_frac * r, size=shape)
    return _normalise(f)


def _perlin_octave(shape, freq, rng, slab=8):
    """Lattice-gradient noise, `freq` cells across the unit cube.

    Per grid point: the 8 surrounding lattice gradients dotted with the
    offsets to their lattice points, blended with the quintic fade weights.
    Evaluated slab by slab in z from per-axis arrays (each value is the same
    sequence of float64 operations as a whole-grid evaluation)."""
    g = rng.normal(size=(freq + 1, freq + 1, freq + 1, 3))
    g /= np.linalg.norm(g, axis=-1, keepdims=True)
    z, y, x = _coords(shape)
    px, py, pz = x * freq, y * freq, z * freq
    ix = np.minimum(np.floor(px).astype(np.int64), freq - 1)
    iy = np.minimum(np.floor(py).astype(np.int64), freq - 1)
    iz = np.minimum(np.floor(pz).astype(np.int64), freq - 1)
    tx, ty, tz = px - ix, py - iy, pz - iz

    def fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    wx, wy, wz = fade(tx), fade(ty), fade(tz)
    side = freq + 1
    gc = [np.ascontiguousarray(g[..., k]).ravel() for k in range(3)]  # g[ix, iy, iz, k] at (ix*side+iy)*side+iz
    out = np.zeros(shape, dtype=np.float64)
    for z0 in range(0, shape[0], slab):
        sl = slice(z0, min(shape[0], z0 + slab))
        o = out[sl]
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    idx = ((ix + cx) * side + (iy + cy)) * side + (iz[sl] + cz)
                    dot = gc[0][idx] * (tx - cx) + gc[1][idx] * (ty - cy) + gc[2][idx] * (tz[sl] - cz)
                    w = (wx if cx else 1 - wx) * (wy if cy else 1 - wy) * (wz[sl] if cz else 1 - wz[sl])
                    o += w * dot
    return out


def gradient_noise(shape, rng, octaves=4, base_freq=4):
    """Fractal lattice-gradient noise: frequency x2 and amplitude x1/2 per octave."""
    out = np.zeros(shape, dtype=np.float64)
    amp = 1.0
    for o in range(octaves):
        out += amp * _perlin_octave(shape, base_freq * (2 ** o), rng)
        amp *= 0.5
    return out


def _seg_dist(p, a, b):
    ab = b - a
    ab2 = np.maximum((ab * ab).sum(-1), 1e-30)
    ap = p[:, None, :] - a[None]
    t = np.clip((ap * ab[None]).sum(-1) / ab2[None], 0.0, 1.0)
    d = ap - t[..., None] * ab[None]
    return np.sqrt((d * d).sum(-1))


def _segment_min_dist(points, a, b, shape, block=8):
    """min over segments [a_k, b_k] of the Euclidean distance, per grid point.

    Exact: for each block of voxels, a segment is skipped only when a lower
    bound of its distance to the block exceeds an upper bound of another
    segment's distance to every voxel of the block."""
    lz, ly, lx = shape
    out = np.empty(points.shape[0], dtype=np.float64)
    lo_s = np.minimum(a, b)
    hi_s = np.maximum(a, b)
    idx = np.arange(points.shape[0]).reshape(shape)
    for z0 in range(0, lz, block):
        for y0 in range(0, ly, block):
            for x0 in range(0, lx, block):
                ids = idx[z0:z0 + block, y0:y0 + block, x0:x0 + block].ravel()
                p = points[ids]
                bmin, bmax = p.min(0), p.max(0)
                centre = 0.5 * (bmin + bmax)
                half = 0.5 * float(np.linalg.norm(bmax - bmin))
                gap = np.maximum(0.0, np.maximum(lo_s - bmax[None], bmin[None] - hi_s))
                lb = np.sqrt((gap * gap).sum(-1))
                ub = _seg_dist(centre[None], a, b)[0] + half
                keep = lb <= ub.min()
                out[ids] = _seg_dist(p, a[keep], b[keep]).min(-1)
    return out


def _blur_axis(f, axis, w):
    r = (len(w) - 1) // 2
    n = f.shape[axis]
    idx = np.arange(n)
    out = np.zeros_like(f)
    for k in range(-r, r + 1):
        src = np.clip(idx + k, 0, n - 1)
        out += w[k + r] * np.take(f, src, axis=axis)
    return out


def filament_field(shape=(128, 128, 128), seed=1, n_loops=64, n_seg=8,
                   tube_radius=0.02, noise_amp=0.1, blur_sigma=1.0):
    """Negative distance to closed piecewise-linear tube loops, blurred, plus noise.

    f = -(min over loops of dist - tube_radius), Gaussian-blurred with
    sigma = `blur_sigma` voxels (radius 3, clamped edges), plus 4-octave
    lattice-gradient noise scaled to `noise_amp` x the blurred range.  Many
    tubes close into loops, which makes the field rich in saddle-saddle pairs.

    Draw order: loop centres (U[0.15,0.85]^3), loop radii (U[0.04,0.15]),
    loop normals (N(0,1)^3), angular jitter, radial jitter, out-of-plane
    wobble (each n_loops x n_seg, U[-1,1]), then the noise lattices.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.15, 0.85, size=(n_loops, 3))
    radii = rng.uniform(0.04, 0.15, size=n_loops)
    normals = rng.normal(size=(n_loops, 3))
    ang_j = rng.uniform(-1, 1, size=(n_loops, n_seg))
    rad_j = rng.uniform(-1, 1, size=(n_loops, n_seg))
    wob = rng.uniform(-1, 1, size=(n_loops, n_seg))
    a_list, b_list = [], []
    for i in range(n_loops):
        n = normals[i] / np.linalg.norm(normals[i])
        helper = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        u = np.cross(n, helper)
        u /= np.linalg.norm(u)
        w = np.cross(n, u)
        th = 2 * np.pi * (np.arange(n_seg) + 0.25 * ang_j[i]) / n_seg
        rr = radii[i] * (1.0 + 0.3 * rad_j[i])
        pts = (centres[i][None] + rr[:, None] * (np.cos(th)[:, None] * u[None] + np.sin(th)[:, None] * w[None])
               + (0.2 * radii[i] * wob[i])[:, None] * n[None])
        a_list.append(pts)
        b_list.append(np.roll(pts, -1, axis=0))
    a = np.concatenate(a_list)
    b = np.concatenate(b_list)
    z, y, x = _coords(shape)
    pts = np.stack(np.broadcast_arrays(x, y, z), axis=-1).reshape(-1, 3)
    dist = _segment_min_dist(pts, a, b, shape).reshape(shape)
    f = -(dist - tube_radius)
    k = np.arange(-3, 4)
    wk = np.exp(-0.5 * (k / blur_sigma) ** 2)
    wk /= wk.sum()
    for ax in range(3):
        f = _blur_axis(f, ax, wk)
    r = float(f.max() - f.min())
    nz = gradient_noise(shape, rng)
    nr = float(nz.max() - nz.min())
    if nr > 0:
        f = f + nz * (noise_amp * r / nr)
    return _normalise(f)


def random_field(shape, seed=0, kind="uniform"):
    """Small adversarial fields for parity tests.

    kind = "uniform": i.i.d. U[0,1); "ties": values drawn from {0, 1, 2} so the
    vertex-id tie-break decides most comparisons; "signed_zero": values from
    {-0.0, +0.0, 1.0} (both zeros must compare equal); "normal": N(0,1).
    """
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        f = rng.uniform(0.0, 1.0, size=shape)
    elif kind == "ties":
        f = rng.integers(0, 3, size=shape).astype(np.float64)
    elif kind == "signed_zero":
        c = rng.integers(0, 3, size=shape)
        f = np.where(c == 0, -0.0, np.where(c == 1, 0.0, 1.0))
    elif kind == "normal":
        f = rng.normal(size=shape)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(f.astype(np.float32))


def linear_field(shape, coeffs=(1.0, 2.1, 4.3)):
    """A generic linear function a*x + b*y + c*z on grid coordinates."""
    z, y, x = _coords(shape)
    f = coeffs[0] * x + coeffs[1] * y + coeffs[2] * z
    return np.ascontiguousarray(np.broadcast_to(f, shape).astype(np.float32))


def gaussian_bumps(shape, centres, sigmas, amps, base=None):
    """Deterministic sum of Gaussians (amplitudes may be negative for wells)."""
    z, y, x = _coords(shape)
    f = np.zeros(shape, dtype=np.float64) if base is None else np.array(base, dtype=np.float64)
    for c, s, a in zip(centres, sigmas, amps):
        d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        f = f + a * np.exp(-d2 / (2.0 * s * s))
    return np.ascontiguousarray(f.astype(np.float32))


def ring_distance(shape, centre=(0.5, 0.5, 0.5), radius=0.3):
    """Distance to a circle of `radius` in the plane z = centre_z (a torus field)."""
    z, y, x = _coords(shape)
    dx, dy, dz = x - centre[0], y - centre[1], z - centre[2]
    rho = np.sqrt(dx * dx + dy * dy)
    f = np.sqrt((rho - radius) ** 2 + dz * dz)
    return np.ascontiguousarray(np.broadcast_to(f, shape).astype(np.float32))


# Named workloads, by what they are.
def plain_32(seed=0):
    """32^3 Gaussian mixture (8 bumps) + 5 % uniform noise."""
    return gaussian_mixture((32, 32, 32), n_bumps=8, seed=seed, noise_frac=0.05)


def mixture_96(seed=3):
    """96^3 Gaussian mixture (32 bumps) + 5 % uniform noise: the field of the
    differentiable-loss workload."""
    return gaussian_mixture((96, 96, 96), n_bumps=32, seed=seed, noise_frac=0.05)


def filament_128(seed=1):
    """128^3 filament-tube field + 4-octave gradient noise at 10 % of range."""
    return filament_field((128, 128, 128), seed=seed)


def uneven_batch_shapes(n=48, seed=2, dims=(48, 64, 96, 128, 160)):
    """Shapes (Lz, Ly, Lx) of n independent fields, each axis drawn from
    dims (anisotropic grids allowed), a per-field signal threshold
    U[0.02, 0.2] (fraction of range), and a per-field generator seed."""
    rng = np.random.default_rng(seed)
    shapes = rng.choice(np.asarray(dims), size=(n, 3))
    thresholds = rng.uniform(0.02, 0.2, size=n).astype(np.float32)
    seeds = rng.integers(0, 2 ** 31 - 1, size=n)
    return [tuple(int(d) for d in s) for s in shapes], thresholds, [int(s) for s in seeds]


def uneven_batch(n=48, seed=2, dims=(48, 64, 96, 128, 160)):
    """n independent fields of the shapes above, each a 16-bump Gaussian
    mixture + 5 % uniform noise.  Returns (fields, thresholds)."""
    shapes, thresholds, seeds = uneven_batch_shapes(n, seed, dims)
    fields = [gaussian_mixture(s, n_bumps=16, seed=k, noise_frac=0.05) for s, k in zip(shapes, seeds)]
    return fields, thresholds


# Learned warm start (not in the paper): training inputs and the large
# evaluation field.
def warm_start_inputs(n, seed=4, shape=(64, 64, 64)):
    """n training inputs (field, threshold fraction), alternating the two
    benchmark generators at `shape`: a Gaussian mixture (8 bumps + 5 %
    uniform noise, threshold 0.1) and a filament field (shape[0] // 8
    loops, threshold 0.05), each with its own seed drawn from `seed`.
    The matching targets g are the solver's simplified fields."""
    return [warm_start_input(i, n, seed, shape) for i in range(n)]


def warm_start_input(i, n, seed=4, shape=(64, 64, 64)):
    """The i-th of warm_start_inputs(n, seed, shape), generated alone."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(0, 2 ** 31 - 1, size=n)[i])
    if i % 2 == 0:
        return gaussian_mixture(shape, n_bumps=8, seed=k, noise_frac=0.05), 0.1
    return filament_field(shape, seed=k, n_loops=max(shape[0] // 8, 1)), 0.05


def warm_start_field(shape=(256, 256, 256), seed=5):
    """Evaluation field of the warm start: the mean of a 64-bump Gaussian
    mixture and a 64-loop filament field (each normalised, the mixture
    without noise, the filament field with its gradient noise), plus
    U[0, 0.05) uniform noise, normalised; threshold 0.05."""
    rng = np.random.default_rng(seed)
    s1, s2, s3 = (int(x) for x in rng.integers(0, 2 ** 31 - 1, size=3))
    g = gaussian_mixture(shape, n_bumps=64, seed=s1, noise_frac=0.0).astype(np.float64)
    fl = filament_field(shape, seed=s2, n_loops=64).astype(np.float64)
    f = 0.5 * (g + fl)
    f = f + np.random.default_rng(s3).uniform(0.0, 0.05, size=shape)
    return _normalise(f)
