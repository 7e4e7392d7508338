"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the scaling method: it only draws
coordinates, reference weights and densities.  Both the CUDA path's tests and
the CPU oracle's tests take their inputs from here.

Every generator draws from numpy's Philox counter-based bit generator with an
explicit seed, so a (seed, shape) pair names one input on every machine.

Shapes follow the paper's experiments:
  * 1-D densities on a uniform grid of [0, 1] (Sec. 5.1, 1-D examples);
  * 2-D images of shapes on [0, 1]^2 (Sec. 5.1, 2-D examples);
  * 3-D colour-like point clouds in [0, 1]^3 (Sec. 5.1, colour transfer);
  * batches of 2-D point clouds and stacks of blob images for barycenters
    (Sec. 5.2);
  * initial tumor densities on [0, 1] for the WF gradient flows (Sec. 5.3);
  * colour images in [0, 1]^3 (rescaled Lab-like coordinates) for the colour
    transfer of Sec. 5.1.
The reference measures are the discretised Lebesgue measure (grid) or the
uniform empirical measure (points), both probability vectors (Sec. 4.2).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def grid_axis(n: int) -> np.ndarray:
    """Cell centres (i + 1/2)/n of a uniform grid of [0, 1]."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def gaussian_mixture_1d(g: np.random.Generator, x: np.ndarray, ncomp: int = 3,
                        std=(0.02, 0.1), mean=(0.1, 0.9)) -> np.ndarray:
    """Unnormalised mixture of `ncomp` Gaussian bumps evaluated at x."""
    out = np.zeros_like(x)
    for _ in range(ncomp):
        mu = g.uniform(*mean)
        sd = g.uniform(*std)
        w = g.uniform(0.5, 1.5)
        out += w * np.exp(-0.5 * ((x - mu) / sd) ** 2)
    return out


def normalise_mass(dens: np.ndarray, w: np.ndarray, mass: float) -> np.ndarray:
    """Scale a density so that sum(dens * w) == mass."""
    return dens * (mass / float(np.sum(dens * w)))


def problem_1d(n: int = 256, m: int = 256, seed: int = 1234, masses=(1.0, 1.6)):
    """1-D unbalanced OT inputs: grid points, weights dx, dy and densities p, q."""
    g = rng(seed)
    x = grid_axis(n)
    y = grid_axis(m)
    dx = np.full(n, 1.0 / n)
    dy = np.full(m, 1.0 / m)
    p = normalise_mass(gaussian_mixture_1d(g, x), dx, masses[0])
    q = normalise_mass(gaussian_mixture_1d(g, y), dy, masses[1])
    return dict(x=x, y=y, dx=dx, dy=dy, p=p, q=q)


def shapes_image(g: np.random.Generator, H: int, W: int, nshape=(1, 6),
                 radius=(0.08, 0.25), soft: float = 0.01, floor: float = 0.0) -> np.ndarray:
    """Image of random filled ellipses with soft edges and (by default) an exactly
    zero background, like the shape densities of the paper's 2-D examples."""
    yy, xx = np.meshgrid(grid_axis(H), grid_axis(W), indexing="ij")
    img = np.zeros((H, W))
    k = int(g.integers(nshape[0], nshape[1] + 1))
    for _ in range(k):
        cy, cx = g.uniform(0.2, 0.8, size=2)
        ra, rb = g.uniform(*radius, size=2)
        th = g.uniform(0.0, np.pi)
        c, s = np.cos(th), np.sin(th)
        u = ((xx - cx) * c + (yy - cy) * s) / ra
        v = (-(xx - cx) * s + (yy - cy) * c) / rb
        r = np.sqrt(u * u + v * v)
        # smooth step from 1 inside to exactly 0 outside, width `soft` (relative)
        t = np.clip((1.0 + soft - r) / (2.0 * soft), 0.0, 1.0)
        img += g.uniform(0.5, 1.5) * t * t * (3.0 - 2.0 * t)
    return img + floor


def problem_grid2d(H: int = 256, W: int = 256, seed: int = 1235,
                   masses=(1.0, 1.3), floor: float = 0.0):
    """2-D grid unbalanced OT inputs on [0,1]^2: per-axis coordinates, per-pixel
    weights 1/(H W) and two shape images scaled to the given masses."""
    g = rng(seed)
    dx = np.full((H, W), 1.0 / (H * W))
    p = normalise_mass(shapes_image(g, H, W, floor=floor), dx, masses[0])
    q = normalise_mass(shapes_image(g, H, W, floor=floor), dx, masses[1])
    ax = [grid_axis(H), grid_axis(W)]
    return dict(xs=ax, ys=[a.copy() for a in ax], dx=dx, dy=dx.copy(), p=p, q=q)


def mixture_points(g: np.random.Generator, n: int, d: int, ncomp: int,
                   std=(0.03, 0.1)) -> np.ndarray:
    """n points in [0,1]^d from an equal-weight Gaussian mixture, clipped."""
    means = g.uniform(0.15, 0.85, size=(ncomp, d))
    stds = g.uniform(*std, size=(ncomp, 1))
    comp = g.integers(0, ncomp, size=n)
    pts = means[comp] + stds[comp] * g.standard_normal((n, d))
    return np.clip(pts, 0.0, 1.0)


def problem_points(n: int = 20000, m: int = 20000, d: int = 3, seed: int = 1236,
                   masses=(1.0, 0.7), ncomp: int = 8):
    """Point-cloud inputs: uniform empirical reference weights dx = 1/n, dy = 1/m
    and constant densities equal to the total masses."""
    g = rng(seed)
    x = mixture_points(g, n, d, ncomp)
    y = mixture_points(g, m, d, ncomp)
    return dict(x=x, y=y, dx=np.full(n, 1.0 / n), dy=np.full(m, 1.0 / m),
                p=np.full(n, float(masses[0])), q=np.full(m, float(masses[1])))


def blob_image(g: np.random.Generator, H: int, W: int, nblob=(1, 6)) -> np.ndarray:
    """Sum of 1-6 isotropic Gaussian blobs (always positive, no zero background)."""
    yy, xx = np.meshgrid(grid_axis(H), grid_axis(W), indexing="ij")
    img = np.zeros((H, W))
    for _ in range(int(g.integers(nblob[0], nblob[1] + 1))):
        cy, cx = g.uniform(0.2, 0.8, size=2)
        sd = g.uniform(0.04, 0.12)
        img += g.uniform(0.5, 1.5) * np.exp(-0.5 * ((xx - cx) ** 2 + (yy - cy) ** 2) / sd ** 2)
    return img


def barycenter_images(K: int = 32, H: int = 128, W: int = 128, seed: int = 1237,
                      floor: float = 1e-6):
    """K blob images with unit mass each on [0,1]^2, plus the grid description."""
    g = rng(seed)
    dx = np.full((H, W), 1.0 / (H * W))
    P = np.stack([normalise_mass(blob_image(g, H, W) + floor, dx, 1.0) for _ in range(K)])
    ax = [grid_axis(H), grid_axis(W)]
    return dict(xs=ax, ys=[a.copy() for a in ax], dx=dx, dy=dx.copy(), P=P)


def batch_points(nprob: int = 4096, size=(64, 2048), d: int = 2, seed: int = 1238,
                 mass=(0.5, 2.0), lam=(0.05, 5.0)):
    """Many independent 2-D point-cloud problems of uneven sizes."""
    g = rng(seed)
    probs = []
    for _ in range(nprob):
        n = int(g.integers(size[0], size[1] + 1))
        m = int(g.integers(size[0], size[1] + 1))
        x = mixture_points(g, n, d, int(g.integers(1, 5)))
        y = mixture_points(g, m, d, int(g.integers(1, 5)))
        mp, mq = g.uniform(*mass, size=2)
        lm = float(np.exp(g.uniform(np.log(lam[0]), np.log(lam[1]))))
        probs.append(dict(x=x, y=y, dx=np.full(n, 1.0 / n), dy=np.full(m, 1.0 / m),
                          p=np.full(n, mp), q=np.full(m, mq), lam=lm))
    return probs


def warmstart_instances(n: int, H: int = 64, W: int = 64, seed: int = 1239, group: int = 64,
                        mass=(0.5, 2.0), eps=(1e-3, 1e-1), lam=(0.1, 10.0), floor: float = 1e-6):
    """Instances for the learned warm start: pairs of 1-6 Gaussian-blob images
    with masses uniform in `mass` (plus a relative floor so every density is
    positive), eps and lambda log-uniform.  Consecutive blocks of `group`
    instances share (eps, lambda) so that they can be solved as one batch.
    Returns dict(P [n,H,W], Q [n,H,W], eps [n], lam [n], dx [H,W])."""
    g = rng(seed)
    dx = np.full((H, W), 1.0 / (H * W))
    P = np.empty((n, H, W))
    Q = np.empty((n, H, W))
    E = np.empty(n)
    L = np.empty(n)
    for k in range(n):
        if k % group == 0:
            e = float(np.exp(g.uniform(np.log(eps[0]), np.log(eps[1]))))
            lm = float(np.exp(g.uniform(np.log(lam[0]), np.log(lam[1]))))
        for arr in (P, Q):
            img = blob_image(g, H, W)
            img = img + floor * img.max()
            arr[k] = normalise_mass(img, dx, float(g.uniform(*mass)))
        E[k] = e
        L[k] = lm
    return dict(P=P, Q=Q, eps=E, lam=L, dx=dx, xs=[grid_axis(H), grid_axis(W)])


def tumor_densities(n: int = 3000, species: int = 1, seed: int = 1240):
    """Initial densities of the growth flows (Sec. 5.3): S species on the
    uniform grid of [0, 1] (the paper uses 3000 samples), each a bump of
    height 0.3-0.7 below the cap 1, with a seeded ripple, on a subinterval of
    width 0.1-0.3, exactly 0 elsewhere.  Returns (x, dx, P [S, n])."""
    g = rng(seed)
    x = grid_axis(n)
    P = np.zeros((species, n))
    for k in range(species):
        c0 = g.uniform(0.25, 0.75)
        w = g.uniform(0.05, 0.15)
        amp = g.uniform(0.3, 0.7)
        f = g.uniform(10.0, 40.0)
        P[k] = np.where(np.abs(x - c0) < w, amp * (1.0 + 0.2 * np.sin(f * x)), 0.0)
    return x, np.full(n, 1.0 / n), P


def color_image(H: int = 512, W: int = 512, seed: int = 1241, ncolors: int = 5):
    """A synthetic colour image [H, W, 3] in [0, 1]^3 (float32), colours as
    rescaled Lab-like coordinates (luminance first): a Voronoi partition of
    the image into `ncolors` regions of random palette colours (luminance
    0.15-0.95, chrominance 0.2-0.8), each with a smooth spatial gradient and
    pixel noise, clipped to the cube.  The paper's photographs are not
    available; two such images with different seeds have different palettes."""
    g = rng(seed)
    pal = np.stack([g.uniform(0.15, 0.95, ncolors), g.uniform(0.2, 0.8, ncolors), g.uniform(0.2, 0.8, ncolors)], 1)
    seeds = g.uniform(0, 1, size=(ncolors, 2))
    yy, xx = np.meshgrid((np.arange(H) + 0.5) / H, (np.arange(W) + 0.5) / W, indexing="ij")
    d2 = (yy[..., None] - seeds[:, 0]) ** 2 + (xx[..., None] - seeds[:, 1]) ** 2
    cell = np.argmin(d2, axis=-1)
    grad = g.uniform(-0.15, 0.15, size=(ncolors, 3, 2))
    img = pal[cell] + grad[cell, :, 0] * (yy - 0.5)[..., None] + grad[cell, :, 1] * (xx - 0.5)[..., None]
    img = img + g.normal(0.0, 0.02, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)
