"""Seeded image-shaped measures standing in for the paper's datasets.

The paper's experiments (Section 6) use MNIST digits, nested ellipses, the
d2_kmeans clusters and letter images, none of which ship with this project.
The generators below draw synthetic images with the same structure: measures
on a K x K pixel grid, sparse supports where zero pixels are dropped, nested
elliptical rings (Section 6.1, Table 1), smooth Gaussian mixtures, stroke
images, and, for the unbalanced case (Section 6.4), measures whose total
masses differ.

Conventions shared by every generator
-------------------------------------
* Pixel (i, j) of a K x K image sits at ((i / (K-1), j / (K-1)) in [0,1]^2
  and has flat index r = i*K + j (row-major).
* A measure is returned UNPRUNED: its support is the full pixel grid and
  its weights q are the pixel values, zeros included.  Dropping zero-weight
  columns is part of the method (Section 4.3, "Storage complexity") and is
  done by each consumer on its own.
* Problem i of workload j draws from ``numpy.random.default_rng(1000*j + i)``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
from scipy import ndimage


@dataclasses.dataclass
class Problem:
    """One fixed-support barycenter problem (the data of eq. HugeLP / UWB)."""

    name: str
    xi: np.ndarray                 # (R, dim) barycenter support points
    zeta: List[np.ndarray]         # M arrays (S_m, dim), unpruned supports
    q: List[np.ndarray]            # M arrays (S_m,), weights (zeros allowed)
    alpha: np.ndarray              # (M,) measure weights alpha_m
    rho: float = 100.0             # prox parameter of eq. DR
    gamma: float = float("inf")    # unbalanced penalty (inf = balanced)
    n_bundles: int = 1             # Remark 2 partition size (1 = deterministic)
    iters: int = 100
    K: Optional[int] = None        # image side when the support is a grid
    cost: Optional[List[np.ndarray]] = None  # optional (S_m, R) general costs
    target: Optional[np.ndarray] = None      # (R,) target image (loss)

    @property
    def M(self) -> int:
        return len(self.q)

    @property
    def R(self) -> int:
        return int(self.xi.shape[0])

    @property
    def dim(self) -> int:
        return int(self.xi.shape[1])


def grid_points(K: int) -> np.ndarray:
    """(K*K, 2) coordinates of a K x K pixel grid on [0,1]^2, row-major."""
    i, j = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    den = max(K - 1, 1)
    return np.stack([i.ravel() / den, j.ravel() / den], axis=1).astype(np.float64)


def problem_from_images(name, images, alpha=None, masses=None, **kw) -> Problem:
    """Wrap K x K images as measures on the full pixel grid."""
    K = images[0].shape[0]
    xi = grid_points(K)
    q = []
    for m, img in enumerate(images):
        v = np.asarray(img, dtype=np.float64).ravel().copy()
        v[v < 0] = 0.0
        tot = v.sum()
        mass = 1.0 if masses is None else float(masses[m])
        q.append(v * (mass / tot))
    M = len(images)
    if alpha is None:
        alpha = np.full(M, 1.0 / M)
    return Problem(name=name, xi=xi, zeta=[xi.copy() for _ in range(M)], q=q,
                   alpha=np.asarray(alpha, dtype=np.float64), K=K, **kw)


# ---------------------------------------------------------------- images

def _pixel_coords(K):
    return np.meshgrid(np.arange(K, dtype=np.float64),
                       np.arange(K, dtype=np.float64), indexing="ij")


def gaussian_blobs_image(rng, K, n_blobs, centre_lo, centre_hi, sig_lo, sig_hi,
                         amp_lo=0.5, amp_hi=1.0, zero_below=0.01):
    """Sum of isotropic Gaussian blobs; pixels below zero_below*max set to 0."""
    I, J = _pixel_coords(K)
    img = np.zeros((K, K))
    for _ in range(n_blobs):
        ci, cj = rng.uniform(centre_lo, centre_hi, size=2)
        s = rng.uniform(sig_lo, sig_hi)
        a = rng.uniform(amp_lo, amp_hi)
        img += a * np.exp(-((I - ci) ** 2 + (J - cj) ** 2) / (2 * s * s))
    img[img < zero_below * img.max()] = 0.0
    return img


def nested_ellipses_image(rng, K=60, s_range=(600, 1500), width=(2.0, 6.0),
                          max_tries=10000):
    """2-3 concentric elliptical rings, uniform intensity.

    A pixel is on when its distance to a ring, measured along the ray from the
    shared centre, is below half the ring width; the width is drawn once per
    image from U[width].  Images are redrawn until the number of nonzero
    pixels falls in s_range (the shape of the paper's nested-ellipse data,
    Section 6.1).  On a 60x60 grid rings 2 px wide hold at most about 700
    pixels, so the width range reaches up to 6 px for the supports to span
    s_range.
    """
    I, J = _pixel_coords(K)
    for _ in range(max_tries):
        n_rings = int(rng.integers(2, 4))
        ci, cj = rng.uniform(22, 38, size=2)
        a, b = rng.uniform(14, 28, size=2)
        phi = rng.uniform(0, np.pi)
        half = 0.5 * rng.uniform(*width)
        x, y = I - ci, J - cj
        u = np.cos(phi) * x + np.sin(phi) * y
        v = -np.sin(phi) * x + np.cos(phi) * y
        rad = np.hypot(u, v)
        ang = np.arctan2(v, u)
        img = np.zeros((K, K))
        for scale in (1.0, 0.72, 0.45)[:n_rings]:
            aa, bb = a * scale, b * scale
            r_ell = aa * bb / np.sqrt((bb * np.cos(ang)) ** 2 + (aa * np.sin(ang)) ** 2)
            img[np.abs(rad - r_ell) < half] = 1.0
        s = int((img > 0).sum())
        if s_range[0] <= s <= s_range[1]:
            return img
    raise RuntimeError("nested_ellipses_image: no draw met the support range")


def bezier_strokes_image(rng, K=28, s_range=(80, 250), max_tries=10000):
    """3-6 cubic Bezier strokes, 1.5 px wide, blurred (sigma 0.7 px)."""
    t = np.linspace(0.0, 1.0, 200)[:, None]
    for _ in range(max_tries):
        img = np.zeros((K, K))
        for _s in range(int(rng.integers(3, 7))):
            P = rng.uniform(3, 24, size=(4, 2))
            pts = ((1 - t) ** 3 * P[0] + 3 * (1 - t) ** 2 * t * P[1]
                   + 3 * (1 - t) * t ** 2 * P[2] + t ** 3 * P[3])
            # every pixel within 0.75 px of some sample point of the curve; a
            # pixel that close is one of the 4 around the point
            i0 = np.floor(pts[:, 0]).astype(np.int64)
            j0 = np.floor(pts[:, 1]).astype(np.int64)
            for di in (0, 1):
                for dj in (0, 1):
                    ii, jj = i0 + di, j0 + dj
                    ok = (ii - pts[:, 0]) ** 2 + (jj - pts[:, 1]) ** 2 <= 0.75 ** 2
                    img[ii[ok], jj[ok]] = 1.0
        img = ndimage.gaussian_filter(img, 0.7)
        img[img < 0.01 * img.max()] = 0.0
        s = int((img > 0).sum())
        if s_range[0] <= s <= s_range[1]:
            return img
    raise RuntimeError("bezier_strokes_image: no draw met the support range")


def gaussian_mixture_image(rng, K, n_lo, n_hi, centre_lo, centre_hi, sig_lo,
                           sig_hi, zero_below=1e-6):
    """Mixture of n ~ U{n_lo..n_hi} Gaussians with weights U[0.5, 1]."""
    n = int(rng.integers(n_lo, n_hi + 1))
    return gaussian_blobs_image(rng, K, n, centre_lo, centre_hi, sig_lo, sig_hi,
                                0.5, 1.0, zero_below)


def keep_largest(img, S):
    """Zero every pixel but the S largest ones."""
    flat = img.ravel().copy()
    if S < flat.size:
        cut = np.argpartition(-flat, S - 1)[:S]
        keep = np.zeros_like(flat, dtype=bool)
        keep[cut] = True
        flat[~keep] = 0.0
    return flat.reshape(img.shape)


# ---------------------------------------------------------------- workloads

def tiny_problem(seed, M=3, K=3, density=0.7, rho=5.0, gamma=float("inf"),
                 masses=None, n_bundles=1, alpha=None) -> Problem:
    """A small random problem on a K x K grid (for exact LP checks)."""
    rng = np.random.default_rng(seed)
    imgs = []
    for _ in range(M):
        v = rng.uniform(0.1, 1.0, size=(K, K))
        v[rng.uniform(size=(K, K)) > density] = 0.0
        if v.sum() == 0:
            v[0, 0] = 1.0
        imgs.append(v)
    return problem_from_images(f"tiny{seed}", imgs, alpha=alpha, masses=masses,
                               rho=rho, gamma=gamma, n_bundles=n_bundles)


def config1(i=0) -> Problem:
    """M=3 16x16 images of 2 Gaussian blobs; R=256; rho=100; 500 iterations."""
    rng = np.random.default_rng(1000 * 1 + i)
    imgs = [gaussian_blobs_image(rng, 16, 2, 3, 12, 1.5, 3.0) for _ in range(3)]
    return problem_from_images("cfg1_blobs16_M3", imgs, rho=100.0, iters=500)


def config2(i=0, rho=100.0) -> Problem:
    """M=10 60x60 nested-ellipse images; R=3600; S_m in [600,1500]."""
    rng = np.random.default_rng(1000 * 2 + i)
    imgs = [nested_ellipses_image(rng) for _ in range(10)]
    return problem_from_images("cfg2_ellipses60_M10", imgs, rho=rho, iters=300)


def config3(n_problems=256, i0=0, M_range=(4, 16)) -> List[Problem]:
    """256 independent problems of M~U{4..16} 28x28 stroke images; R=784."""
    out = []
    for i in range(i0, i0 + n_problems):
        rng = np.random.default_rng(1000 * 3 + i)
        M = int(rng.integers(M_range[0], M_range[1] + 1))
        imgs = [bezier_strokes_image(rng) for _ in range(M)]
        out.append(problem_from_images(f"cfg3_strokes28_p{i}", imgs, rho=100.0,
                                       iters=300))
    return out


def config4(i=0, grid=40, M=8) -> Problem:
    """M=8 40x40 Gaussian mixtures; R=1600; target image for the loss.

    ``grid`` and ``M`` shrink the same recipe (centres and widths scale with
    the grid) for cases the FP64 reference finishes in seconds."""
    rng = np.random.default_rng(1000 * 4 + i)
    f = grid / 40.0
    imgs = [gaussian_mixture_image(rng, grid, 3, 5, 6 * f, 34 * f, 2.0 * f, 6.0 * f)
            for _ in range(M)]
    trng = np.random.default_rng(1000 * 4 + i + 10**6)
    tgt = gaussian_mixture_image(trng, grid, 3, 5, 6 * f, 34 * f, 2.0 * f, 6.0 * f).ravel()
    tgt = tgt / tgt.sum()
    name = "cfg4_mixture40_M8" if (grid, M) == (40, 8) else f"cfg4_mixture{grid}_M{M}"
    return problem_from_images(name, imgs, rho=100.0, iters=200, target=tgt)


def config5(i=0, M=100) -> Problem:
    """M=100 100x100 mixtures, S_m~U{500..3000} kept, masses U[0.5,2]."""
    rng = np.random.default_rng(1000 * 5 + i)
    imgs, masses = [], []
    for _ in range(M):
        img = gaussian_mixture_image(rng, 100, 3, 5, 10, 90, 3.0, 12.0, 0.0)
        S = int(rng.integers(500, 3001))
        imgs.append(keep_largest(img, S))
        masses.append(rng.uniform(0.5, 2.0))
    return problem_from_images("cfg5_mixture100_M100_unbalanced", imgs,
                               masses=masses, rho=100.0, gamma=0.01,
                               n_bundles=4, iters=2000)


def free_support_grid(M: int, K: int) -> np.ndarray:
    """Every point sum_m zeta_(m) / M with zeta_(m) on the K x K pixel grid:
    the (M (K - 1) + 1)^2 points (i / (M (K - 1)), j / (M (K - 1))), the
    support that contains a barycenter of M images with equal weights
    (Theorem 1).  Row-major like ``grid_points``."""
    n = M * (K - 1) + 1
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([i.ravel() / (n - 1), j.ravel() / (n - 1)], axis=1).astype(np.float64)


def config2_free_support(i=0, M=10, rho=100.0) -> Problem:
    """The nested-ellipse images of ``config2`` (60x60, M = 10) on the
    free-support grid of their barycenter: R = (10 * 59 + 1)^2 = 349281."""
    p = config2(i, rho=rho)
    q = p.q[:M]
    xi = free_support_grid(len(q), p.K)
    return Problem(name="cfg2_ellipses60_free_support_grid", xi=xi, zeta=p.zeta[:M], q=q,
                   alpha=np.full(len(q), 1.0 / len(q)), rho=rho, K=p.K, iters=p.iters)


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}
