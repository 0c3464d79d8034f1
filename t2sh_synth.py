"""Seeded synthetic inputs shaped like the paper's knee workload (Table I, Sec. V.A).

This module draws the STRUCTURE of an acquisition and nothing else: the temporal
basis Phi, a phantom (proton density and T2 per voxel), coil sensitivities, per-echo
sampling masks and complex noise.  It holds none of the reconstruction's arithmetic
(no Fourier transform, no space-time kernel, no sensitivity operator): turning these
pieces into k-space is done by whoever consumes them.  Both the CUDA path's tests and
the FP64 oracle's tests take their inputs from here, so the two see identical bytes.

Randomness: numpy's PCG64 seeded through ``numpy.random.SeedSequence`` with the
(base seed, scan, slice) words, so every slice is reproducible on its own.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def rng_for(base_seed: int, *words: int) -> np.random.Generator:
    """Independent generator for (base_seed, *words)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(base_seed), *map(int, words)])))


# ---------------------------------------------------------------------------------
# Temporal basis (the paper builds it from EPG simulations and an SVD, Sec. III.A;
# with no flip-angle schedule here, the decays are plain exponentials exp(-t/T2)).
# ---------------------------------------------------------------------------------
def echo_times_ms(T: int, es_ms: float = 5.0) -> np.ndarray:
    """t_i = (i + 1) * echo spacing, i = 0 .. T-1 (ms)."""
    return (np.arange(T, dtype=np.float64) + 1.0) * es_ms


def t2_basis(T: int, K: int, es_ms: float = 5.0, t2_lo: float = 20.0, t2_hi: float = 200.0,
             n_t2: int = 256) -> np.ndarray:
    """Phi [T][K], float64: top-K left singular vectors of [exp(-t_i / T2_j)],
    T2_j on linspace(t2_lo, t2_hi, n_t2) ms; each column's largest-magnitude entry > 0."""
    t = echo_times_ms(T, es_ms)
    t2 = np.linspace(t2_lo, t2_hi, n_t2)
    sig = np.exp(-t[:, None] / t2[None, :])
    U, _, _ = np.linalg.svd(sig, full_matrices=False)
    phi = U[:, :K].copy()
    for k in range(K):
        if phi[np.argmax(np.abs(phi[:, k])), k] < 0:
            phi[:, k] = -phi[:, k]
    return phi


# ---------------------------------------------------------------------------------
# Phantoms.
# ---------------------------------------------------------------------------------
def ellipse_phantom(ny: int, nz: int, rng: np.random.Generator, n_ellipses: int = 10):
    """2D random-ellipse phantom: (rho, t2_ms) [ny][nz].  A large body ellipse, then
    smaller ones inside it; each has proton density U[0.2, 1] and T2 U[20, 200] ms."""
    yy, zz = np.meshgrid(np.linspace(-1, 1, ny, endpoint=False), np.linspace(-1, 1, nz, endpoint=False),
                         indexing="ij")
    rho = np.zeros((ny, nz))
    t2 = np.full((ny, nz), 50.0)
    for e in range(n_ellipses):
        if e == 0:
            cy, cz, ay, az, th = 0.0, 0.0, 0.8, 0.7, rng.uniform(-0.2, 0.2)
        else:
            cy, cz = rng.uniform(-0.5, 0.5, 2)
            ay, az = rng.uniform(0.08, 0.35, 2)
            th = rng.uniform(0, np.pi)
        c, s = np.cos(th), np.sin(th)
        u = (c * (yy - cy) + s * (zz - cz)) / ay
        v = (-s * (yy - cy) + c * (zz - cz)) / az
        inside = u * u + v * v <= 1.0
        rho[inside] = rng.uniform(0.2, 1.0)
        t2[inside] = rng.uniform(20.0, 200.0)
    return rho, t2


@dataclass
class EllipsoidVolume:
    """A 3D multi-tissue ellipsoid phantom, evaluated one readout slice at a time."""
    centres: np.ndarray   # [E][3] in (x, y, z), unit cube [-1, 1)
    axes: np.ndarray      # [E][3]
    rot: np.ndarray       # [E][3][3]
    rho: np.ndarray       # [E]
    t2: np.ndarray        # [E]

    @staticmethod
    def draw(rng: np.random.Generator, n_ellipsoids: int = 14) -> "EllipsoidVolume":
        cen, ax, rot, rho, t2 = [], [], [], [], []
        for e in range(n_ellipsoids):
            if e == 0:
                cen.append([0.0, 0.0, 0.0]); ax.append([0.85, 0.8, 0.7])
            else:
                cen.append(rng.uniform(-0.5, 0.5, 3)); ax.append(rng.uniform(0.1, 0.4, 3))
            q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
            rot.append(q)
            rho.append(rng.uniform(0.2, 1.0)); t2.append(rng.uniform(20.0, 200.0))
        return EllipsoidVolume(np.array(cen), np.array(ax), np.array(rot), np.array(rho), np.array(t2))

    def slice(self, x: float, ny: int, nz: int):
        """(rho, t2_ms) [ny][nz] of the plane at readout coordinate x in [-1, 1)."""
        yy, zz = np.meshgrid(np.linspace(-1, 1, ny, endpoint=False), np.linspace(-1, 1, nz, endpoint=False),
                             indexing="ij")
        pts = np.stack([np.full_like(yy, x), yy, zz], -1)
        rho = np.zeros((ny, nz))
        t2 = np.full((ny, nz), 50.0)
        for e in range(len(self.rho)):
            d = (pts - self.centres[e]) @ self.rot[e]
            inside = np.sum((d / self.axes[e]) ** 2, -1) <= 1.0
            rho[inside] = self.rho[e]
            t2[inside] = self.t2[e]
        return rho, t2


def decay_series(rho: np.ndarray, t2_ms: np.ndarray, te_ms: np.ndarray) -> np.ndarray:
    """Echo images x_t = rho exp(-t / T2): [T][..] complex128 (phantom signal model)."""
    return (rho[None] * np.exp(-te_ms[:, None, None] / t2_ms[None])).astype(np.complex128)


# ---------------------------------------------------------------------------------
# Coil sensitivities: smooth Gaussian bumps centred on a ring around the FOV, with
# random linear phase, normalised so the largest eigenvalue of S(p)^H S(p) is 1 at
# every pixel (then the step 1/L is 1 under full sampling).
# ---------------------------------------------------------------------------------
def coil_maps(C: int, ny: int, nz: int, rng: np.random.Generator, M: int = 1,
              width: float = 0.4, second_set_scale: float = 0.3) -> np.ndarray:
    """maps [C][M][ny][nz] complex128."""
    yy, zz = np.meshgrid(np.linspace(-1, 1, ny, endpoint=False), np.linspace(-1, 1, nz, endpoint=False),
                         indexing="ij")

    def one_set():
        s = np.empty((C, ny, nz), np.complex128)
        ang0 = rng.uniform(0, 2 * np.pi)
        for c in range(C):
            a = ang0 + 2 * np.pi * c / C
            cy, cz = 1.1 * np.cos(a), 1.1 * np.sin(a)
            mag = np.exp(-((yy - cy) ** 2 + (zz - cz) ** 2) / (2 * (2 * width) ** 2))
            ph = rng.uniform(0, 2 * np.pi) + rng.uniform(-np.pi, np.pi) * yy + rng.uniform(-np.pi, np.pi) * zz
            s[c] = mag * np.exp(1j * ph)
        return s

    sets = [one_set()]
    for _ in range(1, M):
        sets.append(second_set_scale * one_set())
    maps = np.stack(sets, axis=1)  # [C][M][ny][nz]
    sp = np.moveaxis(maps, (0, 1), (-2, -1))  # [ny][nz][C][M]
    lam = np.linalg.eigvalsh(np.conj(np.swapaxes(sp, -1, -2)) @ sp).max(-1)
    return maps / np.sqrt(lam)[None, None]


# ---------------------------------------------------------------------------------
# Sampling: per echo, independent variable-density Bernoulli sampling in centred
# k-space, p(r) ~ (1 - r / r_max)^2 + eps scaled to the target fraction; echo 0
# always holds a calib x calib centre.  Returns uint8 [T][ny][nz] (DC at ny/2, nz/2).
# ---------------------------------------------------------------------------------
def vd_masks(T: int, ny: int, nz: int, frac: float, rng: np.random.Generator, calib: int = 6,
             eps: float = 0.02) -> np.ndarray:
    ky = (np.arange(ny) - ny // 2) / (ny / 2)
    kz = (np.arange(nz) - nz // 2) / (nz / 2)
    r = np.sqrt(ky[:, None] ** 2 + kz[None, :] ** 2)
    w = np.clip(1.0 - r / r.max(), 0.0, 1.0) ** 2 + eps
    # scale so the mean probability is frac (clip at 1, rescale a few times)
    p = w * frac / w.mean()
    for _ in range(20):
        p = np.clip(p, 0.0, 1.0)
        p = p * frac / p.mean()
    p = np.clip(p, 0.0, 1.0)
    masks = (rng.random((T, ny, nz)) < p[None]).astype(np.uint8)
    c0y, c0z = ny // 2 - calib // 2, nz // 2 - calib // 2
    masks[0, c0y:c0y + calib, c0z:c0z + calib] = 1
    return masks


def complex_noise(shape, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Circular complex Gaussian: Re, Im ~ N(0, sigma^2/2), so E|w|^2 = sigma^2."""
    s = sigma / np.sqrt(2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


# ---------------------------------------------------------------------------------
# The configurations the solver is measured on (synthetic stand-ins for the paper's
# pediatric knee scans, which are not available).
# ---------------------------------------------------------------------------------
@dataclass(frozen=True)
class ScanShape:
    name: str
    nslices: int
    ny: int
    nz: int
    ncoils: int
    nechoes: int
    nbasis: int
    frac: float
    lam: float
    iters: int
    block: int = 8
    nmaps: int = 1
    seed: int = 1809


SINGLE_SLICE_64x48 = ScanShape("single slice 64x48, C=8, T=32, K=4, 10%/echo, 50 iterations",
                               1, 64, 48, 8, 32, 4, 0.10, 0.01, 50, seed=1809)
KNEE_320x256x160 = ScanShape("knee scan 320 slices of 256x160, C=12, T=80, K=4, 5%/echo, 100 iterations",
                             320, 256, 160, 12, 80, 4, 0.05, 0.005, 100, seed=1810)
# Table I: 288 readout slices of 260 x 240, C = 7 virtual coils, T = 80, K = 4, M = 2
# soft-SENSE map sets, 12 x 12 LLR blocks, lambda = 0.0125, 250 FISTA iterations; each echo
# undersampled by 139 (Sec. V)
PAPER_288x260x240 = ScanShape("paper scan (Table I) 288 slices of 260x240, C=7, T=80, K=4, M=2, b=12, "
                              "1/139 per echo, 250 iterations",
                              288, 260, 240, 7, 80, 4, 1.0 / 139.0, 0.0125, 250, block=12, nmaps=2, seed=1815)
BATCH_SCANS = (
    KNEE_320x256x160,
    ScanShape("scan 288 slices of 240x128, C=8", 288, 240, 128, 8, 80, 4, 0.05, 0.005, 100, seed=1812),
    ScanShape("scan 256 slices of 192x192, C=16", 256, 192, 192, 16, 80, 4, 0.05, 0.005, 100, seed=1813),
)


@dataclass
class SliceStructure:
    """Per-slice phantom and coil maps for one scan."""
    rho: np.ndarray
    t2: np.ndarray
    maps: np.ndarray


def scan_common(shape: ScanShape):
    """(phi [T][K] float64, masks [T][ny][nz] uint8, te_ms [T]) shared by all slices."""
    phi = t2_basis(shape.nechoes, shape.nbasis)
    masks = vd_masks(shape.nechoes, shape.ny, shape.nz, shape.frac, rng_for(shape.seed, 0, 0))
    return phi, masks, echo_times_ms(shape.nechoes)


def slice_structure(shape: ScanShape, s: int, volume: EllipsoidVolume | None = None) -> SliceStructure:
    """Phantom and maps of slice ``s``; 3D phantom slices when ``volume`` is given."""
    rng = rng_for(shape.seed, 1, s)
    if volume is None:
        rho, t2 = ellipse_phantom(shape.ny, shape.nz, rng)
    else:
        x = -1.0 + 2.0 * (s + 0.5) / max(shape.nslices, 1)
        rho, t2 = volume.slice(x, shape.ny, shape.nz)
    maps = coil_maps(shape.ncoils, shape.ny, shape.nz, rng_for(shape.seed, 2, s), M=shape.nmaps)
    return SliceStructure(rho, t2, maps)
