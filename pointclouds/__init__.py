"""Seeded synthetic point clouds shared by the CUDA path, the oracle, the tests and the bench.

This module only draws random points and rounds them to the 2^-16 grid. It contains none of
the persistent-homology arithmetic (no diameters, no filtration, no reduction), so both the
CUDA path and the CPU oracle may consume its output without sharing any method code.

Grid convention: a coordinate x is stored as the int32 value rint(x * 65536) (round half to
even, as ``numpy.rint`` does). Squared distances of grid points are then exact int64 values,
which makes the Vietoris-Rips filtration order exact on every machine.

Workloads (the paper's own Javaplex point clouds, Sec. 4, are not available, so these seeded
clouds stand in for them; they follow the sizes and shapes of the benchmark configurations):

* ``circle40``   40 points, angle uniform on the unit circle in R^2 plus N(0, 0.05^2 I_2).
* ``torus400``   400 points on the torus of radii R=2, r=1 in R^3, both angles uniform.
* ``gauss8_120`` 120 points i.i.d. N(0, I_8), truncated later at squared diameter 16.
* ``batch512``   512 clouds, n_i uniform in {20..120}; cloud i is drawn from family i mod 3:
                 unit 2-sphere (normalised N(0, I_3)), torus (R=2, r=1), N(0, I_3).
* ``diff256``    256 clouds of 64 points, unit 2-sphere plus N(0, 0.02^2 I_3), kept in fp32.
* ``ensemble15`` the four ensembles of the paper's iteration experiments (Sec. 4: Gaussian
                 points in R^3, figure-8, trefoil knot, S^2 x S^2; N = 15, complete complex up
                 to dimension 5). The paper gives no sampling laws, so these are stand-ins:
                 N(0, I_3); a figure-8 (lemniscate of Gerono) and a trefoil knot, each with the
                 curve parameter uniform and N(0, 0.05^2 I_3) noise; normalised N(0, I_3) pairs
                 in R^6 for S^2 x S^2.
"""
from __future__ import annotations

import numpy as np

GRID_SCALE = 65536  # 2^16 grid units per unit length
BASE_SEED = 1708_04710

CONFIG_IDS = {"circle40": 1, "torus400": 2, "gauss8_120": 3, "batch512": 4, "diff256": 5,
              "gaussian15": 10, "figure8_15": 11, "trefoil15": 12, "sphere_product15": 13}
ENSEMBLES = ("gaussian15", "figure8_15", "trefoil15", "sphere_product15")


def to_grid(x: np.ndarray) -> np.ndarray:
    """Round real coordinates to int32 grid units (round half to even)."""
    g = np.rint(np.asarray(x, dtype=np.float64) * GRID_SCALE)
    if np.abs(g).max(initial=0) >= 2**30:
        raise ValueError("coordinates too large for the int32 grid")
    return g.astype(np.int32)


def rng_for(config_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + config_id + 1000 * salt))


def circle(n: int, rng: np.random.Generator, sigma: float = 0.05) -> np.ndarray:
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n)
    pts = np.stack([np.cos(theta), np.sin(theta)], axis=1)
    return pts + rng.normal(0.0, sigma, size=(n, 2))


def torus(n: int, rng: np.random.Generator, R: float = 2.0, r: float = 1.0) -> np.ndarray:
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n)
    return np.stack([(R + r * np.cos(phi)) * np.cos(theta),
                     (R + r * np.cos(phi)) * np.sin(theta),
                     r * np.sin(phi)], axis=1)


def sphere(n: int, rng: np.random.Generator, noise: float = 0.0) -> np.ndarray:
    g = rng.standard_normal(size=(n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    if noise > 0:
        g = g + rng.normal(0.0, noise, size=(n, 3))
    return g


def gaussian(n: int, d: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal(size=(n, d))


# ----------------------------------------------------------------------------------------------
# Benchmark workloads. Each returns int32 grid coordinates; the batched ones also return the
# per-cloud point offsets (int64, length n_clouds + 1).
# ----------------------------------------------------------------------------------------------

def circle40(n: int = 40) -> np.ndarray:
    return to_grid(circle(n, rng_for(1)))


def torus400(n: int = 400) -> np.ndarray:
    return to_grid(torus(n, rng_for(2)))


# squared-diameter cut of the 8-dimensional Gaussian workload, in grid units^2 (16 * 2^32)
GAUSS8_MAX_DIAM2 = 16 * GRID_SCALE * GRID_SCALE


def gauss8_120(n: int = 120) -> np.ndarray:
    return to_grid(gaussian(n, 8, rng_for(3)))


def batch512(n_clouds: int = 512, n_lo: int = 20, n_hi: int = 120):
    rng = rng_for(4)
    sizes = rng.integers(n_lo, n_hi + 1, size=n_clouds)
    clouds = []
    for i, n in enumerate(sizes):
        fam = i % 3
        if fam == 0:
            pts = sphere(int(n), rng)
        elif fam == 1:
            pts = torus(int(n), rng)
        else:
            pts = gaussian(int(n), 3, rng)
        clouds.append(to_grid(pts))
    offsets = np.zeros(n_clouds + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.concatenate(clouds, axis=0), offsets


def diff256(n_clouds: int = 256, n: int = 64):
    """fp32 coordinates (n_clouds*n, 3) and offsets; the pairing uses to_grid of these values."""
    rng = rng_for(5)
    pts = np.concatenate([sphere(n, rng, noise=0.02) for _ in range(n_clouds)], axis=0)
    offsets = np.arange(n_clouds + 1, dtype=np.int64) * n
    return pts.astype(np.float32), offsets


def random_cloud(n: int, d: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Small Gaussian cloud for unit and parity tests."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 7919 * (seed + 1)))
    return to_grid(scale * rng.standard_normal(size=(n, d)))


def lattice_cloud(n: int, d: int, seed: int, side: int = 4) -> np.ndarray:
    """Points on a coarse integer lattice: many exactly equal squared distances (tie stress)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 104729 * (seed + 1)))
    return (rng.integers(0, side, size=(n, d)) * GRID_SCALE).astype(np.int32)


def figure8(n: int, rng: np.random.Generator, noise: float = 0.05) -> np.ndarray:
    t = rng.uniform(0.0, 2.0 * np.pi, size=n)
    pts = np.stack([np.cos(t), np.sin(t) * np.cos(t), np.zeros(n)], axis=1)
    return pts + rng.normal(0.0, noise, size=(n, 3))


def trefoil(n: int, rng: np.random.Generator, noise: float = 0.05) -> np.ndarray:
    t = rng.uniform(0.0, 2.0 * np.pi, size=n)
    pts = np.stack([np.sin(t) + 2.0 * np.sin(2.0 * t), np.cos(t) - 2.0 * np.cos(2.0 * t),
                    -np.sin(3.0 * t)], axis=1)
    return pts + rng.normal(0.0, noise, size=(n, 3))


def sphere_product(n: int, rng: np.random.Generator) -> np.ndarray:
    return np.concatenate([sphere(n, rng), sphere(n, rng)], axis=1)


def ensemble15(name: str, sample: int = 0, n: int = 15) -> np.ndarray:
    """One point cloud of an iteration-experiment ensemble (names in ENSEMBLES), on the grid."""
    rng = rng_for(CONFIG_IDS[name], salt=sample)
    if name == "gaussian15":
        x = gaussian(n, 3, rng)
    elif name == "figure8_15":
        x = figure8(n, rng)
    elif name == "trefoil15":
        x = trefoil(n, rng)
    elif name == "sphere_product15":
        x = sphere_product(n, rng)
    else:
        raise ValueError(name)
    return to_grid(x)
