"""Seeded synthetic inputs shaped like the paper's five benchmark workloads.

The paper's inputs come from the AMD APP SDK and the EngineCL bench-suite,
neither of which is available; these generators stand in for them with the
shapes, sizes and value distributions of the five configurations:

* Mandelbrot   -- no input buffer; the region [-2,1] x [-1.5,1.5] at W x H.
* Gaussian     -- U[0,1) FP32 image; 31-tap weights exp(-(t-15)^2 / (2 sigma^2)),
                  normalised in FP64 and rounded to FP32 (Table 2: the filter
                  weights are the kernel's second input buffer).
* NBody        -- positions U[0,1)^3, masses U[0.5,1.5] packed as float4
                  (x, y, z, m) like Listing 2; velocities 0.
* Binomial     -- spot U[10,100], strike = spot * U[0.8,1.2], maturity
                  U[0.25,2], volatility U[0.1,0.5], depth N uniform integer in
                  [256, 2048], rate 0.02.
* GEMM         -- A (M x K) and B stored transposed (N x K), N(0,1) FP32.
* Ray          -- a seeded scene (the paper's scenes are not available): a
                  large ground sphere, spheres scattered in front of the
                  camera (40% reflective), three point lights; sky above.

This module holds none of the method's arithmetic; the oracle and the CUDA
path both take these arrays as they are.  Every generator is a pure function
of its seed (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1805


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- Mandelbrot
def mandelbrot_region(width: int = 1024, height: int = 1024, max_iter: int = 256) -> dict:
    """The classic view [-2,1] x [-1.5,1.5]; dx = 3/width (exact for powers of 2)."""
    return dict(width=width, height=height, x0=-2.0, y0=-1.5,
                dx=float(np.float32(3.0 / width)), dy=float(np.float32(3.0 / height)),
                max_iter=max_iter)


# ---------------------------------------------------------------- Gaussian
def gaussian_image(height: int, width: int, seed: int = SEED_BASE + 1) -> np.ndarray:
    return rng(seed).random((height, width), dtype=np.float32)


def gaussian_weights(taps: int = 31, sigma: float = 5.0) -> np.ndarray:
    r = taps // 2
    w = np.array([math.exp(-((t - r) ** 2) / (2.0 * sigma * sigma)) for t in range(taps)],
                 dtype=np.float64)
    return (w / w.sum()).astype(np.float32)


# ---------------------------------------------------------------- NBody
def nbody_bodies(n: int, seed: int = SEED_BASE + 2):
    g = rng(seed)
    pos = np.empty((n, 4), dtype=np.float32)
    pos[:, :3] = g.random((n, 3), dtype=np.float32)
    pos[:, 3] = g.uniform(0.5, 1.5, n).astype(np.float32)
    vel = np.zeros((n, 4), dtype=np.float32)
    return pos, vel


# ---------------------------------------------------------------- Binomial
BINOMIAL_RATE = 0.02


def binomial_options(n: int, seed: int = SEED_BASE + 3, min_steps: int = 256,
                     max_steps: int = 2048) -> dict:
    g = rng(seed)
    S = g.uniform(10.0, 100.0, n).astype(np.float32)
    ratio = g.uniform(0.8, 1.2, n).astype(np.float32)
    K = (S * ratio).astype(np.float32)
    T = g.uniform(0.25, 2.0, n).astype(np.float32)
    sigma = g.uniform(0.1, 0.5, n).astype(np.float32)
    steps = g.integers(min_steps, max_steps + 1, n).astype(np.int32)
    return dict(S=S, K=K, T=T, sigma=sigma, steps=steps, r=BINOMIAL_RATE)


# ---------------------------------------------------------------- GEMM
def gemm_matrices(M: int, N: int, K: int, seed: int = SEED_BASE + 4):
    g = rng(seed)
    A = g.standard_normal((M, K), dtype=np.float32)
    Bt = g.standard_normal((N, K), dtype=np.float32)
    return A, Bt


# ---------------------------------------------------------------- Ray
RAY_SPHERE_FLOATS = 12  # x y z r | colour r g b | reflectivity kd ks log2(spec exponent) | pad
RAY_LIGHT_FLOATS = 8    # x y z pad | intensity r g b pad


def ray_scene(nspheres: int = 64, nlights: int = 3, seed: int = SEED_BASE + 5) -> dict:
    """Scene buffer (spheres then lights, float32) and the tracer's scalars."""
    g = rng(seed)
    sph = np.zeros((nspheres, RAY_SPHERE_FLOATS), dtype=np.float64)
    if nspheres > 0:  # the ground: a large, slightly reflective sphere
        sph[0] = [0.0, -1001.0, -10.0, 1000.0, 0.6, 0.6, 0.55, 0.2, 0.8, 0.1, 2.0, 0.0]
    for k in range(1, nspheres):
        refl = 0.0 if g.random() < 0.6 else g.uniform(0.3, 0.9)
        sph[k] = [g.uniform(-6.0, 6.0), g.uniform(-0.8, 3.0), g.uniform(-22.0, -6.0), g.uniform(0.3, 1.2),
                  *g.uniform(0.2, 1.0, 3), refl, g.uniform(0.5, 0.9), g.uniform(0.1, 0.6),
                  float(g.integers(3, 7)), 0.0]
    pos = np.array([[-10.0, 10.0, 0.0], [10.0, 8.0, -5.0], [0.0, 20.0, -15.0]])
    lig = np.zeros((nlights, RAY_LIGHT_FLOATS), dtype=np.float64)
    for l in range(nlights):
        lig[l, :3] = pos[l % 3] + (l // 3) * np.array([1.5, 0.5, -2.0])
        lig[l, 4:7] = g.uniform(0.4, 0.8, 3)
    scene = np.concatenate([sph.ravel(), lig.ravel()]).astype(np.float32)
    return dict(scene=scene, nspheres=nspheres, nlights=nlights, ka=0.1, bg=(0.05, 0.07, 0.12), max_depth=3)


def ray_scene_from(spheres, lights) -> np.ndarray:
    """Scene buffer from explicit rows (lists of 12 and 8 numbers)."""
    sph = np.asarray(spheres, dtype=np.float64).reshape(-1, RAY_SPHERE_FLOATS)
    lig = np.asarray(lights, dtype=np.float64).reshape(-1, RAY_LIGHT_FLOATS)
    return np.concatenate([sph.ravel(), lig.ravel()]).astype(np.float32)
