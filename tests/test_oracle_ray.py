"""Pins of the ray-tracer oracle against closed forms, symmetry and exact special cases.

The oracle evaluates the tracer in FP32 (its definition is in oracle.c);
these checks come from geometry and the shading formula, not from the code.
"""
import math

import numpy as np
import pytest

import workloads as W

BG = (0.05, 0.07, 0.12)


def sphere(x, y, z, r, col=(1.0, 1.0, 1.0), refl=0.0, kd=1.0, ks=0.0, e=0):
    return [x, y, z, r, *col, refl, kd, ks, float(e), 0.0]


def light(x, y, z, I=(1.0, 1.0, 1.0)):
    return [x, y, z, 0.0, *I, 0.0]


def trace(oracle_mod, sph, lig, W_, H_, ka=0.0, bg=BG, depth=3):
    scene = W.ray_scene_from(sph, lig) if sph else W.ray_scene_from(np.zeros((0, 12)), lig)
    return oracle_mod.ray(scene, len(sph), len(lig), W_, H_, ka, bg, depth)


def test_empty_scene_is_background(oracle_mod):
    img = trace(oracle_mod, [], [light(0, 5, 0)], 33, 17)
    assert np.array_equal(img[..., 0], np.full((17, 33), np.float32(BG[0])))
    assert np.array_equal(img[..., 2], np.full((17, 33), np.float32(BG[2])))
    assert (img[..., 3] == 1.0).all()  # one camera ray per pixel


def test_head_on_diffuse_and_specular(oracle_mod):
    # sphere straight ahead, light at the camera: at the image centre the normal,
    # the light and the view directions coincide, so n.l = 1 and r.(-d) = 1
    col = (0.5, 0.25, 0.75)
    ka, kd, ks = 0.125, 0.5, 0.25
    img = trace(oracle_mod, [sphere(0, 0, -10, 2, col, 0.0, kd, ks, 3)], [light(0, 0, 0, (1.0, 0.5, 2.0))],
                65, 65, ka=ka)
    c = img[32, 32]
    want = [ka * col[k] + kd * col[k] * I + ks * I for k, I in enumerate((1.0, 0.5, 2.0))]
    assert np.allclose(c[:3], want, rtol=2e-6)
    assert c[3] == 2.0  # camera ray + one shadow ray


def test_silhouette_matches_geometry(oracle_mod):
    # a ray hits the sphere iff its distance to the centre is below r; check every
    # pixel whose analytic margin exceeds rounding
    Wd = Hd = 96
    cx, cy, cz, r = 0.7, -0.4, -8.0, 2.5
    img = trace(oracle_mod, [sphere(cx, cy, cz, r)], [light(0, 10, 0)], Wd, Hd)
    hit = img[..., 3] > 1.0
    j, i = np.mgrid[0:Hd, 0:Wd]
    u = (2 * i + 1 - Wd) / Hd
    v = (Hd - 2 * j - 1) / Hd
    d = np.stack([u, v, -np.ones_like(u)], -1)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    c = np.array([cx, cy, cz])
    proj = d @ c
    miss_dist = np.sqrt(np.maximum(c @ c - proj ** 2, 0.0))
    sure = np.abs(miss_dist - r) > 1e-4
    assert np.array_equal(hit[sure], (miss_dist < r)[sure])
    assert hit.sum() > 100 and (~hit).sum() > 100


def test_shadow_leaves_ambient(oracle_mod):
    # light above the big sphere and a small sphere on the shadow ray of the point the
    # camera sees at u = 0, v = 38/129 (p ~ (0, 2.43, -8.24)): ambient term only
    ka = 0.25
    col = (0.8, 0.6, 0.4)
    sph = [sphere(0, 0, -10, 3, col, 0.0, 1.0, 0.0), sphere(0, 7.35, -9.15, 0.6)]
    lig = [light(0, 12, -10)]
    img = trace(oracle_mod, sph, lig, 129, 129, ka=ka)
    c = img[45, 64]  # u = 0, v = 38/129
    assert c[3] == 2.0  # camera ray + shadow ray
    assert np.allclose(c[:3], [ka * x for x in col], rtol=1e-6), c
    # without the occluder the same pixel is lit
    lit = trace(oracle_mod, sph[:1], lig, 129, 129, ka=ka)[45, 64]
    assert (lit[:3] > c[:3] + 0.1).all()


def test_mirror_head_on_sees_background(oracle_mod):
    # a reflective sphere hit head-on reflects the ray back past the camera into the
    # background: colour = (1 - refl) local + refl bg
    refl, ka = 0.5, 0.2
    col = (0.6, 0.4, 0.2)
    img = trace(oracle_mod, [sphere(0, 0, -6, 1, col, refl, 0.0, 0.0)], [light(0, 0, 0)], 33, 33, ka=ka)
    c = img[16, 16]
    want = [(1 - refl) * ka * col[k] + refl * BG[k] for k in range(3)]
    assert np.allclose(c[:3], want, rtol=1e-6)
    assert c[3] == 3.0  # camera, shadow, reflected ray
    # with max depth 0 the reflection is not followed
    img0 = trace(oracle_mod, [sphere(0, 0, -6, 1, col, refl, 0.0, 0.0)], [light(0, 0, 0)], 33, 33, ka=ka, depth=0)
    assert np.allclose(img0[16, 16, :3], [ka * x for x in col], rtol=1e-6) and img0[16, 16, 3] == 2.0


def test_mirror_symmetric_scene_gives_symmetric_image(oracle_mod):
    # u is computed from integers, so mirrored pixels get exactly negated x components
    g = np.random.default_rng(11)
    sph, lig = [sphere(0, -1001, -10, 1000, (0.6, 0.6, 0.6), 0.3, 0.8, 0.1, 2)], [light(0, 10, -3)]
    for _ in range(6):
        x, y, z, r = g.uniform(0.5, 4), g.uniform(-0.5, 2), g.uniform(-15, -5), g.uniform(0.3, 1)
        col = tuple(g.uniform(0.2, 1, 3))
        refl = float(g.choice([0.0, 0.5]))
        sph += [sphere(x, y, z, r, col, refl, 0.7, 0.3, 4), sphere(-x, y, z, r, col, refl, 0.7, 0.3, 4)]
    lig += [light(5, 8, -2), light(-5, 8, -2)]
    img = trace(oracle_mod, sph, lig, 80, 60, ka=0.1)
    assert np.array_equal(img[..., 3], img[:, ::-1, 3])
    assert np.allclose(img[..., :3], img[:, ::-1, :3], rtol=0, atol=1e-5)


def test_workload_scene_properties(oracle_mod):
    sc = W.ray_scene()
    img = oracle_mod.ray(sc["scene"], sc["nspheres"], sc["nlights"], 128, 128, sc["ka"], sc["bg"], sc["max_depth"])
    rays = img[..., 3]
    # sky pixels cost one ray; hits cost 1 + lights per bounce (up to 1 + 3 bounces)
    assert rays.min() == 1.0 and rays.max() <= 1 + (1 + 3) * (1 + sc["nlights"])
    assert (rays == 1.0).mean() > 0.2 and (rays > 4).mean() > 0.05  # irregular: both kinds present
    assert np.isfinite(img).all() and img[..., :3].min() >= 0.0
