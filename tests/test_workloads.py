"""The seeded synthetic inputs (the stand-ins for the paper's benchmark
inputs): reproducible from their seeds, and with the shapes and ranges the
five configurations state."""
import numpy as np

import workloads as W


def test_seeds_reproduce_and_differ():
    a1, _ = W.nbody_bodies(1000)
    a2, _ = W.nbody_bodies(1000)
    assert np.array_equal(a1, a2)
    b, _ = W.nbody_bodies(1000, seed=W.SEED_BASE + 99)
    assert not np.array_equal(a1, b)
    assert W.SEED_BASE == 1805


def test_mandelbrot_view():
    r = W.mandelbrot_region()
    assert (r["width"], r["height"], r["max_iter"]) == (1024, 1024, 256)
    assert (r["x0"], r["y0"]) == (-2.0, -1.5)
    # 3 / 1024 is a power-of-two fraction of 3: exact in FP32, so every pixel's c is exact
    assert np.float32(r["dx"]) == 3.0 / 1024 and np.float32(r["dy"]) == 3.0 / 1024
    big = W.mandelbrot_region(8192, 8192, 1024)
    assert np.float32(big["dx"]) == 3.0 / 8192 and big["max_iter"] == 1024


def test_gaussian_image_uniform_unit_interval():
    img = W.gaussian_image(512, 768)
    assert img.shape == (512, 768) and img.dtype == np.float32
    assert img.min() >= 0.0 and img.max() < 1.0
    assert abs(float(img.mean()) - 0.5) < 0.01


def test_nbody_positions_and_masses():
    pos, vel = W.nbody_bodies(65536)
    assert pos.shape == (65536, 4) and pos.dtype == np.float32
    assert pos[:, :3].min() >= 0.0 and pos[:, :3].max() < 1.0
    assert pos[:, 3].min() >= 0.5 and pos[:, 3].max() <= 1.5
    assert not vel.any()


def test_binomial_options_ranges():
    o = W.binomial_options(1 << 16)
    assert o["r"] == 0.02
    assert o["S"].min() >= 10.0 and o["S"].max() <= 100.0
    ratio = o["K"].astype(np.float64) / o["S"]
    assert ratio.min() >= 0.8 - 1e-6 and ratio.max() <= 1.2 + 1e-6
    assert o["T"].min() >= 0.25 and o["T"].max() <= 2.0
    assert o["sigma"].min() >= 0.1 and o["sigma"].max() <= 0.5
    st = o["steps"]
    assert st.dtype == np.int32 and st.min() == 256 and st.max() == 2048  # both ends drawn at this size
    assert abs(float(st.mean()) - 1152.0) < 10.0


def test_gemm_inputs_standard_normal():
    A, Bt = W.gemm_matrices(512, 384, 256)
    assert A.shape == (512, 256) and Bt.shape == (384, 256) and A.dtype == np.float32
    for X in (A, Bt):
        assert abs(float(X.mean())) < 0.02 and abs(float(X.std()) - 1.0) < 0.02


def test_ray_scene_recipe():
    sc = W.ray_scene()
    assert (sc["nspheres"], sc["nlights"], sc["max_depth"], sc["ka"]) == (64, 3, 3, 0.1)
    sph = sc["scene"][:64 * W.RAY_SPHERE_FLOATS].reshape(64, W.RAY_SPHERE_FLOATS)
    lig = sc["scene"][64 * W.RAY_SPHERE_FLOATS:].reshape(3, W.RAY_LIGHT_FLOATS)
    assert sph[0, 3] == 1000.0 and sph[0, 1] == -1001.0  # the ground sphere, top at y = -1
    rest = sph[1:]
    assert rest[:, 0].min() >= -6 and rest[:, 0].max() <= 6 and rest[:, 2].min() >= -22 and rest[:, 2].max() <= -6
    assert rest[:, 3].min() >= 0.3 and rest[:, 3].max() <= 1.2
    refl = (rest[:, 7] > 0).mean()
    assert 0.2 < refl < 0.6  # about 40% reflective
    assert set(np.unique(rest[:, 10]).tolist()) <= {3.0, 4.0, 5.0, 6.0}  # specular exponent 2^3..2^6
    assert (lig[:, 1] >= 8.0).all()  # lights above the scene
