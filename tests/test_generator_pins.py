"""Pins of the seeded synthetic Kikuchi generator (the stand-in for the paper's simulated patterns;
input generation only, none of the method's arithmetic).

- the counter-based RNG is SplitMix64 (Vigna) keyed by (seed, stream, counter), restated here with
  Python integers;
- kinematic bands: with one lattice plane the intensity is a decreasing function of the angle to the
  plane, so the band centre is the trace of n . g = 0 (the gnomonic projection of the plane);
- the 25 planes of {111}, {200}, {220}, {311} form whole families: the pattern of orientation g C is
  that of g for each of the 24 proper rotations C of the cube;
- the Poisson noise (Cornish-Fisher form) has mean `counts` and unit variance in units of sqrt(lambda).
The GPU twin of the generator is compared with this one in tests/test_gpu_generator.py."""
import itertools
import math

import numpy as np
import pytest

from synth import kikuchi as K

M64 = (1 << 64) - 1


def splitmix64(z):
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_rng_is_splitmix64():
    seed, stream = 12345, 16 * 77 + K.P_NOISE
    key = splitmix64((splitmix64(seed) + stream * 0xD1B54A32D192ED03) & M64)
    assert int(K.stream_key(seed, stream)) == key
    u = K.uniforms(seed, stream, 6, start=10)
    for i, c in enumerate(range(10, 16)):
        bits = splitmix64((key + c * 0x632BE59BD9B4E019) & M64)
        assert u[i] == (bits >> 11) * 2.0 ** -53
    # Box-Muller (cosine branch) on consecutive pairs
    z = K.normals(seed, stream, 3)
    uu = K.uniforms(seed, stream, 6)
    for i in range(3):
        assert abs(z[i] - math.sqrt(-2 * math.log(1 - uu[2 * i])) * math.cos(2 * math.pi * uu[2 * i + 1])) < 1e-14


def cube_rotations():
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            C = np.zeros((3, 3))
            for i, (p, s) in enumerate(zip(perm, signs)):
                C[i, p] = s
            if np.linalg.det(C) > 0:
                out.append(C)
    assert len(out) == 24
    return out


def test_plane_set_is_whole_families():
    hkl = K.fcc_planes()
    assert len(hkl) == 4 + 3 + 6 + 12
    key = lambda v: tuple(np.round(v).astype(int))
    signed = {key(v) for v in hkl} | {key(-v) for v in hkl}
    for C in cube_rotations():
        assert {key(C @ v) for v in hkl} <= signed


def test_pattern_invariant_under_cube_symmetry():
    g = K.random_rotation(5, 3)
    a = K.render(g, np.eye(3), 48, 64, noise=False)
    for C in cube_rotations()[:: 5]:
        b = K.render(g @ C, np.eye(3), 48, 64, noise=False)
        assert np.abs(b - a).max() <= 1e-5 * np.abs(a).max()
    # a rotation that is not a cube symmetry changes the pattern
    c = K.render(g @ K.axis_angle([1, 2, 3], math.radians(5)), np.eye(3), 48, 64, noise=False)
    assert np.abs(c - a).max() > 0.05 * np.abs(a).max()


def test_band_centre_on_plane_trace(monkeypatch):
    plane = np.array([[1.0, 1.0, 1.0]])
    monkeypatch.setattr(K, "fcc_planes", lambda: plane)
    # orientation that puts the (111) normal at (cos 0.4, sin 0.4, 0.1): an oblique trace through the
    # middle of the detector
    a = plane[0] / np.linalg.norm(plane[0])
    b = np.array([math.cos(0.4), math.sin(0.4), 0.1])
    b /= np.linalg.norm(b)
    axis = np.cross(a, b)
    g = K.axis_angle(axis, math.asin(np.linalg.norm(axis)) if a @ b > 0 else math.pi - math.asin(np.linalg.norm(axis)))
    assert np.abs(g @ a - b).max() < 1e-12
    H, W = 64, 80
    img = K.render(g, np.eye(3), H, W, noise=False, background=False).astype(np.float64)
    n = g @ plane[0]
    n /= np.linalg.norm(n)
    d = K.pixel_directions(H, W, K.Geometry())
    ang = np.abs(np.arcsin(d @ n)).reshape(H, W)
    # intensity decreases with the angle to the plane: same order, and the brightest pixel of every
    # row that the trace crosses is the pixel nearest to n . d = 0
    order = np.argsort(ang.ravel(), kind="stable")
    assert np.all(np.diff(img.ravel()[order]) <= 1e-4)
    rows = 0
    for i in range(H):
        if ang[i].min() < 0.01:
            assert np.argmax(img[i]) == np.argmin(ang[i])
            rows += 1
    assert rows > H // 2
    assert img.max() - img.min() > 0.1 * img.mean()


def test_poisson_noise_mean_and_variance():
    g = K.random_rotation(9, 1)
    clean = K.render(g, np.eye(3), 256, 256, counts=500.0, noise=False).astype(np.float64)
    noisy = K.render(g, np.eye(3), 256, 256, counts=500.0, noise=True, seed=9, stream=4).astype(np.float64)
    assert abs(clean.mean() - 500.0) < 1e-3
    assert abs(noisy.mean() - 500.0) < 0.5          # sd of the mean: sqrt(500 / 65536) = 0.087
    r = (noisy - clean) / np.sqrt(clean)
    assert abs(r.var() - 1.0) < 0.03                # Poisson: variance = mean
    assert np.all(noisy == np.rint(noisy)) and noisy.min() >= 0
