"""Pins of the strain/stress oracle (Eq. 13-16, Supplementary Part 2)."""
import numpy as np

from oracle import strain as S
from synth import kikuchi as K

rng = np.random.default_rng(11)


def test_uniaxial_strain_in_crystal_axes():
    C = S.cubic_stiffness(*S.NI_C)
    e = 1e-3
    sig = S.stress(C, np.diag([e, 0.0, 0.0]))
    assert np.allclose(sig, np.diag([S.NI_C[0] * e, S.NI_C[1] * e, S.NI_C[1] * e]), rtol=1e-14, atol=1e-3)
    shear = np.zeros((3, 3))
    shear[0, 1] = shear[1, 0] = e
    assert abs(S.stress(C, shear)[0, 1] - 2 * S.NI_C[2] * e) < 1e-3


def test_isotropic_stiffness_is_rotation_invariant_and_cubic_symmetry():
    iso = S.cubic_stiffness(3.0, 1.0, 1.0)   # C11 - C12 = 2 C44
    g = K.axis_angle(rng.normal(size=3), 0.7)
    assert np.abs(S.rotate_stiffness(iso, g) - iso).max() < 1e-14
    C = S.cubic_stiffness(*S.NI_C)
    q = K.axis_angle([0, 0, 1], np.pi / 2)   # a symmetry operation of the cube
    assert np.abs(S.rotate_stiffness(C, q) - C).max() < 1e-3
    assert np.abs(S.rotate_stiffness(C, g) - C).max() > 1e9   # anisotropic: a general rotation changes it


def test_pure_rotation_gives_zero_strain_and_stress():
    R = K.axis_angle(rng.normal(size=3), np.radians(10))
    g = K.random_rotation(3, 0)
    F_S, eps, sig = S.strain_stress(R, g, np.radians(20), traction_free=True)
    assert np.abs(eps).max() < 1e-15 and np.abs(sig).max() < 1e-3


def test_traction_free_and_tilt():
    g = K.random_rotation(5, 0)
    F = K.axis_angle([1, 2, 0], 0.05) @ (np.eye(3) + np.array([[2e-4, 1e-4, 0], [1e-4, -3e-4, 2e-4], [0, 2e-4, 1e-4]]))
    F = F / np.cbrt(np.linalg.det(F))
    F_S, eps, sig = S.strain_stress(F, g, np.radians(30), traction_free=True)
    assert abs(sig[2, 2]) < 1e-6 * np.abs(sig).max()
    assert np.allclose(sig, sig.T)
    # without the traction-free scale the strain rotates with the tilt (Eq. 14)
    _, e0, _ = S.strain_stress(F, g, 0.0, traction_free=False)
    _, e1, _ = S.strain_stress(F, g, np.radians(30), traction_free=False)
    T = S.tilt_matrix(np.radians(30))
    assert np.abs(e1 - T @ e0 @ T.T).max() < 1e-15
