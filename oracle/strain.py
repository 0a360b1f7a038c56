"""FP64 numpy oracle of the strain/stress post-processing -- TEST INFRASTRUCTURE.

Follows Eq. 13-16 and Supplementary Part 2 of the paper: the detector-frame
deformation gradient is brought to the sample frame (Eq. 13-14), the strain is
epsilon = 1/2 (F F^T - I) (Eq. 15, first form: it removes the finite rotation
exactly), and the stress is sigma = C : epsilon (Eq. 16) with the cubic
stiffness rotated from the crystal to the sample frame by the passive
orientation matrix g (sample -> crystal; Supp. Eq. 2.4-2.5: T_S = g^T T_C g).
The 4th-order tensor is rotated and contracted directly (no Voigt matrices).

Readings: Eq. 13 is used as printed (a rotation by theta_tilt in the first two
axes).  The deformation gradient of Eq. 3 is known up to its scale; with
``traction_free`` the scale lambda is the one that makes sigma_33 = 0 (the
traction-free condition of Eq. 16 on the normal component): with
epsilon(lambda) = 1/2 (lambda^2 F F^T - I) this is linear in lambda^2.
Only the tests may import this module.
"""
from __future__ import annotations

import numpy as np

NI_C = (276e9, 159e9, 132e9)   # C11, C12, C44 of nickel in Pa (Section 2)


def tilt_matrix(theta):
    """Eq. 13."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])


def to_sample(F, theta):
    """Eq. 14: F_S = R F R^T."""
    R = tilt_matrix(theta)
    return R @ F @ R.T


def cubic_stiffness(c11, c12, c44):
    """C_ijkl of a cubic crystal in its own axes."""
    d = np.eye(3)
    C = (c12 * np.einsum("ij,kl->ijkl", d, d)
         + c44 * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))
    for p in range(3):
        C[p, p, p, p] += c11 - c12 - 2 * c44
    return C


def rotate_stiffness(C, g):
    """Stiffness in the sample frame: C_S = g^T . C . g on every index (g: sample -> crystal)."""
    a = g.T   # crystal -> sample
    return np.einsum("ip,jq,kr,ls,pqrs->ijkl", a, a, a, a, C)


def strain(F_S):
    """Eq. 15: 1/2 (F F^T - I)."""
    return 0.5 * (F_S @ F_S.T - np.eye(3))


def stress(C_S, eps):
    """Eq. 16: sigma = C : epsilon."""
    return np.einsum("ijkl,kl->ij", C_S, eps)


def traction_free_scale(F_S, C_S):
    """lambda with sigma_33(1/2 (lambda^2 F F^T - I)) = 0."""
    a = stress(C_S, 0.5 * F_S @ F_S.T)[2, 2]
    b = stress(C_S, 0.5 * np.eye(3))[2, 2]
    return np.sqrt(b / a)


def strain_stress(F, g, theta, C=NI_C, traction_free=True):
    """(F_S, epsilon_S, sigma_S) of one scan point."""
    F_S = to_sample(np.asarray(F, dtype=np.float64), theta)
    C_S = rotate_stiffness(cubic_stiffness(*C), np.asarray(g, dtype=np.float64))
    if traction_free:
        F_S = traction_free_scale(F_S, C_S) * F_S
    eps = strain(F_S)
    return F_S, eps, stress(C_S, eps)
