"""Seeded synthetic Kikuchi patterns (input generator, CPU / numpy).

The paper evaluates its method on EMsoft dynamical simulations of FCC nickel
(Section 3.1) and on experimental scans; neither is available here, so every
input of the tests and the benchmark comes from this kinematic generator.
It holds none of the registration / fitting arithmetic of the method: it only
renders patterns for a known crystal orientation and deformation gradient.

Recipe (one pattern):
  * FCC lattice, a = 3.6 Angstrom; band families {111}, {200}, {220}, {311}
    (25 planes, each counted once up to sign).
  * Reciprocal vector of plane hkl in the detector frame: G = g (h,k,l)/a,
    with g the crystal-to-detector rotation.  A deformed crystal with
    deformation gradient F (detector frame) has G' = F^-T G, so that the
    detector direction r of a band point moves to F r (the forward model of
    Eq. 2).
  * Gnomonic projection: pixel (i, j) has centre x = j + 0.5, y = i + 0.5
    (rows downward); its direction from the source point is
    r = (x - xstar*W, y - ystar*H, zstar*W).
  * Band profile exp(-theta^2 / (2 theta_B^2)), theta = asin(G'.r / |G'||r|),
    theta_B = asin(lambda |G'| / 2) the Bragg angle at 20 kV (relativistic
    electron wavelength), amplitude 3/(h^2+k^2+l^2).
  * Quadratic background 1 - 0.3 (xd^2 + yd^2) + 0.05 yd on detector
    coordinates xd, yd in [-1, 1]; intensity bg * (1 + 0.5 sum of bands),
    scaled to a mean of `counts`.
  * Noise: counts drawn per pixel as round(l + sqrt(l) z + (z^2 - 1)/6), the
    Poisson(l) variate approximated by its first-order Cornish-Fisher
    expansion (z standard normal by Box-Muller); exact enough for l >= 50,
    which all configurations satisfy (mean 200 or 500 counts).
  * Random numbers: SplitMix64 (Vigna) finaliser on (seed, stream, counter),
    so that any single pattern of a scan can be rendered on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_KSTREAM = np.uint64(0xD1B54A32D192ED03)
_KCTR = np.uint64(0x632BE59BD9B4E019)

# stream purposes (stream id = 16 * object id + purpose)
P_REF_ORI, P_MIS_AXIS, P_MIS_ANGLE, P_STRAIN, P_NOISE = 0, 1, 2, 3, 4


def _mix(z):
    """SplitMix64 output function (Vigna), on uint64 arrays (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLD
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return _mix(_mix(np.uint64(seed)) + np.uint64(stream) * _KSTREAM)


def uniforms(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) from counters start..start+n-1 of one stream."""
    key = stream_key(seed, stream)
    ctr = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        bits = _mix(key + ctr * _KCTR)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n standard normals (Box-Muller, cosine branch) from 2n uniforms."""
    u = uniforms(seed, stream, 2 * n, 2 * start)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------- rotations
def quat_to_matrix(q) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def random_rotation(seed: int, stream: int) -> np.ndarray:
    """Uniform rotation on SO(3) (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = uniforms(seed, stream, 3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    q = (b * math.cos(2 * math.pi * u3), a * math.sin(2 * math.pi * u2),
         a * math.cos(2 * math.pi * u2), b * math.sin(2 * math.pi * u3))
    return quat_to_matrix(q)


def random_axis(seed: int, stream: int) -> np.ndarray:
    u1, u2 = uniforms(seed, stream, 2)
    z = 2.0 * u1 - 1.0
    s = math.sqrt(max(0.0, 1.0 - z * z))
    return np.array([s * math.cos(2 * math.pi * u2), s * math.sin(2 * math.pi * u2), z])


def axis_angle(axis, angle_rad: float) -> np.ndarray:
    """Rodrigues' rotation formula."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle_rad) * K + (1 - math.cos(angle_rad)) * (K @ K)


# ---------------------------------------------------------------- crystal
def fcc_planes() -> np.ndarray:
    """Unique (up to sign) plane indices of {111},{200},{220},{311}."""
    out = []
    seen = set()
    for fam in ((1, 1, 1), (2, 0, 0), (2, 2, 0), (3, 1, 1)):
        import itertools
        for perm in set(itertools.permutations(fam)):
            for sgn in itertools.product((1, -1), repeat=3):
                v = tuple(p * s for p, s in zip(perm, sgn))
                if v == (0, 0, 0):
                    continue
                neg = tuple(-c for c in v)
                if v in seen or neg in seen:
                    continue
                seen.add(v)
                out.append(v)
    return np.array(sorted(out), dtype=np.float64)


def electron_wavelength_angstrom(kv: float) -> float:
    h, m0, e, c = 6.62607015e-34, 9.1093837015e-31, 1.602176634e-19, 299792458.0
    V = kv * 1e3
    lam = h / math.sqrt(2 * m0 * e * V * (1 + e * V / (2 * m0 * c * c)))
    return lam * 1e10


LATTICE_A = 3.6
KV = 20.0


@dataclass(frozen=True)
class Geometry:
    xstar: float = 0.5
    ystar: float = 0.5
    zstar: float = 0.6


def pixel_directions(H: int, W: int, geom: Geometry, pc_shift=(0.0, 0.0)) -> np.ndarray:
    """Unit directions [H*W, 3] of the pixel centres."""
    x = np.arange(W, dtype=np.float64) + 0.5 - geom.xstar * W - pc_shift[0]
    y = np.arange(H, dtype=np.float64) + 0.5 - geom.ystar * H - pc_shift[1]
    X, Y = np.meshgrid(x, y)
    Z = np.full_like(X, geom.zstar * W)
    d = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def render(g: np.ndarray, F: np.ndarray, H: int, W: int, geom: Geometry = Geometry(),
           counts: float = 500.0, noise: bool = True, seed: int = 0, stream: int = 0,
           background: bool = True, pc_shift=(0.0, 0.0)) -> np.ndarray:
    """Render one pattern [H, W] float32 for orientation g and deformation F."""
    hkl = fcc_planes()
    G = (g @ (hkl / LATTICE_A).T).T                     # detector frame [P, 3]
    G = (np.linalg.inv(F).T @ G.T).T                    # deformed: F^-T G
    gn = np.linalg.norm(G, axis=1)
    lam = electron_wavelength_angstrom(KV)
    theta_b = np.arcsin(lam * gn / 2.0)
    amp = 3.0 / np.sum(hkl * hkl, axis=1)
    d = pixel_directions(H, W, geom, pc_shift)
    s = np.clip(d @ (G / gn[:, None]).T, -1.0, 1.0)     # [HW, P]
    th = np.arcsin(s)
    bands = np.exp(-(th * th) / (2.0 * theta_b * theta_b)) @ amp
    if background:
        xd = (np.arange(W) + 0.5) / W * 2.0 - 1.0
        yd = (np.arange(H) + 0.5) / H * 2.0 - 1.0
        XD, YD = np.meshgrid(xd, yd)
        bg = (1.0 - 0.3 * (XD * XD + YD * YD) + 0.05 * YD).reshape(-1)
    else:
        bg = np.ones(H * W)
    img = bg * (1.0 + 0.5 * bands)
    lam_px = img * (counts / img.mean())
    if noise:
        z = normals(seed, stream, H * W)
        k = np.rint(lam_px + np.sqrt(lam_px) * z + (z * z - 1.0) / 6.0)
        img = np.maximum(k, 0.0)
    else:
        img = lam_px
    return img.reshape(H, W).astype(np.float32)


# ---------------------------------------------------------------- scans
@dataclass(frozen=True)
class ScanSpec:
    """A seeded scan: n_pairs test patterns against n_refs grain references.

    strain_mode 'norm': symmetric strain of Frobenius norm `strain`;
    'sigma': each independent component ~ N(0, strain).
    """
    n_pairs: int
    H: int
    W: int
    n_refs: int = 1
    mis_lo_deg: float = 0.0
    mis_hi_deg: float = 6.0
    strain: float = 5e-4
    strain_mode: str = "sigma"
    counts: float = 500.0
    seed: int = 1
    geom: Geometry = field(default_factory=Geometry)
    fixed_mis_deg: float | None = None


def ref_orientation(spec: ScanSpec, r: int) -> np.ndarray:
    return random_rotation(spec.seed, 16 * (1_000_000 + r) + P_REF_ORI)


def pair_truth(spec: ScanSpec, p: int) -> np.ndarray:
    """Deformation gradient F = R_mis (I + eps) of pair p (detector frame)."""
    axis = random_axis(spec.seed, 16 * p + P_MIS_AXIS)
    if spec.fixed_mis_deg is not None:
        ang = spec.fixed_mis_deg
    else:
        (u,) = uniforms(spec.seed, 16 * p + P_MIS_ANGLE, 1)
        ang = spec.mis_lo_deg + (spec.mis_hi_deg - spec.mis_lo_deg) * u
    Rm = axis_angle(axis, math.radians(ang))
    z = normals(spec.seed, 16 * p + P_STRAIN, 6)
    E = np.array([[z[0], z[3], z[4]], [z[3], z[1], z[5]], [z[4], z[5], z[2]]])
    if spec.strain_mode == "norm":
        E = E * (spec.strain / np.linalg.norm(E))
    else:
        E = E * spec.strain
    return Rm @ (np.eye(3) + E)


def ref_index(spec: ScanSpec, p: int) -> int:
    """Grain of scan point p: the scan is a square grid cut into n_refs vertical strips
    (with as many references as pairs, every pair has its own)."""
    if spec.n_refs >= spec.n_pairs:
        return p
    side = int(math.isqrt(spec.n_pairs))
    if side * side != spec.n_pairs or spec.n_refs == 1:
        return p % spec.n_refs
    col = p % side
    return min(spec.n_refs - 1, col * spec.n_refs // side)


def render_ref(spec: ScanSpec, r: int, noise: bool = True) -> np.ndarray:
    return render(ref_orientation(spec, r), np.eye(3), spec.H, spec.W, spec.geom,
                  spec.counts, noise, spec.seed, 16 * (1_000_000 + r) + P_NOISE)


def render_test(spec: ScanSpec, p: int, noise: bool = True) -> np.ndarray:
    r = ref_index(spec, p)
    return render(ref_orientation(spec, r), pair_truth(spec, p), spec.H, spec.W, spec.geom,
                  spec.counts, noise, spec.seed, 16 * p + P_NOISE)


def make_scan(spec: ScanSpec, pairs=None, noise: bool = True):
    """Return (refs [R,H,W], tests [len(pairs),H,W], ref_idx, F_true [n,3,3])."""
    if pairs is None:
        pairs = range(spec.n_pairs)
    pairs = list(pairs)
    refs = np.stack([render_ref(spec, r, noise) for r in range(spec.n_refs)])
    tests = np.stack([render_test(spec, p, noise) for p in pairs]) if pairs else \
        np.zeros((0, spec.H, spec.W), np.float32)
    ridx = np.array([ref_index(spec, p) for p in pairs], dtype=np.int32)
    Ft = np.stack([pair_truth(spec, p) for p in pairs]) if pairs else np.zeros((0, 3, 3))
    return refs, tests, ridx, Ft


# The five workloads (sizes as stated by the method's evaluation plan).
def config1() -> ScanSpec:
    """Single pair 128x128, 2 deg about a random axis, strain norm 1e-4."""
    return ScanSpec(n_pairs=1, H=128, W=128, n_refs=1, fixed_mis_deg=2.0, strain=1e-4,
                    strain_mode="norm", counts=500.0, seed=1)


def config2(n_pairs: int = 10_000) -> ScanSpec:
    """Batched scan 100x100 at 256x256, 4 grains, mis U(0,6) deg, strain N(0,5e-4)."""
    return ScanSpec(n_pairs=n_pairs, H=256, W=256, n_refs=4, mis_lo_deg=0.0, mis_hi_deg=6.0,
                    strain=5e-4, strain_mode="sigma", counts=500.0, seed=2)


def config3(n_pairs: int = 20_000) -> ScanSpec:
    """Large-misorientation scan at 256x256, mis U(6,12) deg, 200 counts."""
    return ScanSpec(n_pairs=n_pairs, H=256, W=256, n_refs=4, mis_lo_deg=6.0, mis_hi_deg=12.0,
                    strain=5e-4, strain_mode="sigma", counts=200.0, seed=3)


def config4(n_pairs: int = 200_000) -> ScanSpec:
    """Training pairs of the learned initialiser: as the single pair (128x128, strain norm
    1e-4, 500 counts) with misorientation U(0, 12) deg, one reference orientation per pair."""
    return ScanSpec(n_pairs=n_pairs, H=128, W=128, n_refs=n_pairs, mis_lo_deg=0.0, mis_hi_deg=12.0, strain=1e-4,
                    strain_mode="norm", counts=500.0, seed=4)


def config5(n_pairs: int = 160_000) -> ScanSpec:
    """Learned-init vs plain scan 400x400 at 256x256, 8 grains, mis U(0,12) deg."""
    return ScanSpec(n_pairs=n_pairs, H=256, W=256, n_refs=8, mis_lo_deg=0.0, mis_hi_deg=12.0,
                    strain=5e-4, strain_mode="sigma", counts=500.0, seed=5)


def roi_grid(H: int, W: int, S: int, drop_corners: bool) -> np.ndarray:
    """ROI centres (continuous pixel coordinates) on a 5x5 grid.

    128x128 with 32x32 ROIs: centres 24 + 20k; 256x256 with 64x64: 48 + 40k.
    The four corners are dropped for the 21-ROI layout.
    """
    step = (W - 2 * (S // 2 + S // 4)) // 4
    c0 = S // 2 + S // 4
    out = []
    for a in range(5):
        for b in range(5):
            if drop_corners and a in (0, 4) and b in (0, 4):
                continue
            out.append((c0 + b * step, c0 + a * step))
    return np.array(out, dtype=np.int32)


def roi_grid_n(H: int, W: int, S: int, n: int) -> np.ndarray:
    """n x n ROI centres (continuous pixel coordinates) spread evenly over the pattern with every S x S
    ROI inside it (the paper's 100 ROIs of 256 x 256 on 1244 x 1024 simulations: n = 10)."""
    xs = np.rint(np.linspace(S // 2, W - S // 2, n)).astype(np.int32)
    ys = np.rint(np.linspace(S // 2, H - S // 2, n)).astype(np.int32)
    return np.array([(x, y) for y in ys for x in xs], dtype=np.int32)
