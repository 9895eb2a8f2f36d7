"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4) and the
benchmark configurations: mesh descriptions, laser pulses, initial orbitals
and CI vectors.  Holds none of the method's arithmetic; both the CUDA path and
the CPU oracle draw their inputs from here.

Random numbers are functions of the support-point coordinates (a
counter-based hash), so two implementations that number their unknowns
differently still receive identical inputs.
"""
import math

import numpy as np

BASE_SEED = 2301

# Sec. 4 / workload sizes.  nuclei: (position, charge, refinement levels).
WORKLOADS = {
    # hydrogen atom, Q2, 8^3 coarse cells refined 3 levels toward the nucleus
    "hydrogen_q2": dict(lo=-20.0, hi=20.0, nc=8, p=2, c=2.0,
                        nuclei=[((0.0, 0.0, 0.0), 1.0, 3)],
                        n_orb=1, n_alpha=1, n_beta=0, dt=0.01, m=8, steps=100,
                        pulse=None),
    # H2 at R = 1.4 bohr along z, Q4, 20^3 coarse (h0 = 4), 5 levels at each nucleus
    "h2_q4": dict(lo=-40.0, hi=40.0, nc=20, p=4, c=2.0,
                  nuclei=[((0.0, 0.0, 0.7), 1.0, 5), ((0.0, 0.0, -0.7), 1.0, 5)],
                  n_orb=4, n_alpha=1, n_beta=1, dt=0.02, m=10, steps=500,
                  pulse=dict(intensity=1e14, wavelength_nm=800.0, cycles=3, pol=(0.0, 0.0, 1.0))),
    # water-shaped molecule, Q4, 32^3 coarse, 6 levels at O, 5 at each H
    "water_q4": dict(lo=-50.0, hi=50.0, nc=32, p=4, c=2.0,
                     nuclei=[((0.0, 0.0, 0.0), 8.0, 6),
                             ((1.4311, 1.1081, 0.0), 1.0, 5),
                             ((-1.4311, 1.1081, 0.0), 1.0, 5)],
                     n_orb=8, n_alpha=5, n_beta=5, dt=0.01, m=10, steps=1000,
                     pulse=dict(intensity=2e14, wavelength_nm=800.0, cycles=4, pol=(0.0, 0.0, 1.0))),
}

# Atomic-unit conversions for the pulse (peak field from intensity, photon energy).
_AU_INTENSITY_W_CM2 = 3.50945e16
_AU_ENERGY_NM = 45.5634


def mesh_args(name):
    w = WORKLOADS[name]
    return (w["lo"], w["hi"], w["nc"], w["p"], w["nuclei"], w["c"])


def sin2_pulse(t, intensity, wavelength_nm, cycles, pol):
    """E(t) = E0 sin^2(pi t / tau) sin(omega t) pol for 0 <= t <= tau, else 0."""
    E0 = math.sqrt(intensity / _AU_INTENSITY_W_CM2)
    omega = _AU_ENERGY_NM / wavelength_nm
    tau = cycles * 2.0 * math.pi / omega
    if t < 0.0 or t > tau:
        return (0.0, 0.0, 0.0)
    e = E0 * math.sin(math.pi * t / tau) ** 2 * math.sin(omega * t)
    return tuple(e * float(c) for c in pol)


def triangular_pulse(t, intensity, wavelength_nm, pol=(1.0, 0.0, 0.0)):
    """The paper's 2-cycle triangular-envelope pulse (Sec. 4)."""
    E0 = math.sqrt(intensity / _AU_INTENSITY_W_CM2)
    omega = _AU_ENERGY_NM / wavelength_nm
    ph = omega * t
    if ph < 0.0 or ph > 4.0 * math.pi:
        return (0.0, 0.0, 0.0)
    env = ph / (2 * math.pi) if ph <= 2 * math.pi else (4 * math.pi - ph) / (2 * math.pi)
    e = E0 * env * math.sin(ph)
    return tuple(e * float(c) for c in pol)


def triangular_vector_potential(t, intensity, wavelength_nm, pol=(1.0, 0.0, 0.0)):
    """A(t) = -int_-inf^t E of the triangular pulse (the velocity gauge's field
    input): with ph = omega t and int u sin u = sin u - u cos u,
    -A / (E0 / omega) = (sin ph - ph cos ph) / (2 pi) up to ph = 2 pi and
    (ph cos ph - 4 pi cos ph - sin ph) / (2 pi) up to 4 pi; 0 outside."""
    E0 = math.sqrt(intensity / _AU_INTENSITY_W_CM2)
    omega = _AU_ENERGY_NM / wavelength_nm
    ph = omega * t
    if ph <= 0.0 or ph >= 4.0 * math.pi:
        return (0.0, 0.0, 0.0)
    if ph <= 2 * math.pi:
        f = (math.sin(ph) - ph * math.cos(ph)) / (2 * math.pi)
    else:
        f = (ph * math.cos(ph) - 4 * math.pi * math.cos(ph) - math.sin(ph)) / (2 * math.pi)
    a = -E0 / omega * f
    return tuple(a * float(c) for c in pol)


def _splitmix64(x):
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = x
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    return z ^ (z >> np.uint64(31))


def coord_normal(X, seed, stream=0):
    """Standard normal numbers keyed by coordinates (N, 3): hash -> two uniforms -> Box-Muller."""
    q = np.round(np.asarray(X, dtype=np.float64) * 2.0 ** 20).astype(np.int64).view(np.uint64)
    with np.errstate(over="ignore"):
        h = np.full(len(q), np.uint64(seed * 1000003 + stream), dtype=np.uint64)
        for ax in range(3):
            h = _splitmix64(h ^ q[:, ax])
        h1 = _splitmix64(h)
        h2 = _splitmix64(h1)
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 0.5) / 2.0 ** 53
    u2 = ((h2 >> np.uint64(11)).astype(np.float64) + 0.5) / 2.0 ** 53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_orbital(X, interior, center=(0.0, 0.0, 0.0), alpha=1.0, phase_noise=1e-3, seed=BASE_SEED):
    """exp(-alpha |x - c|^2) exp(i theta), theta ~ N(0, phase_noise^2) per point; zero on the surface."""
    c = np.asarray(center, dtype=np.float64)
    amp = np.exp(-alpha * np.sum((X - c) ** 2, axis=1))
    theta = phase_noise * coord_normal(X, seed)
    return np.where(interior, amp * np.exp(1j * theta), 0.0)


def molecular_orbitals(X, interior, nuclei, n, seed=BASE_SEED, phase_noise=1e-3):
    """n seeded Gaussian / 1s-like orbitals on the nuclei (not yet orthonormal).

    Orbital j sits on nucleus j mod n_nuclei with exponent 0.5 + 0.4 j / n and a
    small seeded displacement, times a polynomial factor (1, x, y, z, ...) of
    the displacement so that the set is linearly independent; phase_noise is
    the standard deviation of a per-point random phase (0 for smooth orbitals).
    """
    out = np.zeros((len(X), n), dtype=np.complex128)
    rng = np.random.default_rng(seed)
    for j in range(n):
        R = np.asarray(nuclei[j % len(nuclei)][0], dtype=np.float64) + 0.05 * rng.standard_normal(3)
        d = X - R
        alpha = 0.5 + 0.4 * j / max(n, 1)
        poly = np.ones(len(X)) if j < len(nuclei) else d[:, (j - len(nuclei)) % 3]
        theta = phase_noise * coord_normal(X, seed, stream=j + 1) if phase_noise else 0.0
        out[:, j] = poly * np.exp(-alpha * np.sum(d * d, axis=1)) * np.exp(1j * theta)
    out[~interior] = 0
    return out


def lowdin(phi, ml):
    """Symmetric orthonormalisation phi S^{-1/2}, S = phi^H diag(ml) phi (input preparation)."""
    S = np.conj(phi).T @ (ml[:, None] * phi)
    w, V = np.linalg.eigh(S)
    return phi @ (V @ np.diag(w ** -0.5) @ V.conj().T)


def initial_ci(n_orb, n_alpha, n_beta, seed=BASE_SEED, amp=1e-2):
    """CI vector: the lowest determinant (first orbitals occupied) plus seeded
    amplitudes `amp` on every other determinant, normalised; determinants are
    ordered as (alpha string, beta string) with strings in ascending bit-mask order."""
    from itertools import combinations
    na_str = len(list(combinations(range(n_orb), n_alpha)))
    nb_str = len(list(combinations(range(n_orb), n_beta)))
    rng = np.random.default_rng(seed)
    C = amp * (rng.standard_normal(na_str * nb_str) + 1j * rng.standard_normal(na_str * nb_str))
    C[0] = 1.0
    return C / np.linalg.norm(C)


def batch_instances(count=64, seed=BASE_SEED, dof_range=(5e4, 2e6), box=30.0):
    """Seeded instances of the batching form: target DoF counts log-uniform in
    dof_range, degree p in {2, 3, 4}, 1-3 nuclei with Z in 1..8 uniformly within
    3 bohr of the origin (2 refinement levels each), an orbital count in 1..8,
    and a field of
    amplitude uniform in [0.01, 0.08] along a random direction.  The coarse
    count n_c = round(N_target^(1/3) / p) (at least 2) sets the size; the
    refinement adds a few percent.  Returns a list of dicts with mesh_args,
    n_orb and E."""
    rng = np.random.default_rng(seed + 7)
    out = []
    for i in range(count):
        target = float(np.exp(rng.uniform(np.log(dof_range[0]), np.log(dof_range[1]))))
        p = int(rng.integers(2, 5))
        nc = max(2, int(round(target ** (1.0 / 3.0) / p)))
        nnuc = int(rng.integers(1, 4))
        nuclei = []
        for _ in range(nnuc):
            d = rng.standard_normal(3)
            d *= rng.uniform(0.0, 3.0) / max(np.linalg.norm(d), 1e-12)
            nuclei.append(((float(d[0]), float(d[1]), float(d[2])), float(rng.integers(1, 9)), 2))
        n_orb = int(rng.integers(1, 9))
        e = rng.standard_normal(3)
        e *= rng.uniform(0.01, 0.08) / np.linalg.norm(e)
        out.append(dict(mesh_args=(-box, box, nc, p, nuclei, 2.0), n_orb=n_orb, E=tuple(float(v) for v in e),
                        target_dofs=target))
    return out
