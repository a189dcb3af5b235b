"""Seeded synthetic particle sets for the oct-tree gravity path.

This module only draws inputs: positions (float64), velocities (float64) and
masses (float32).  It holds none of the tree method's arithmetic, so both the
CPU oracle tests and the GPU path (tests and benchmark) may use it.

The paper's own workloads are a random sphere (Sec. "Test and Optimization"),
a random cube (Sec. "Fast Multipole Method on GPU") and a cosmological sphere
of N = 2,874,551 particles built from COSMICS initial conditions (Sec.
"Cosmological Simulation").  COSMICS output is not available, so the clustered
generators below stand in for it: uniform background, Gaussian-random-field
displacements and embedded NFW halos, with the particle counts, theta and
softening of that run.

Units: G = 1, total mass 1.  Every generator takes an integer seed and is
deterministic for a given (seed, arguments) on any machine (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20090909

__all__ = [
    "ParticleSet", "plummer", "hernquist", "uniform_sphere", "uniform_cube",
    "nfw_halo", "clustered_cosmo", "halo_mix", "batched_systems",
    "two_body", "workload",
]


@dataclass
class ParticleSet:
    pos: np.ndarray    # (n, 3) float64
    vel: np.ndarray    # (n, 3) float64
    mass: np.ndarray   # (n,) float32
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(ph), rxy * np.sin(ph), z], axis=1)


def _equal_masses(n: int, total: float = 1.0) -> np.ndarray:
    return np.full(n, total / max(n, 1), dtype=np.float32)


def plummer(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0,
            rmax: float = 20.0) -> ParticleSet:
    """Plummer sphere with isotropic velocities.

    Radii by inverting M(<r) = M r^3 / (r^2 + a^2)^{3/2}, redrawn above rmax;
    speeds by the Aarseth-Henon-Wielen (1974) rejection on
    g(q) = q^2 (1 - q^2)^{7/2}, q = v / v_esc.
    """
    rng = _rng(seed)
    r = np.empty(0)
    while r.size < n:
        u = rng.uniform(0.0, 1.0, 2 * (n - r.size) + 16)
        u = u[(u > 0.0)]
        rr = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= rmax]])
    r = r[:n]
    pos = r[:, None] * _unit_vectors(rng, n)
    q = np.empty(0)
    while q.size < n:
        x1 = rng.uniform(0.0, 1.0, 2 * (n - q.size) + 16)
        x2 = rng.uniform(0.0, 1.0, x1.size)
        keep = 0.1 * x2 < x1 * x1 * (1.0 - x1 * x1) ** 3.5
        q = np.concatenate([q, x1[keep]])
    q = q[:n]
    vesc = math.sqrt(2.0 * total_mass / a) * (1.0 + (r / a) ** 2) ** -0.25
    vel = (q * vesc)[:, None] * _unit_vectors(rng, n)
    return ParticleSet(pos, vel, _equal_masses(n, total_mass), f"plummer{n}")


def _hernquist_sigma2(r: np.ndarray) -> np.ndarray:
    # isotropic 1-D velocity dispersion of a G = M = a = 1 Hernquist sphere
    # (Hernquist 1990, ApJ 356, 359, eq. 10)
    t = 12.0 * r * (1.0 + r) ** 3 * np.log1p(1.0 / r)
    u = r / (1.0 + r) * (25.0 + 52.0 * r + 42.0 * r * r + 12.0 * r ** 3)
    return np.maximum((t - u) / 12.0, 0.0)


def hernquist(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0,
              rmax: float = 20.0) -> ParticleSet:
    """Hernquist sphere: r = a sqrt(u) / (1 - sqrt(u)), redrawn above rmax;
    isotropic Gaussian velocities with the Jeans dispersion, capped below
    0.95 of the local escape speed."""
    rng = _rng(seed)
    r = np.empty(0)
    while r.size < n:
        u = rng.uniform(0.0, 1.0, 2 * (n - r.size) + 16)
        su = np.sqrt(u)
        su = su[su < 1.0]
        rr = a * su / (1.0 - su)
        r = np.concatenate([r, rr[(rr <= rmax) & (rr > 0)]])
    r = r[:n]
    pos = r[:, None] * _unit_vectors(rng, n)
    scale = math.sqrt(total_mass / a)
    sig = np.sqrt(_hernquist_sigma2(r / a)) * scale
    vel = rng.normal(size=(n, 3)) * sig[:, None]
    vesc = np.sqrt(2.0 * total_mass / (r + a))
    sp = np.linalg.norm(vel, axis=1)
    cap = 0.95 * vesc
    over = sp > cap
    vel[over] *= (cap[over] / sp[over])[:, None]
    return ParticleSet(pos, vel, _equal_masses(n, total_mass), f"hernquist{n}")


def uniform_sphere(n: int, seed: int, radius: float = 1.0,
                   total_mass: float = 1.0) -> ParticleSet:
    """Random points in a sphere (the paper's basic test set)."""
    rng = _rng(seed)
    r = radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = r[:, None] * _unit_vectors(rng, n)
    return ParticleSet(pos, np.zeros((n, 3)), _equal_masses(n, total_mass),
                       f"usphere{n}")


def uniform_cube(n: int, seed: int, side: float = 1.0,
                 total_mass: float = 1.0) -> ParticleSet:
    """Random points in a cube (the paper's comparison with GPU FMM)."""
    rng = _rng(seed)
    pos = rng.uniform(-0.5 * side, 0.5 * side, (n, 3))
    return ParticleSet(pos, np.zeros((n, 3)), _equal_masses(n, total_mass),
                       f"ucube{n}")


def _nfw_radii(rng: np.random.Generator, n: int, rvir: float,
               conc: float) -> np.ndarray:
    # inverse of the truncated NFW enclosed-mass profile mu(x) = ln(1+x) - x/(1+x)
    x = np.concatenate([[0.0], np.geomspace(1e-6 * conc, conc, 2048)])
    mu = np.log1p(x) - x / (1.0 + x)
    u = rng.uniform(0.0, mu[-1], n)
    return np.interp(u, mu, x) * (rvir / conc)


def nfw_halo(n: int, seed: int, rvir: float = 1.0, conc: float = 10.0,
             total_mass: float = 1.0) -> ParticleSet:
    rng = _rng(seed)
    r = _nfw_radii(rng, n, rvir, conc)
    pos = r[:, None] * _unit_vectors(rng, n)
    return ParticleSet(pos, np.zeros((n, 3)), _equal_masses(n, total_mass),
                       f"nfw{n}")


def _grf_displacement(rng: np.random.Generator, pts: np.ndarray, rms: float,
                      ngrid: int = 128, box: float = 2.2,
                      index: float = -2.0) -> np.ndarray:
    """Zel'dovich-style displacement of a Gaussian random field with
    P(k) ~ k^index on an ngrid^3 periodic grid of side `box`, trilinearly
    interpolated at pts and scaled to a 3-D rms of `rms`."""
    k1 = np.fft.fftfreq(ngrid, d=box / ngrid) * 2.0 * math.pi
    kz1 = np.fft.rfftfreq(ngrid, d=box / ngrid) * 2.0 * math.pi
    kx, ky, kz = np.meshgrid(k1, k1, kz1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = np.sqrt(k2 ** (0.5 * index))
    amp[0, 0, 0] = 0.0
    noise = (rng.normal(size=k2.shape) + 1j * rng.normal(size=k2.shape))
    delta = noise * amp
    disp = []
    for kc in (kx, ky, kz):
        psi_k = 1j * kc / k2 * delta
        disp.append(np.fft.irfftn(psi_k, s=(ngrid, ngrid, ngrid), axes=(0, 1, 2)))
    disp = np.stack(disp, axis=-1)               # (g, g, g, 3)
    # trilinear interpolation, periodic
    f = (pts / box + 0.5) * ngrid
    i0 = np.floor(f).astype(np.int64)
    w = f - i0
    out = np.zeros_like(pts)
    for dx in (0, 1):
        wx = w[:, 0] if dx else 1.0 - w[:, 0]
        ix = (i0[:, 0] + dx) % ngrid
        for dy in (0, 1):
            wy = w[:, 1] if dy else 1.0 - w[:, 1]
            iy = (i0[:, 1] + dy) % ngrid
            for dz in (0, 1):
                wz = w[:, 2] if dz else 1.0 - w[:, 2]
                iz = (i0[:, 2] + dz) % ngrid
                out += (wx * wy * wz)[:, None] * disp[ix, iy, iz]
    cur = math.sqrt(float(np.mean(np.sum(out * out, axis=1))))
    return out * (rms / cur if cur > 0 else 0.0)


def _halo_particles(rng, counts, rvirs, concs, centres):
    chunks = []
    for k in range(len(counts)):
        m = int(counts[k])
        if m == 0:
            continue
        r = _nfw_radii(rng, m, float(rvirs[k]), float(concs[k]))
        chunks.append(centres[k] + r[:, None] * _unit_vectors(rng, m))
    return np.concatenate(chunks) if chunks else np.zeros((0, 3))


def _split_counts(n_total: int, weights: np.ndarray) -> np.ndarray:
    raw = n_total * weights / weights.sum()
    cnt = np.floor(raw).astype(np.int64)
    rest = n_total - int(cnt.sum())
    if rest > 0:
        order = np.argsort(-(raw - cnt), kind="stable")
        cnt[order[:rest]] += 1
    return cnt


def clustered_cosmo(n: int = 1 << 21, seed: int = BASE_SEED + 2,
                    n_halos: int = 500, conc: float = 10.0,
                    mlo: float = 1e-5, mhi: float = 1e-3,
                    rms_disp: float = 0.02) -> ParticleSet:
    """Clustered cosmological-like set in a unit sphere: uniform points with
    Gaussian-random-field displacements (P(k) ~ k^-2, rms 0.02) plus n_halos
    NFW halos (concentration `conc`, masses log-uniform in [mlo, mhi] of the
    total, r_vir = (M / 200)^{1/3}), equal particle masses."""
    rng = _rng(seed)
    mh = np.exp(rng.uniform(math.log(mlo), math.log(mhi), n_halos))
    counts = np.round(mh * n).astype(np.int64)
    n_bg = n - int(counts.sum())
    if n_bg < 0:
        raise ValueError("halo masses exceed the particle budget")
    centres = rng.uniform(0.0, 1.0, n_halos) ** (1.0 / 3.0)
    centres = centres[:, None] * _unit_vectors(rng, n_halos)
    rvir = (mh / 200.0) ** (1.0 / 3.0)
    bg = (rng.uniform(0.0, 1.0, n_bg) ** (1.0 / 3.0))[:, None] * _unit_vectors(rng, n_bg)
    bg = bg + _grf_displacement(rng, bg, rms_disp)
    halos = _halo_particles(rng, counts, rvir, np.full(n_halos, conc), centres)
    pos = np.concatenate([bg, halos])
    perm = rng.permutation(n)
    pos = np.ascontiguousarray(pos[perm])
    return ParticleSet(pos, np.zeros((n, 3)), _equal_masses(n), f"cosmo{n}")


def halo_mix(n: int = 2_870_000, seed: int = BASE_SEED + 4, n_halos: int = 2000,
             slope: float = -1.9, mlo: float = 1e-6, mhi: float = 1e-2,
             halo_fraction: float = 0.8, clo: float = 5.0,
             chi: float = 15.0) -> ParticleSet:
    """Sum of NFW halos (mass function dN/dM ~ M^slope on [mlo, mhi], scaled
    to `halo_fraction` of the mass, concentration uniform in [clo, chi],
    r_vir = (M/200)^{1/3}) plus a uniform background in a unit sphere."""
    rng = _rng(seed)
    g = slope + 1.0
    u = rng.uniform(0.0, 1.0, n_halos)
    mh = (mlo ** g + u * (mhi ** g - mlo ** g)) ** (1.0 / g)
    mh = mh * (halo_fraction / mh.sum())
    n_halo_total = int(round(halo_fraction * n))
    counts = _split_counts(n_halo_total, mh)
    n_bg = n - n_halo_total
    concs = rng.uniform(clo, chi, n_halos)
    centres = rng.uniform(0.0, 1.0, n_halos) ** (1.0 / 3.0)
    centres = centres[:, None] * _unit_vectors(rng, n_halos)
    rvir = (mh / 200.0) ** (1.0 / 3.0)
    bg = (rng.uniform(0.0, 1.0, n_bg) ** (1.0 / 3.0))[:, None] * _unit_vectors(rng, n_bg)
    halos = _halo_particles(rng, counts, rvir, concs, centres)
    pos = np.concatenate([bg, halos])
    perm = rng.permutation(n)
    pos = np.ascontiguousarray(pos[perm])
    return ParticleSet(pos, np.zeros((n, 3)), _equal_masses(n), f"halomix{n}")


def batched_systems(n_systems: int = 512, seed: int = BASE_SEED + 3,
                    nmin: int = 1024, nmax: int = 65536):
    """Independent Plummer / Hernquist systems with N log-uniform in
    [nmin, nmax]; even index Plummer, odd index Hernquist."""
    rng = _rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_systems))
    ns = np.round(ns).astype(np.int64)
    out = []
    for k in range(n_systems):
        s = int(rng.integers(0, 2**31 - 1))
        gen = plummer if k % 2 == 0 else hernquist
        out.append(gen(int(ns[k]), s))
    return out


def two_body(sep: float, m1: float = 0.5, m2: float = 0.5,
             circular: bool = True) -> ParticleSet:
    """Two bodies on the x axis about their centre of mass; with
    circular=True their velocities give a circular orbit (G = 1)."""
    mt = m1 + m2
    pos = np.array([[-sep * m2 / mt, 0.0, 0.0], [sep * m1 / mt, 0.0, 0.0]])
    vel = np.zeros((2, 3))
    if circular:
        vrel = math.sqrt(mt / sep)
        vel[0, 1] = -vrel * m2 / mt
        vel[1, 1] = vrel * m1 / mt
    return ParticleSet(pos, vel, np.array([m1, m2], dtype=np.float32), "twobody")


def mlp_initial_weights(seed: int, n_in: int = 12, hidden: int = 64) -> dict:
    """Seeded random draws for the learned-theta network's initial weights
    (He-style normal draws; zero biases): W1 (hidden, n_in), W2, W3 (hidden,
    hidden), w4 (hidden,).  Only random numbers: the network is elsewhere."""
    rng = _rng(seed)
    return dict(W1=rng.normal(0.0, math.sqrt(2.0 / n_in), (hidden, n_in)),
                W2=rng.normal(0.0, math.sqrt(2.0 / hidden), (hidden, hidden)),
                W3=rng.normal(0.0, math.sqrt(2.0 / hidden), (hidden, hidden)),
                w4=rng.normal(0.0, math.sqrt(1.0 / hidden), hidden),
                b1=np.zeros(hidden), b2=np.zeros(hidden), b3=np.zeros(hidden), b4=0.0)


# Named workloads with their method parameters (softening eps, opening angle
# theta, group size n_crit, time step dt).
WORKLOADS = {
    "plummer16k": dict(gen=lambda: plummer(16384, BASE_SEED + 1), eps=1.0 / 64,
                       theta=0.75, n_crit=64, dt=1.0 / 128),
    "cosmo2m": dict(gen=lambda: clustered_cosmo(1 << 21, BASE_SEED + 2), eps=1e-3,
                    theta=0.75, n_crit=256, dt=1.0 / 1024),
    "halomix2.87m": dict(gen=lambda: halo_mix(2_870_000, BASE_SEED + 4), eps=5e-4,
                         theta=0.6, n_crit=256, dt=1.0 / 1024),
    "halomix0.5m": dict(gen=lambda: halo_mix(500_000, BASE_SEED + 6, n_halos=350),
                        eps=5e-4, theta=0.6, n_crit=256, dt=1.0 / 1024),
    "halomix4.19m": dict(gen=lambda: halo_mix(4_194_304, BASE_SEED + 5,
                                              n_halos=3000), eps=5e-4,
                         theta=0.6, n_crit=256, dt=1.0 / 1024),
    # the same mix at larger N (halo count in proportion), for size sweeps
    "halomix8m": dict(gen=lambda: halo_mix(8_000_000, BASE_SEED + 7, n_halos=5575),
                      eps=5e-4, theta=0.6, n_crit=256, dt=1.0 / 1024),
    "halomix16m": dict(gen=lambda: halo_mix(16_000_000, BASE_SEED + 8, n_halos=11150),
                       eps=5e-4, theta=0.6, n_crit=256, dt=1.0 / 1024),
}


def workload(name: str):
    w = dict(WORKLOADS[name])
    ps = w.pop("gen")()
    return ps, w
