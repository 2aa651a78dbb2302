"""Seeded synthetic inputs for the S1xR2 hot path (shared by the CUDA path's
callers and by the oracle's tests; holds no force, integrator or surrogate
arithmetic).

Particle load (Sect. 3.1, eqs. inversestereographic and omegatovarrho): the
compact radial coordinate w is drawn uniformly in [0, 0.9 pi), the azimuth phi
uniformly in [0, 2 pi) and z uniformly in [0, L). The radius is
rho = D_s tan(w/2) with D_s = L/2, so R_sim = (L/2) tan(0.45 pi). A uniform draw
in w carries the volume element rho d(rho) = (D_s^2/2) tan(w/2) sec^2(w/2) dw,
so each particle's mass is proportional to J(w) = tan(w/2) sec^2(w/2) and the
comoving density is uniform (m_i = rho_bar V_i, Sect. 3.1).

Softening: eps_i = 0.01 L (m_i/m_min)^(1/3) (the literal law), or for the
production-shaped run a 1:8 range eps_i = 0.01 L 8^(ln(m_i/m_min)/ln(m_max/m_min)).

Units: L = 1, G = 1, H0 = 1 (time in 1/H0). Static runs use M_tot = 1; comoving
runs use the comoving mean density rho_bar = 3 Omega_m H0^2 / (8 pi G) and
M_tot = rho_bar pi R_sim^2 L.

The five workloads (sizes, seeds, image cut-offs and integration spans) are
those of the benchmark configurations of this project: the plain-method small
case (N=2048), the comoving LCDM run (N=65,536), the precision study with a
central filament (N=262,144), the learned-surrogate case (N=1,048,576) and the
production-shaped run (N=524,288).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

L_BOX = 1.0
G_NEWTON = 1.0
D_S = 0.5 * L_BOX
W_MAX = 0.9 * math.pi
R_SIM = D_S * math.tan(0.5 * W_MAX)


def comoving_rho_bar(Omega_m: float = 0.3, H0: float = 1.0, G: float = G_NEWTON) -> float:
    return 3.0 * Omega_m * H0 * H0 / (8.0 * math.pi * G)


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    seed: int
    n_cut: int
    comoving: bool
    displaced: bool = False
    filament_frac: float = 0.0
    eps_law: str = "literal"      # "literal" | "ratio8"
    a_start: float = 1.0
    a_end: float = 1.0
    nsteps: int = 0
    dt: float = 0.0               # static runs: fixed dt
    n0: int = 4
    Omega_m: float = 0.3
    Omega_L: float = 0.7

    @property
    def M_tot(self) -> float:
        if not self.comoving:
            return 1.0
        return comoving_rho_bar(self.Omega_m) * math.pi * R_SIM * R_SIM * L_BOX

    @property
    def rho_bar(self) -> float:
        return self.M_tot / (math.pi * R_SIM * R_SIM * L_BOX)


WORKLOADS = {
    "plain_small_n2048": Workload("plain_small_n2048", 2048, 0, 64, comoving=False, nsteps=10, dt=1e-3),
    "lcdm_n65536": Workload("lcdm_n65536", 65536, 1, 16, comoving=True, displaced=True,
                            a_start=0.02, a_end=0.1, nsteps=200),
    "precision_n262144": Workload("precision_n262144", 262144, 2, 64, comoving=True, displaced=True,
                                  filament_frac=0.2, a_start=0.02, a_end=0.02),
    "surrogate_n1048576": Workload("surrogate_n1048576", 1048576, 3, 64, comoving=True, displaced=True,
                                   a_start=0.02, a_end=0.02),
    # the surrogate workload's law at a size that profiles quickly
    "surrogate_n65536": Workload("surrogate_n65536", 65536, 3, 64, comoving=True, displaced=True,
                                 a_start=0.02, a_end=0.02),
    "production_n524288": Workload("production_n524288", 524288, 4, 64, comoving=True, displaced=True,
                                   eps_law="ratio8", a_start=0.02, a_end=1.0, nsteps=1000),
    # the production-shaped law at a size that profiles quickly
    "production_n65536": Workload("production_n65536", 65536, 4, 64, comoving=True, displaced=True,
                                  eps_law="ratio8", a_start=0.02, a_end=1.0, nsteps=1000),
}


def lcdm_time_of_a(a: float, Omega_m: float = 0.3, Omega_L: float = 0.7, H0: float = 1.0) -> float:
    """Cosmic time of flat LCDM (textbook closed form), used only to size the
    constant time step of a run that must span [a_start, a_end]."""
    return 2.0 / (3.0 * math.sqrt(Omega_L) * H0) * math.asinh(math.sqrt(Omega_L / Omega_m) * a ** 1.5)


def run_schedule(w: Workload):
    """(t_start, dt) for a workload: constant dt in cosmic time."""
    if not w.comoving:
        return 0.0, w.dt
    t0 = lcdm_time_of_a(w.a_start, w.Omega_m, w.Omega_L)
    if w.nsteps == 0:
        return t0, 0.0
    t1 = lcdm_time_of_a(w.a_end, w.Omega_m, w.Omega_L)
    return t0, (t1 - t0) / w.nsteps


def particle_load(n: int, seed: int, M_tot: float = 1.0, *, displaced: bool = False,
                  rho_bar: float | None = None, filament_frac: float = 0.0, eps_law: str = "literal",
                  L: float = L_BOX):
    """Returns dict(pos (n,3), vel (n,3), m (n,), h (n,)) in FP64, z in [0, L)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.0, W_MAX, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    z = rng.uniform(0.0, L, n)
    rho = D_S * np.tan(0.5 * w)
    x, y = rho * np.cos(phi), rho * np.sin(phi)
    J = np.tan(0.5 * w) / np.cos(0.5 * w) ** 2
    m = J / J.sum() * M_tot
    if rho_bar is None:
        rho_bar = M_tot / (math.pi * R_SIM * R_SIM * L)
    if filament_frac > 0.0:
        nf = int(round(filament_frac * n))
        sel = rng.permutation(n)[:nf]
        mmed = float(np.median(m))
        x[sel] = rng.normal(0.0, 0.05 * L, nf)
        y[sel] = rng.normal(0.0, 0.05 * L, nf)
        z[sel] = rng.uniform(0.0, L, nf)
        m[sel] = mmed
        m *= M_tot / m.sum()
    if displaced:
        sig = 0.02 * (m / rho_bar) ** (1.0 / 3.0)
        d = rng.normal(0.0, 1.0, (n, 3)) * sig[:, None]
        x += d[:, 0]
        y += d[:, 1]
        z += d[:, 2]
    z = np.mod(z, L)
    z[z >= L] -= L
    mmin, mmax = float(m.min()), float(m.max())
    if eps_law == "literal":
        h = 0.01 * L * (m / mmin) ** (1.0 / 3.0)
    elif eps_law == "ratio8":
        h = 0.01 * L * 8.0 ** (np.log(m / mmin) / math.log(mmax / mmin))
    else:
        raise ValueError(eps_law)
    pos = np.stack([x, y, z], axis=1)
    return {"pos": pos, "vel": np.zeros((n, 3)), "m": m, "h": h}


def workload_ics(w: Workload | str, n: int | None = None):
    """Particle load of a named workload (optionally with a smaller n, same law)."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    nn = w.n if n is None else n
    return particle_load(nn, w.seed, w.M_tot, displaced=w.displaced, rho_bar=w.rho_bar,
                         filament_frac=w.filament_frac, eps_law=w.eps_law)


def subsample(n: int, k: int, seed: int = 12345) -> np.ndarray:
    """Sorted random subset of k particle indices (the error-metric subsample)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)


def ball_load(n: int, seed: int, R: float = 2.0):
    """R^3 topology load: n particles uniform in a ball of radius R (units of L),
    masses uniform in [0.5, 2] normalised to 1, softenings uniform in [0.02, 0.2];
    returns dict(pos, vel, m, h, rho_bar) with rho_bar = 1 / (4 pi R^3 / 3)."""
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n, 3))
    pos = u / np.linalg.norm(u, axis=1)[:, None] * R * rng.uniform(0, 1, n)[:, None] ** (1.0 / 3.0)
    m = rng.uniform(0.5, 2.0, n)
    m /= m.sum()
    h = rng.uniform(0.02, 0.2, n)
    return {"pos": pos, "vel": np.zeros((n, 3)), "m": m, "h": h, "rho_bar": 1.0 / (4.0 / 3.0 * math.pi * R ** 3)}


def tail_training_inputs(ns: int, seed: int, dR_max: float, h_max: float, L: float = L_BOX):
    """Surrogate training inputs (dR, |dz_w|, h): dR with a density that puts
    more samples near the axis, |dz_w| uniform in [0, L/2], h uniform."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, ns)
    dR = dR_max * u * u
    dz = rng.uniform(0.0, 0.5 * L, ns)
    h = rng.uniform(0.0, h_max, ns)
    return np.stack([dR, dz, h], axis=1)


def random_surrogate_params(seed: int, dR_max: float, mu=(0.0, 0.0), sc=(0.05, 0.05)) -> np.ndarray:
    """A seeded parameter vector of the 3 -> 32 -> 32 -> 2 tail network in the
    library's layout (W1[32][3], b1, W2[32][32], b2, W3[2][32], b3, then mu[2],
    sc[2], dR_max): entries uniform in +-1/sqrt(fan-in). Random numbers only, for
    checks of the network form that need weights from outside the library."""
    rng = np.random.default_rng(seed)
    parts = []
    for cnt, fan_in in ((32 * 3, 3), (32, 3), (32 * 32, 32), (32, 32), (2 * 32, 32), (2, 32)):
        b = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-b, b, cnt))
    parts.append(np.array([mu[0], mu[1], sc[0], sc[1], dR_max]))
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------------------
# The paper's tessellated particle load (Sect. 3.1, eqs. inversestereographic
# and omegatovarrho, Fig. 4).
#
# The compact radius w = 2 arctan(rho / D_s) runs over [0, w_max) with
# w_max = 2 arctan(R_sim / D_s). The region w >= w_c is cut into n_out rings of
# equal width dw in w, each ring into n_phi equal azimuth sectors and n_z equal
# z slabs: a uniform grid in (w, phi, z). Inside the core w < w_c the mass
# resolution is held constant. The core is cut into n_in rings of equal area
# (equal width in rho^2), with the same n_phi x n_z cells per ring. n_in is
# chosen so that a core cell has the volume of a cell of the first outer ring,
# rounded to a whole number of rings, so the resolution is continuous at
# rho_c = D_s tan(w_c / 2).
#
# Each cell holds one particle at a uniformly random point of its volume, with
# mass m_i = rho_bar V_i, where V_i = (rho_hi^2 - rho_lo^2) / 2 * dphi * dz is
# the cell's exact comoving volume. The cells tile the cylinder rho < R_sim,
# 0 <= z < L exactly, so the masses sum to rho_bar pi R_sim^2 L.
#
# The paper only says "random location in each compact cell". This generator
# draws uniformly in volume, so the expected density is exactly rho_bar. A draw
# uniform in w would differ only at second order in dw.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CompactRings:
    """Ring structure of the tessellated load. s_edges are the ring edges in
    s = rho^2 (n_in + n_out + 1 values, s_edges[-1] = R_sim^2). cell_volume
    holds one value per ring; the cells of a ring share it."""
    s_edges: np.ndarray
    n_in: int
    n_out: int
    n_phi: int
    n_z: int
    omega_c: float
    rho_c: float
    omega_max: float
    L: float

    @property
    def cell_volume(self) -> np.ndarray:
        ds = np.diff(self.s_edges)
        ds[: self.n_in] = self.s_edges[self.n_in] / max(self.n_in, 1)  # one exact core volume
        return 0.5 * ds * (2.0 * math.pi / self.n_phi) * (self.L / self.n_z)

    @property
    def n(self) -> int:
        return (self.n_in + self.n_out) * self.n_phi * self.n_z


def compact_rings(n_out: int, n_phi: int, n_z: int, *, D_s: float = D_S, R_sim: float = R_SIM,
                  omega_c: float = 0.0, L: float = L_BOX) -> CompactRings:
    """Ring edges and cell volumes of the tessellated load (no particles drawn).
    omega_c = 0 gives the plain uniform grid in w with no constant-mass core."""
    if n_out < 1 or n_phi < 1 or n_z < 1:
        raise ValueError("n_out, n_phi and n_z must be >= 1")
    if not (D_s > 0.0 and R_sim > 0.0 and L > 0.0):
        raise ValueError("D_s, R_sim and L must be positive")
    w_max = 2.0 * math.atan(R_sim / D_s)
    if not (0.0 <= omega_c < w_max):
        raise ValueError("omega_c must lie in [0, 2 arctan(R_sim / D_s))")
    dw = (w_max - omega_c) / n_out
    w_edges = omega_c + dw * np.arange(n_out + 1)
    rho_out = D_s * np.tan(0.5 * w_edges)
    rho_out[0] = D_s * math.tan(0.5 * omega_c)
    rho_out[-1] = R_sim
    s_out = rho_out * rho_out
    rho_c = float(rho_out[0])
    if omega_c > 0.0:
        a1 = s_out[1] - s_out[0]
        n_in = max(1, int(round(s_out[0] / a1)))
        s_in = s_out[0] * np.arange(n_in) / n_in
    else:
        n_in = 0
        s_in = np.zeros(0)
    return CompactRings(np.concatenate([s_in, s_out]), n_in, n_out, n_phi, n_z, float(omega_c), rho_c,
                        w_max, float(L))


def compact_load(n_out: int, n_phi: int, n_z: int, seed: int, *, D_s: float = D_S, R_sim: float = R_SIM,
                 omega_c: float = 0.0, L: float = L_BOX, rho_bar: float = 1.0, eps0: float = 0.01):
    """One particle per cell of compact_rings(...), uniform in the cell's volume,
    with m_i = rho_bar V_i and softening eps0 (m_i / m_min)^(1/3).

    Returns dict(pos (n,3), vel (n,3), m (n,), h (n,), rings), particles in
    ring-major order (ring, then azimuth sector, then z slab); z in [0, L)."""
    rings = compact_rings(n_out, n_phi, n_z, D_s=D_s, R_sim=R_sim, omega_c=omega_c, L=L)
    nr = rings.n_in + rings.n_out
    ring = np.repeat(np.arange(nr), n_phi * n_z)
    sec = np.tile(np.repeat(np.arange(n_phi), n_z), nr)
    slab = np.tile(np.arange(n_z), nr * n_phi)
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, (rings.n, 3))
    s_lo, s_hi = rings.s_edges[ring], rings.s_edges[ring + 1]
    rho = np.sqrt(s_lo + u[:, 0] * (s_hi - s_lo))
    rho = np.minimum(rho, np.nextafter(R_sim, 0.0))
    phi = (sec + u[:, 1]) * (2.0 * math.pi / n_phi)
    z = (slab + u[:, 2]) * (L / n_z)
    z[z >= L] -= L
    m = rho_bar * rings.cell_volume[ring]
    h = eps0 * (m / m.min()) ** (1.0 / 3.0)
    pos = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    return {"pos": pos, "vel": np.zeros((rings.n, 3)), "m": m, "h": h, "rings": rings}


# Table 1's geometry in units of L_z = 1 Gpc: R_sim = 500 Mpc, D_S = 70 Mpc,
# omega_c = 1.63973 rad; its cosmology (Omega_m = 0.3111, Omega_L = 0.6889)
# and initial redshift z = 49 (a = 0.02).
TABLE1_GEOMETRY = dict(D_s=0.07, R_sim=0.5, omega_c=1.63973)
TABLE1_OMEGA_M, TABLE1_OMEGA_L, TABLE1_A_INIT = 0.3111, 0.6889, 1.0 / 50.0


def table1_load(n_out: int = 12, n_phi: int = 64, n_z: int = 64, seed: int = 6):
    """The tessellated load in Table 1's geometry with comoving masses
    (rho_bar = 3 Omega_m / (8 pi), G = H0 = L = 1) and the literal softening law
    eps_i = 0.01 L (m_i / m_min)^(1/3). The defaults give N = 65,536: 4 core
    rings and 12 outer rings of 64 x 64 cells."""
    rho_bar = comoving_rho_bar(TABLE1_OMEGA_M)
    d = compact_load(n_out, n_phi, n_z, seed, L=L_BOX, rho_bar=rho_bar, eps0=0.01 * L_BOX, **TABLE1_GEOMETRY)
    d["rho_bar"] = rho_bar
    return d
