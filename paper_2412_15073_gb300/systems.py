"""Seeded synthetic systems: flexible 3-site water and charged LJ beads.

This module only builds inputs (coordinates, velocities, topology and
force-field tables). It holds none of the integrator or force arithmetic, so
both the CUDA path and the CPU oracle take their inputs from it.

The water model stands in for the SPC/Fw water of the paper's experiments
(Sec. 4): harmonic O-H bonds and H-O-H angles (1/2 k convention), O-O
Lennard-Jones, fixed point charges. Parameters default to the values of the
benchmark configurations (r0 = 1.0 A, k_b = 1059 kcal/mol/A^2,
theta0 = 109.47 deg, k_theta = 75.9 kcal/mol/rad^2, eps_OO = 0.155 kcal/mol,
sigma_OO = 3.166 A, q_O = -0.82 e, q_H = +0.41 e).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KB_KCAL = 0.0019872042586      # kcal/mol/K
KCAL_AMU = 418.4               # 1 kcal/mol = 418.4 amu A^2 / ps^2
M_O, M_H = 15.9994, 1.008
WATER_DENSITY_MOL = 0.03338    # molecules / A^3 (0.1001 atoms / A^3)


@dataclasses.dataclass
class System:
    """One periodic system in the layout both engines accept."""
    box: float
    x: np.ndarray              # (n, 3) float64, A
    v: np.ndarray              # (n, 3) float64, A/ps
    mass: np.ndarray           # (n,) amu
    charge: np.ndarray         # (n,) e
    type: np.ndarray           # (n,) int32 LJ type
    lj_eps: np.ndarray         # (nt, nt) kcal/mol, mixing already applied
    lj_sigma: np.ndarray       # (nt, nt) A
    bonds: np.ndarray          # (nb, 2) int32
    bond_k: np.ndarray         # (nb,)
    bond_r0: np.ndarray        # (nb,)
    angles: np.ndarray         # (na, 3) int32, centre atom in the middle
    angle_k: np.ndarray        # (na,)
    angle_t0: np.ndarray       # (na,) rad
    excl: np.ndarray           # (ne, 2) int32 excluded nonbonded pairs

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def copy(self) -> "System":
        return dataclasses.replace(self, **{f.name: (np.array(getattr(self, f.name), copy=True)
                                                   if isinstance(getattr(self, f.name), np.ndarray)
                                                   else getattr(self, f.name))
                                            for f in dataclasses.fields(self)})


def _random_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """k uniformly distributed rotation matrices (from unit quaternions)."""
    q = rng.normal(size=(k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def maxwell_velocities(rng: np.random.Generator, mass: np.ndarray, temperature: float) -> np.ndarray:
    """Velocities drawn from the Maxwell law at `temperature` (A/ps)."""
    sd = np.sqrt(KB_KCAL * temperature * KCAL_AMU / mass)
    return rng.normal(size=(mass.shape[0], 3)) * sd[:, None]


def water_box(n_mol: int, box: float | None = None, seed: int = 0, temperature: float = 300.0,
              r0: float = 1.0, theta0_deg: float = 109.47, k_bond: float = 1059.0,
              k_angle: float = 75.9, eps_oo: float = 0.155, sigma_oo: float = 3.166,
              q_o: float = -0.82, hh_min: float = 1.6) -> System:
    """Water molecules on a cubic lattice with random orientations.

    n_side = ceil(n_mol^(1/3)) sites per edge filled in row-major order, the O
    atom on the site and the two H atoms at r0 with the angle theta0, each
    molecule turned by a uniform random rotation drawn from `seed`. Rotations
    that put two H atoms of neighbouring molecules closer than `hh_min` are
    redrawn. Velocities are Maxwellian at `temperature`.
    """
    if box is None:
        box = (n_mol / WATER_DENSITY_MOL) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    n_side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    a = box / n_side
    idx = np.arange(n_mol)
    site = np.stack([idx % n_side, (idx // n_side) % n_side, idx // (n_side * n_side)], 1)
    o_pos = (site + 0.5) * a
    th = math.radians(theta0_deg)
    body = np.array([[r0 * math.sin(th / 2), 0.0, r0 * math.cos(th / 2)],
                     [-r0 * math.sin(th / 2), 0.0, r0 * math.cos(th / 2)]])
    rot = _random_rotations(rng, n_mol)
    # site -> molecule map to find lattice neighbours
    grid = -np.ones((n_side,) * 3, dtype=np.int64)
    grid[site[:, 0], site[:, 1], site[:, 2]] = idx
    offs = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)
                     if (i, j, k) > (0, 0, 0)])
    for _ in range(200):
        h = o_pos[:, None, :] + np.einsum("mij,hj->mhi", rot, body)
        bad = np.zeros(n_mol, dtype=bool)
        for off in offs:
            nb_site = (site + off) % n_side
            nb = grid[nb_site[:, 0], nb_site[:, 1], nb_site[:, 2]]
            ok = nb >= 0
            if not ok.any():
                continue
            m1, m2 = idx[ok], nb[ok]
            d = h[m1][:, :, None, :] - h[m2][:, None, :, :]
            d -= box * np.round(d / box)
            close = (np.sqrt((d * d).sum(-1)) < hh_min).any(axis=(1, 2))
            bad[m2[close]] = True
        if not bad.any():
            break
        rot[bad] = _random_rotations(rng, int(bad.sum()))
    h = o_pos[:, None, :] + np.einsum("mij,hj->mhi", rot, body)
    n = 3 * n_mol
    x = np.empty((n, 3))
    x[0::3] = o_pos
    x[1::3] = h[:, 0]
    x[2::3] = h[:, 1]
    x %= box
    mass = np.tile([M_O, M_H, M_H], n_mol).astype(np.float64)
    charge = np.tile([q_o, -q_o / 2, -q_o / 2], n_mol).astype(np.float64)
    typ = np.tile([0, 1, 1], n_mol).astype(np.int32)
    v = maxwell_velocities(rng, mass, temperature)
    o = 3 * idx
    bonds = np.concatenate([np.stack([o, o + 1], 1), np.stack([o, o + 2], 1)]).astype(np.int32)
    angles = np.stack([o + 1, o, o + 2], 1).astype(np.int32)
    excl = np.concatenate([np.stack([o, o + 1], 1), np.stack([o, o + 2], 1),
                           np.stack([o + 1, o + 2], 1)]).astype(np.int32)
    lj_eps = np.array([[eps_oo, 0.0], [0.0, 0.0]])
    lj_sigma = np.array([[sigma_oo, 1.0], [1.0, 1.0]])
    return System(box=float(box), x=x, v=v, mass=mass, charge=charge, type=typ,
                  lj_eps=lj_eps, lj_sigma=lj_sigma, bonds=bonds,
                  bond_k=np.full(len(bonds), k_bond), bond_r0=np.full(len(bonds), r0),
                  angles=angles, angle_k=np.full(n_mol, k_angle),
                  angle_t0=np.full(n_mol, math.radians(theta0_deg)), excl=excl)


def point_charges(x: np.ndarray, box: float, charge, mass, seed: int = 0, temperature: float = 300.0,
                  lj_eps: float = 0.0, lj_sigma: float = 1.0) -> System:
    """Free atoms of one LJ type with given positions and charges (small tests)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3) % box
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    mass = np.broadcast_to(np.asarray(mass, dtype=np.float64), (n,)).copy()
    charge = np.broadcast_to(np.asarray(charge, dtype=np.float64), (n,)).copy()
    v = maxwell_velocities(rng, mass, temperature)
    e = np.zeros((0, 2), dtype=np.int32)
    return System(box=float(box), x=x, v=v, mass=mass, charge=charge,
                  type=np.zeros(n, dtype=np.int32), lj_eps=np.array([[lj_eps]]),
                  lj_sigma=np.array([[lj_sigma]]), bonds=e, bond_k=np.zeros(0), bond_r0=np.zeros(0),
                  angles=np.zeros((0, 3), dtype=np.int32), angle_k=np.zeros(0),
                  angle_t0=np.zeros(0), excl=e)


def replica_sizes(n_replicas: int = 64, lo_mol: int = 216, hi_mol: int = 2000, seed: int = 1) -> list[int]:
    """Molecule counts of a batched ensemble, uniform in [lo_mol, hi_mol]."""
    rng = np.random.default_rng(seed)
    return [int(k) for k in rng.integers(lo_mol, hi_mol + 1, size=n_replicas)]


def water_with_beads(n_total: int = 1_000_000, n_beads: int = 50_002, seed: int = 2,
                     temperature: float = 300.0, bead_eps: float = 0.2, bead_sigma: float = 3.5,
                     bead_q: float = 0.5, bead_mass: float = 39.948, bead_rho_sigma3: float = 0.85,
                     box: float | None = None) -> System:
    """Water with an embedded dense sphere of charged LJ beads.

    The beads (half +bead_q, half -bead_q, in rock-salt order on their lattice)
    fill a sphere at reduced density rho sigma^3 = bead_rho_sigma3 at the box
    centre on a jittered cubic lattice; water molecules fill the rest of the
    box at liquid density. LJ
    cross terms use Lorentz-Berthelot mixing with the water oxygen.
    """
    n_mol = (n_total - n_beads) // 3
    rho_b = bead_rho_sigma3 / bead_sigma ** 3
    vol_b = n_beads / rho_b
    r_b = (3.0 * vol_b / (4.0 * math.pi)) ** (1.0 / 3.0)
    if box is None:
        box = (vol_b + n_mol / WATER_DENSITY_MOL) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    centre = np.full(3, box / 2)
    # beads: jittered cubic lattice inside the sphere
    a_b = rho_b ** (-1.0 / 3.0)
    k = int(math.ceil(2 * r_b / a_b)) + 2
    lat = np.stack(np.meshgrid(*[np.arange(-k // 2, k // 2 + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    lat = lat[np.argsort((lat * lat).sum(1), kind="stable")][:n_beads]
    g = lat * a_b
    xb = centre + g + rng.uniform(-0.05, 0.05, size=g.shape) * a_b
    # water: a lattice over the box slightly denser than the liquid; sites
    # inside the bead sphere (+ margin) are removed and n_mol of the rest kept
    # at random, so the water fills the box uniformly at liquid density
    frac_out = 1.0 - 4.0 / 3.0 * math.pi * (r_b + 2.0) ** 3 / box ** 3
    n_side = int(math.ceil((1.02 * n_mol / frac_out) ** (1.0 / 3.0)))
    w = water_box(n_side ** 3, box=box, seed=seed, temperature=temperature)
    o = w.x[0::3]
    d = o - centre
    d -= box * np.round(d / box)
    outside = np.flatnonzero(np.sqrt((d * d).sum(1)) > r_b + 2.0)
    if outside.size < n_mol:
        raise ValueError("box too small for the requested water count")
    keep = np.sort(rng.choice(outside, n_mol, replace=False))
    atoms = np.stack([3 * keep, 3 * keep + 1, 3 * keep + 2], 1).reshape(-1)
    xw = w.x[atoms]
    n_w = xw.shape[0]
    x = np.concatenate([xw, xb % box])
    mass = np.concatenate([w.mass[atoms], np.full(n_beads, bead_mass)])
    # rock-salt order on the bead lattice (nearest neighbours of opposite
    # sign), balanced by flipping the outermost beads of the larger sign
    qb = np.where(lat.sum(1) % 2 == 0, bead_q, -bead_q)
    excess = int((qb > 0).sum() - (qb < 0).sum())
    if excess:
        big = np.flatnonzero(qb > 0 if excess > 0 else qb < 0)
        qb[big[-(abs(excess) // 2):]] *= -1.0
    charge = np.concatenate([w.charge[atoms], qb])
    typ = np.concatenate([w.type[atoms], np.full(n_beads, 2, dtype=np.int32)]).astype(np.int32)
    eo, so = w.lj_eps[0, 0], w.lj_sigma[0, 0]
    lj_eps = np.zeros((3, 3))
    lj_sigma = np.ones((3, 3))
    lj_eps[0, 0], lj_sigma[0, 0] = eo, so
    lj_eps[2, 2], lj_sigma[2, 2] = bead_eps, bead_sigma
    lj_eps[0, 2] = lj_eps[2, 0] = math.sqrt(eo * bead_eps)
    lj_sigma[0, 2] = lj_sigma[2, 0] = 0.5 * (so + bead_sigma)
    mol = np.arange(len(keep))
    o3 = 3 * mol
    bonds = np.concatenate([np.stack([o3, o3 + 1], 1), np.stack([o3, o3 + 2], 1)]).astype(np.int32)
    angles = np.stack([o3 + 1, o3, o3 + 2], 1).astype(np.int32)
    excl = np.concatenate([np.stack([o3, o3 + 1], 1), np.stack([o3, o3 + 2], 1),
                           np.stack([o3 + 1, o3 + 2], 1)]).astype(np.int32)
    v = np.concatenate([w.v[atoms], maxwell_velocities(rng, np.full(n_beads, bead_mass), temperature)])
    assert n_w + n_beads == x.shape[0]
    return System(box=float(box), x=x, v=v, mass=mass, charge=charge, type=typ,
                  lj_eps=lj_eps, lj_sigma=lj_sigma, bonds=bonds,
                  bond_k=np.full(len(bonds), w.bond_k[0]), bond_r0=np.full(len(bonds), w.bond_r0[0]),
                  angles=angles, angle_k=np.full(len(mol), w.angle_k[0]),
                  angle_t0=np.full(len(mol), w.angle_t0[0]), excl=excl)
