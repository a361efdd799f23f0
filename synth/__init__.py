"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the boundary-element method itself: it only
makes geometry (icosphere surfaces standing in for molecular surfaces) and
point-charge sets with fixed seeds, so that the CUDA path and the CPU oracle
see byte-identical inputs.

Workloads follow the paper's model problem (a dielectric molecule with point
charges inside a closed triangulated surface, Sec. 2.1) with sphere-shaped
stand-ins for the protein meshes, which are not available:

* ``born``      R = 2 A, subdivision 3 (1,280 panels), one +1 e charge at the
                centre, eps_in = 1, eps_out = 80.
* ``globular``  R = 20 A, subdivision 6 (81,920 panels), 2,000 charges uniform
                in the ball r <= 17 A, values U[-0.8, 0.8] e shifted to a net
                +8 e, eps_in = 4, eps_out = 80, seed 2.
* ``globular7`` the same molecule at subdivision 7 (327,680 panels).
* ``batch``     64 spheres, R ~ U[10, 25] A, subdivision in {5, 6, 7},
                500..4,000 charges in the ball of radius R - 3 A, seed 4.
* ``lattice``   1,000 rotated copies of ``globular`` on a 10x10x10 lattice at
                50 A spacing, seed 5.
* ``complex_pair`` a two-sphere "complex": a receptor sphere and a ligand
                sphere a small gap apart, each with its own charges, plus the
                two unbound molecules (for binding free energies).

Panels are returned as float64 arrays of shape [n, 3, 3] (three vertices per
triangle, counter-clockwise seen from outside so that the right-hand normal
points into the solvent); charges as float64 [n_c, 4] rows (x, y, z, q).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "icosphere", "ball_charges", "random_rotation", "Molecule", "born",
    "globular", "lattice", "batch", "small_molecule", "complex_pair",
]


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


def icosphere_mesh(subdivisions: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Vertices [nv, 3] and faces [20*4**s, 3] of a subdivided icosahedron.

    Each subdivision splits every triangle into four at its edge midpoints and
    pushes the new vertices out to the sphere; faces stay counter-clockwise
    seen from outside.
    """
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(int(subdivisions)):
        cache = {}
        vlist = verts

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = np.add(vlist[a], vlist[b]) * 0.5
                m = m / np.linalg.norm(m)
                idx = len(vlist)
                vlist.append(tuple(m))
                cache[key] = idx
            return idx

        nf = np.empty((len(f) * 4, 3), dtype=np.int64)
        for k, (a, b, c) in enumerate(f):
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf[4 * k + 0] = (a, ab, ca)
            nf[4 * k + 1] = (b, bc, ab)
            nf[4 * k + 2] = (c, ca, bc)
            nf[4 * k + 3] = (ab, bc, ca)
        f = nf
        verts = vlist
    v = np.asarray(verts, dtype=np.float64) * float(radius) + np.asarray(center, dtype=np.float64)
    return v, f


_ICO_CACHE: dict = {}


def icosphere(subdivisions: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Flat triangular panels [20*4**s, 3, 3] of an icosphere (float64)."""
    s = int(subdivisions)
    if s not in _ICO_CACHE:
        _ICO_CACHE[s] = icosphere_mesh(s, 1.0)
    v, f = _ICO_CACHE[s]
    pan = v[f] * float(radius)
    pan += np.asarray(center, dtype=np.float64)
    return np.ascontiguousarray(pan)


def ball_charges(n: int, radius: float, rng: np.random.Generator, net: float = 8.0,
                 qmax: float = 0.8, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n charges uniform in a ball; values U[-qmax, qmax] shifted so they sum to `net`.

    Positions: direction from a normalised Gaussian 3-vector, radius
    ``radius * u**(1/3)``.  Values: ``q_k = u_k + (net - sum(u)) / n``.
    """
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    pos = d * r[:, None] + np.asarray(center, dtype=np.float64)
    u = rng.uniform(-qmax, qmax, n)
    q = u + (net - u.sum()) / n
    return np.ascontiguousarray(np.column_stack([pos, q]))


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix (Shoemake's quaternion method)."""
    u1, u2, u3 = rng.random(3)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x, y = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    z, w = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


@dataclasses.dataclass
class Molecule:
    name: str
    panels: np.ndarray      # [n_p, 3, 3] float64
    charges: np.ndarray     # [n_c, 4] float64 (x, y, z, q)
    eps_in: float
    eps_out: float
    radius: float = 0.0     # sphere radius (analytic checks); 0 when not a sphere
    center: tuple = (0.0, 0.0, 0.0)

    @property
    def n_p(self) -> int:
        return int(self.panels.shape[0])

    @property
    def n_c(self) -> int:
        return int(self.charges.shape[0])


def born(subdivisions: int = 3, radius: float = 2.0, q: float = 1.0,
         eps_in: float = 1.0, eps_out: float = 80.0) -> Molecule:
    """A single charge at the centre of a sphere (the Born ion)."""
    ch = np.array([[0.0, 0.0, 0.0, q]])
    return Molecule("born", icosphere(subdivisions, radius), ch, eps_in, eps_out, radius)


def globular(subdivisions: int = 6, radius: float = 20.0, n_charges: int = 2000,
             charge_radius: float = 17.0, seed: int = 2, eps_in: float = 4.0,
             eps_out: float = 80.0) -> Molecule:
    """Sphere-shaped stand-in for a globular protein with random interior charges."""
    rng = np.random.default_rng(seed)
    ch = ball_charges(n_charges, charge_radius, rng)
    return Molecule(f"globular-s{subdivisions}", icosphere(subdivisions, radius), ch,
                    eps_in, eps_out, radius)


def small_molecule(subdivisions: int = 3, radius: float = 6.0, n_charges: int = 40,
                   seed: int = 7, eps_in: float = 4.0, eps_out: float = 80.0) -> Molecule:
    """A small sphere with a handful of off-centre charges (quick tests)."""
    rng = np.random.default_rng(seed)
    ch = ball_charges(n_charges, radius - 3.0, rng, net=1.0)
    return Molecule(f"small-s{subdivisions}", icosphere(subdivisions, radius), ch,
                    eps_in, eps_out, radius)


def lattice(n_side: int = 10, spacing: float = 50.0, subdivisions: int = 6,
            seed: int = 5, base: Molecule | None = None) -> Molecule:
    """n_side**3 randomly rotated copies of one molecule on a cubic lattice."""
    base = base if base is not None else globular(subdivisions)
    rng = np.random.default_rng(seed)
    pans, chs = [], []
    for i in range(n_side):
        for j in range(n_side):
            for k in range(n_side):
                rot = random_rotation(rng)
                off = spacing * np.array([i, j, k], dtype=np.float64)
                pans.append(base.panels @ rot.T + off)
                c = base.charges.copy()
                c[:, :3] = c[:, :3] @ rot.T + off
                chs.append(c)
    return Molecule(f"lattice{n_side}", np.ascontiguousarray(np.concatenate(pans)),
                    np.ascontiguousarray(np.concatenate(chs)), base.eps_in, base.eps_out)


def batch(n_molecules: int = 64, seed: int = 4, subdivisions=(5, 6, 7),
          radius_range=(10.0, 25.0), charge_range=(500, 4000),
          eps_in: float = 4.0, eps_out: float = 80.0) -> list:
    """Uneven molecules: R ~ U[10, 25] A, s drawn from `subdivisions`,
    n_c ~ U{500..4000} charges in the ball of radius R - 3 A, net +8 e."""
    rng = np.random.default_rng(seed)
    mols = []
    for b in range(n_molecules):
        R = float(rng.uniform(*radius_range))
        s = int(rng.choice(subdivisions))
        nc = int(rng.integers(charge_range[0], charge_range[1] + 1))
        ch = ball_charges(nc, R - 3.0, rng)
        mols.append(Molecule(f"batch{b}-s{s}", icosphere(s, R), ch, eps_in, eps_out, R))
    return mols


def complex_pair(s_rec: int = 6, r_rec: float = 20.0, n_rec: int = 2000, s_lig: int = 4,
                 r_lig: float = 6.0, n_lig: int = 60, gap: float = 2.0, seed: int = 11,
                 eps_in: float = 4.0, eps_out: float = 80.0):
    """A receptor sphere at the origin and a ligand sphere centred on the x
    axis with `gap` A between the two surfaces; charges in balls 3 A inside
    each surface (receptor net +8 e, ligand net -1 e).  Returns (complex,
    receptor, ligand): the complex is both closed surfaces and both charge
    sets (the solvent surrounds two disjoint dielectric balls)."""
    rng = np.random.default_rng(seed)
    c_lig = (r_rec + gap + r_lig, 0.0, 0.0)
    ch_r = ball_charges(n_rec, r_rec - 3.0, rng)
    ch_l = ball_charges(n_lig, r_lig - 3.0, rng, net=-1.0, center=c_lig)
    pan_r = icosphere(s_rec, r_rec)
    pan_l = icosphere(s_lig, r_lig) + np.asarray(c_lig)
    rec = Molecule(f"receptor-s{s_rec}", pan_r, ch_r, eps_in, eps_out, r_rec)
    lig = Molecule(f"ligand-s{s_lig}", np.ascontiguousarray(pan_l), ch_l, eps_in, eps_out, r_lig, c_lig)
    cpx = Molecule(f"complex-s{s_rec}-s{s_lig}", np.ascontiguousarray(np.concatenate([pan_r, pan_l])),
                   np.ascontiguousarray(np.concatenate([ch_r, ch_l])), eps_in, eps_out)
    return cpx, rec, lig

