"""Seeded synthetic localized-orbital systems.

This module is the one place both sides of every parity check take their inputs from: the CUDA
library and the CPU oracle each receive the arrays built here and nothing else. It holds none of
the TDDFT method's arithmetic. It only does what the ground-state calculation does before a
linear-response run starts (the paper's Sec. II C takes all of it as given):

* draws atom positions (random sequential adsorption, minimum separation);
* tabulates atom-centred Gaussian support functions {phi} (valence) and {chi} (conduction) on a
  periodic real-space grid, inside one cubic box per atom, hard-cut at a localisation radius and
  normalised on the grid (dV * sum f^2 = 1);
* forms their overlap matrices S^phi, S^chi from those tables;
* draws random sparse symmetric Hamiltonians H^phi, H^chi with exponentially decaying entries,
  shifts H^chi so the Kohn-Sham gap is a set value, and builds the density kernels P^v, P^c as
  spectral projectors of the generalised eigenproblems H c = eps S c;
* tabulates the ground-state density n0 = 2 sum_ab phi_a P^v_ab phi_b.

It also draws the random starting vectors the eigensolver needs, which each side then masks and
projects itself.

Units: Hartree atomic units (bohr, Ha) everywhere in the returned arrays. Grid arrays are C-order
[ix][iy][iz] (z fastest); a box of extent (ex, ey, ez) with origin (ox, oy, oz) covers the grid
points ((ox+i) mod n, (oy+j) mod n, (oz+l) mod n).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import hashlib
import math
import os

import numpy as np
import scipy.linalg

BOHR_PER_ANG = 1.0 / 0.529177210903  # CODATA 2018
HA_PER_EV = 1.0 / 27.211386246


@dataclasses.dataclass(frozen=True)
class Recipe:
    """Parameters of one synthetic chromophore-like system (lengths in Angstrom, energies in eV/Ha)."""

    natoms: int
    cell_ang: float
    ngrid: int
    nphi: int = 4              # valence functions per atom: s, px, py, pz
    nchi: int = 4              # conduction functions per atom: 4 (s, p) or 9 (s, p, d)
    radius_ang: float = 7.0    # localisation radius of every support function
    width_ang: tuple = (0.6, 1.2)
    min_sep_ang: float = 1.4
    gap_ev: float = 2.0
    h_sigma: float = 0.1       # Ha, std of the random Hamiltonian entries
    h_decay_ang: float = 2.0   # entries decay as exp(-d / h_decay)
    kernel_cutoff_ang: float = 0.0   # <= 0: response kernels not truncated
    density_kernel_cutoff_ang: float = 0.0   # > 0: P^v, P^c truncated at this radius (sparse form)
    seed: int = 0
    cluster_ang: float = 0.0   # > 0: atoms only inside a centred cube of this side (vacuum around)
    sphere_density: float = 0.0   # > 0: atoms fill a centred sphere at this density (A^-3) ...
    core_atoms: int = 0           # ... the first core_atoms its inner sphere, the rest the shell
    fast: bool = False            # large systems: float32 tables, separable overlap sums, one
                                  # eigendecomposition per Hamiltonian, atomic n0 (see generate)


# The smallest workload: 8 atoms, 16 A cell, 48^3 grid, 4 phi + 4 chi (s, p) per atom, 7 A radius,
# no truncation. Small enough for the dense oracle.
CONFIG_SMALL = Recipe(natoms=8, cell_ang=16.0, ngrid=48, nphi=4, nchi=4, radius_ang=7.0, seed=1)

# The chromophore-sized workload: 140 atoms in a 30 A cell, 0.25 A grid (120^3), 4 phi + 9 chi per
# atom, 8 A radius, response kernels truncated at 12 A.
CONFIG_CHROMOPHORE = Recipe(natoms=140, cell_ang=30.0, ngrid=120, nphi=4, nchi=9, radius_ang=8.0,
                            kernel_cutoff_ang=12.0, seed=2)


def scaling_recipe(natoms: int, seed: int = 5) -> Recipe:
    """The linear-scaling series: a 140-atom core sphere and a shell grown to natoms, both at
    0.1 atoms per A^3 (RSA, 1.4 A minimum separation); cell = cluster diameter + 2R + 10 A of
    vacuum, rounded up to a 2/3/5-smooth grid at 0.25 A (500 atoms: 48 A, 192^3; 1000: 54 A,
    216^3; 2000: 60 A, 240^3); 4 phi + 9 chi per atom, R = 8 A, kernels truncated at 15 A."""
    density, R, h = 0.1, 8.0, 0.25
    r_cluster = (3.0 * natoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    n = smooth_grid(int(math.ceil((2.0 * r_cluster + 2.0 * R + 10.0) / h)))
    return Recipe(natoms=natoms, cell_ang=n * h, ngrid=n, nphi=4, nchi=9, radius_ang=R,
                  kernel_cutoff_ang=15.0, density_kernel_cutoff_ang=15.0, seed=seed, sphere_density=density,
                  core_atoms=min(140, natoms), fast=True)


@dataclasses.dataclass
class FunctionSet:
    """Support functions tabulated in per-function periodic boxes (Hartree atomic units)."""

    atom: np.ndarray   # int32 [nfun]   owning atom; functions are grouped by atom
    box: np.ndarray    # int32 [nfun,6] origin (ox,oy,oz) in [0,n) and extent (ex,ey,ez)
    off: np.ndarray    # int64 [nfun+1] offsets into val
    val: np.ndarray    # float64 [off[-1]] box values, C order [i][j][l] (z fastest)

    @property
    def nfun(self) -> int:
        return int(self.atom.shape[0])

    def values(self, f: int) -> np.ndarray:
        ex, ey, ez = (int(v) for v in self.box[f, 3:])
        return self.val[self.off[f]:self.off[f + 1]].reshape(ex, ey, ez)


@dataclasses.dataclass
class System:
    recipe: Recipe
    cell: float            # bohr, cubic periodic cell side
    n: int                 # grid points per side
    pos: np.ndarray        # float64 [natoms,3] bohr
    phi: FunctionSet
    chi: FunctionSet
    S_phi: np.ndarray
    S_chi: np.ndarray
    H_phi: np.ndarray
    H_chi: np.ndarray
    P_v: np.ndarray
    P_c: np.ndarray
    n0: np.ndarray         # float64 [n,n,n]
    kernel_cutoff: float   # bohr; <= 0 means no truncation
    n_occ: int
    n_cond: int
    density_kernel_cutoff: float = 0.0   # bohr; > 0: P^v, P^c truncated there (sparse form)

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def h(self) -> float:
        return self.cell / self.n

    @property
    def dV(self) -> float:
        return self.h ** 3


# ----------------------------------------------------------------------------------------------
# geometry and tables

def _workers():
    return max(1, min(32, os.cpu_count() or 1))


def _rsa_positions(rng, natoms, cell, min_sep, cluster=0.0):
    pos = np.zeros((natoms, 3))
    placed = 0
    tries = 0
    lo, hi = (0.0, cell) if cluster <= 0.0 else (0.5 * (cell - cluster), 0.5 * (cell + cluster))
    while placed < natoms:
        tries += 1
        if tries > 2000000:
            raise RuntimeError("could not place atoms at the requested minimum separation")
        x = rng.uniform(lo, hi, size=3)
        if placed:
            d = pos[:placed] - x
            d -= cell * np.round(d / cell)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        pos[placed] = x
        placed += 1
    return pos


def _rsa_sphere_positions(rng, natoms, cell, min_sep, density, core):
    """RSA inside a centred sphere holding natoms at the given density (bohr^-3): atoms
    0..core-1 in the inner sphere that holds core atoms at that density, the rest between the two
    spheres."""
    r_out = (3.0 * natoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    r_in = (3.0 * core / (4.0 * math.pi * density)) ** (1.0 / 3.0) if core > 0 else 0.0
    centre = np.full(3, 0.5 * cell)
    pos = np.zeros((natoms, 3))
    placed = 0
    tries = 0
    while placed < natoms:
        tries += 1
        if tries > 20000000:
            raise RuntimeError("could not place atoms at the requested minimum separation")
        lo, hi = (0.0, r_in) if placed < core else (r_in, r_out)
        v = rng.standard_normal(3)
        r = hi * rng.uniform() ** (1.0 / 3.0)
        if r < lo:
            continue
        x = centre + r * v / np.linalg.norm(v)
        if placed:
            d = pos[:placed] - x
            d -= cell * np.round(d / cell)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        pos[placed] = x
        placed += 1
    return pos


def _angular(kind, dx, dy, dz, w):
    """Real solid-harmonic prefactors (up to normalisation): s, p_x, p_y, p_z, then 5 d."""
    if kind == 0:
        return np.ones_like(dx)
    if kind == 1:
        return dx / w
    if kind == 2:
        return dy / w
    if kind == 3:
        return dz / w
    w2 = w * w
    if kind == 4:
        return dx * dy / w2
    if kind == 5:
        return dy * dz / w2
    if kind == 6:
        return dz * dx / w2
    if kind == 7:
        return 0.5 * (dx * dx - dy * dy) / w2
    if kind == 8:
        return (2.0 * dz * dz - dx * dx - dy * dy) / (2.0 * math.sqrt(3.0) * w2)
    raise ValueError(kind)


def box_half_width(radius, h):
    """Half width m (grid points) of the cube that holds a sphere of the given radius."""
    return int(math.ceil(radius / h)) + 1


def _tabulate(rng_w, pos, nper, cell, n, radius, width, dtype=np.float64, params=None):
    """Tables of the functions of every atom; `params` (a dict), when given, receives the widths,
    the normalisation factors, the box centres (grid index of each atom) and the half width m."""
    h = cell / n
    m = box_half_width(radius, h)
    e = 2 * m + 1
    if e > n:
        raise ValueError("localisation box wider than the cell: the cell must exceed 2R + 2h")
    natoms = pos.shape[0]
    nfun = natoms * nper
    atom = np.repeat(np.arange(natoms, dtype=np.int32), nper)
    box = np.zeros((nfun, 6), dtype=np.int32)
    off = np.arange(nfun + 1, dtype=np.int64) * (e ** 3)
    val = np.empty(int(off[-1]), dtype=dtype)
    widths = rng_w.uniform(width[0], width[1], size=nfun)   # one draw per function, in order
    norms = np.zeros(nfun)
    dV = h ** 3
    t = np.arange(-m, m + 1, dtype=np.float64)

    def one_atom(ia):
        c = np.rint(pos[ia] / h).astype(np.int64)
        d = [(c[a] + t) * h - pos[ia, a] for a in range(3)]
        dx, dy, dz = np.meshgrid(d[0], d[1], d[2], indexing="ij")
        r2 = dx * dx + dy * dy + dz * dz
        inside = r2 <= radius * radius
        for kf in range(nper):
            f = ia * nper + kf
            w = widths[f]
            g = np.exp(-r2 / (w * w)) * _angular(kf, dx, dy, dz, w)
            g[~inside] = 0.0
            norms[f] = 1.0 / math.sqrt(dV * np.sum(g * g))
            g *= norms[f]
            val[off[f]:off[f + 1]] = g.ravel()
            box[f, :3] = np.mod(c - m, n)
            box[f, 3:] = e

    with concurrent.futures.ThreadPoolExecutor(_workers()) as ex:
        list(ex.map(one_atom, range(natoms)))
    if params is not None:
        params.update(widths=widths, norms=norms, centre=np.rint(pos / h).astype(np.int64), m=m, h=h, n=n)
    return FunctionSet(atom=atom, box=box, off=off, val=val)


# ---- sums that factor along the axes (large systems) ------------------------------------------
# A tabulated function is N_f exp(-|r - R_a|^2 / w_f^2) A_f(r - R_a) inside the radius R and zero
# beyond, with A_f a polynomial of degree <= 2 (_angular). Beyond R the Gaussian is below
# exp(-R^2 / w^2) <= exp(-44) of its peak for the widths used, so the sum over the grid of a
# product of two tables equals, to double rounding, the sum of the uncut functions over the
# common points of their boxes, and that factors into one-dimensional sums along x, y and z.

_SQ3 = math.sqrt(3.0)
_MONO = {   # kind -> [(coefficient times w^degree, (px, py, pz))], the monomials of _angular
    0: [(1.0, (0, 0, 0))],
    1: [(1.0, (1, 0, 0))], 2: [(1.0, (0, 1, 0))], 3: [(1.0, (0, 0, 1))],
    4: [(1.0, (1, 1, 0))], 5: [(1.0, (0, 1, 1))], 6: [(1.0, (1, 0, 1))],
    7: [(0.5, (2, 0, 0)), (-0.5, (0, 2, 0))],
    8: [(1.0 / _SQ3, (0, 0, 2)), (-0.5 / _SQ3, (2, 0, 0)), (-0.5 / _SQ3, (0, 2, 0))],
}


def _axis_factors(pos, nper, params):
    """U[atom, axis, t, f * 3 + p] = exp(-d^2 / w_f^2) d^p along one axis of the atom's box
    (d the displacement of box point t from the atom), and the monomial tables of the set."""
    natoms = pos.shape[0]
    m, h = params["m"], params["h"]
    T = 2 * m + 1
    t = np.arange(-m, m + 1, dtype=np.float64)
    w = params["widths"].reshape(natoms, nper)
    U = np.empty((natoms, 3, T, nper * 3))
    for ax in range(3):
        d = (params["centre"][:, ax][:, None] + t[None, :]) * h - pos[:, ax][:, None]      # [atoms, T]
        e = np.exp(-(d[:, :, None] ** 2) / (w[:, None, :] ** 2))                            # [atoms, T, f]
        for p in range(3):
            U[:, ax, :, p::3] = e * (d[:, :, None] ** p)
    coef = np.zeros((nper, 3))
    expo = np.zeros((nper, 3, 3), dtype=np.int64)
    for kf in range(nper):
        for q, (c, ex) in enumerate(_MONO[kf]):
            coef[kf, q] = c
            expo[kf, q] = ex
    return U, coef, expo


def _separable_overlaps(fs, nper, pos, cell, n, dV, rmax, params, chunk=2048):
    """S_ab = dV sum_r f_a(r) f_b(r) for atom pairs within rmax, from the factored axis sums
    (needs boxes no wider than half the cell, so that two boxes meet in one run per axis)."""
    natoms = pos.shape[0]
    m = params["m"]
    T = 2 * m + 1
    if 2 * T > n:
        raise ValueError("separable overlaps need boxes no wider than half the cell")
    U, coef, expo = _axis_factors(pos, nper, params)
    w = params["widths"].reshape(natoms, nper)
    nrm = params["norms"].reshape(natoms, nper)
    deg = expo[:, 0, :].sum(axis=1)     # degree of each kind (every monomial of a kind has it)
    N = natoms * nper
    S = np.zeros((N, N))
    pairs = np.array([(i, j) for (i, j, _) in _atom_pairs_within(pos, cell, rmax)], dtype=np.int64)
    cen = params["centre"]
    fi = np.arange(nper)
    for c0 in range(0, len(pairs), chunk):
        pr = pairs[c0:c0 + chunk]
        a, b = pr[:, 0], pr[:, 1]
        P = len(pr)
        G = []
        for ax in range(3):
            s_ = (cen[a, ax] - cen[b, ax]) % n
            s_ = np.where(s_ > n // 2, s_ - n, s_)                     # b index = a index + s
            idx = np.arange(T)[None, :] + s_[:, None]                  # [P, T]
            ok = (idx >= 0) & (idx < T)
            Ub = U[b[:, None], ax, np.clip(idx, 0, T - 1)] * ok[:, :, None]   # [P, T, nper*3]
            Ua = U[a, ax]                                               # [P, T, nper*3]
            G.append(np.matmul(Ua.transpose(0, 2, 1), Ub).reshape(P, nper, 3, nper, 3))
        blk = np.zeros((P, nper, nper))
        for q in range(3):
            for r in range(3):
                cq = coef[:, q][None, :, None] * coef[:, r][None, None, :]
                if not np.any(cq):
                    continue
                term = cq * np.ones((P, 1, 1))
                for ax in range(3):
                    term = term * G[ax][:, fi[:, None], expo[:, q, ax][:, None], fi[None, :], expo[:, r, ax][None, :]]
                blk += term
        scale = (dV * nrm[a][:, :, None] * nrm[b][:, None, :] /
                 (w[a][:, :, None] ** deg[None, :, None] * w[b][:, None, :] ** deg[None, None, :]))
        blk *= scale
        for (i, j), B in zip(pr, blk):
            S[i * nper:(i + 1) * nper, j * nper:(j + 1) * nper] = B
            if i != j:
                S[j * nper:(j + 1) * nper, i * nper:(i + 1) * nper] = B.T
    return 0.5 * (S + S.T)


def _atomic_density(fs, nper, K, n):
    """sum over atoms I of sum_{a, b on I} f_a(r) K_ab f_b(r) on the full grid (the on-site
    blocks of K only: a superposition of atomic densities)."""
    out = np.zeros((n, n, n))
    for ia in range(fs.nfun // nper):
        A, o, e = _atom_block(fs, ia, nper)
        Kaa = K[ia * nper:(ia + 1) * nper, ia * nper:(ia + 1) * nper]
        Af = A.reshape(nper, -1).astype(np.float64)
        contrib = np.einsum("ar,ar->r", Kaa @ Af, Af).reshape(e, e, e)
        _add_parts(out, [(int(o[0]), int(o[1]), int(o[2]), contrib)], n)
    return out


def _axis_overlaps(oa, ob, e, n):
    """Common grid points of two wrapped ranges [oa, oa+e) and [ob, ob+e) (mod n).

    Returns a list of (start_in_a, start_in_b, length) runs.
    """
    shift = (ob - oa) % n
    runs = []
    if shift < e:
        runs.append((shift, 0, e - shift))
    if shift + e > n:
        ln = shift + e - n
        runs.append((0, n - shift, min(ln, e)))
    return runs


def _atom_pairs_within(pos, cell, rmax):
    natoms = pos.shape[0]
    pairs = []
    for i in range(natoms):
        d = pos[i:] - pos[i]
        d -= cell * np.round(d / cell)
        dist = np.sqrt(np.einsum("ij,ij->i", d, d))
        for jj in np.nonzero(dist <= rmax)[0]:
            pairs.append((i, i + int(jj), float(dist[jj])))
    return pairs


def _atom_block(fs, ia, nper):
    f0 = ia * nper
    e = int(fs.box[f0, 3])
    return fs.val[fs.off[f0]:fs.off[f0 + nper]].reshape(nper, e, e, e), fs.box[f0, :3], e


# The per-pair sums below run over the common points XB planes (of x) at a time: the slices of
# a few planes stay in cache while they are copied and multiplied, where one slice of the whole
# common box (megabytes) would not.
XB = 2


def _pair_overlap(fa, fb, nper_a, nper_b, ia, ib, n):
    """sum_r f_a(r) f_b(r) for all functions of atoms ia (set fa) and ib (set fb)."""
    A, oa, e = _atom_block(fa, ia, nper_a)
    B, ob, _ = _atom_block(fb, ib, nper_b)
    out = np.zeros((nper_a, nper_b))
    rx = _axis_overlaps(int(oa[0]), int(ob[0]), e, n)
    ry = _axis_overlaps(int(oa[1]), int(ob[1]), e, n)
    rz = _axis_overlaps(int(oa[2]), int(ob[2]), e, n)
    for (ax, bx, lx) in rx:
        for (ay, by, ly) in ry:
            for (az, bz, lz) in rz:
                for x in range(0, lx, XB):
                    px = min(XB, lx - x)
                    a = A[:, ax + x:ax + x + px, ay:ay + ly, az:az + lz].reshape(nper_a, -1)
                    b = B[:, bx + x:bx + x + px, by:by + ly, bz:bz + lz].reshape(nper_b, -1)
                    out += a @ b.T
    return out


def _overlap_matrix(fs, nper, pos, cell, n, dV, rmax):
    natoms = pos.shape[0]
    N = natoms * nper
    S = np.zeros((N, N))
    pairs = _atom_pairs_within(pos, cell, rmax)
    blocks = _pooled(fs, nper, n, None, _w_overlap, pairs)
    if blocks is not None:
        blocks = [dV * b for part in blocks for b in part]
    else:
        with concurrent.futures.ThreadPoolExecutor(_workers()) as ex:
            blocks = list(ex.map(lambda p: dV * _pair_overlap(fs, fs, nper, nper, p[0], p[1], n), pairs))
    for (i, j, _), blk in zip(pairs, blocks):
        S[i * nper:(i + 1) * nper, j * nper:(j + 1) * nper] = blk
        if i != j:
            S[j * nper:(j + 1) * nper, i * nper:(i + 1) * nper] = blk.T
    return 0.5 * (S + S.T)


def _random_hamiltonian(rng, pos, cell, nper, rmax, sigma, decay):
    natoms = pos.shape[0]
    N = natoms * nper
    H = np.zeros((N, N))
    for (i, j, d) in _atom_pairs_within(pos, cell, rmax):
        blk = rng.normal(0.0, sigma, size=(nper, nper)) * math.exp(-d / decay)
        if i == j:
            blk = 0.5 * (blk + blk.T)
        H[i * nper:(i + 1) * nper, j * nper:(j + 1) * nper] = blk
        if i != j:
            H[j * nper:(j + 1) * nper, i * nper:(i + 1) * nper] = blk.T
    return H


def _density_contrib(fs, nper, K, n, ia, ib, w=1.0):
    """(index arrays, values) of w sum_ab f_a K_ab f_b over the common points of atoms ia, ib."""
    A, oa, e = _atom_block(fs, ia, nper)
    B, ob, _ = _atom_block(fs, ib, nper)
    Kab = K[ia * nper:(ia + 1) * nper, ib * nper:(ib + 1) * nper]
    out = []
    rx = _axis_overlaps(int(oa[0]), int(ob[0]), e, n)
    ry = _axis_overlaps(int(oa[1]), int(ob[1]), e, n)
    rz = _axis_overlaps(int(oa[2]), int(ob[2]), e, n)
    for (ax, bx, lx) in rx:
        for (ay, by, ly) in ry:
            for (az, bz, lz) in rz:
                planes = []
                for x in range(0, lx, XB):
                    px = min(XB, lx - x)
                    a = A[:, ax + x:ax + x + px, ay:ay + ly, az:az + lz].reshape(nper, -1)
                    b = B[:, bx + x:bx + x + px, by:by + ly, bz:bz + lz].reshape(nper, -1)
                    planes.append(w * np.einsum("ar,ar->r", Kab @ b, a))
                contrib = np.concatenate(planes).reshape(lx, ly, lz)
                out.append(((int(oa[0]) + ax) % n, (int(oa[1]) + ay) % n, (int(oa[2]) + az) % n,
                            contrib))
    return out


def _split(start, length, n):
    """Split the wrapped range [start, start+length) (mod n) into (dst, src, len) slices."""
    if start + length <= n:
        return [(start, 0, length)]
    first = n - start
    return [(start, 0, first), (0, first, length - first)]


def _add_parts(out, parts, n):
    for x0, y0, z0, contrib in parts:
        lx, ly, lz = contrib.shape
        for (dx, sx, nx) in _split(x0, lx, n):
            for (dy, sy, ny) in _split(y0, ly, n):
                for (dz, sz, nz) in _split(z0, lz, n):
                    out[dx:dx + nx, dy:dy + ny, dz:dz + nz] += contrib[sx:sx + nx, sy:sy + ny, sz:sz + nz]


def _density_on_grid(fs, nper, K, pos, cell, n, rmax):
    """sum_ab f_a(r) K_ab f_b(r) on the full grid, over atom pairs within rmax, for a symmetric K:
    the (i, j) and (j, i) blocks of a pair of atoms give the same values, so each pair i < j is
    summed once with weight 2."""
    K = 0.5 * (K + K.T)
    jobs = [(i, j, 1.0 if i == j else 2.0) for (i, j, _) in _atom_pairs_within(pos, cell, rmax)]
    partial = _pooled(fs, nper, n, K, _w_density, jobs)
    if partial is not None:
        out = partial[0]
        for g in partial[1:]:
            out += g
        return out
    out = np.zeros((n, n, n))
    with concurrent.futures.ThreadPoolExecutor(_workers()) as ex:
        for parts in ex.map(lambda p: _density_contrib(fs, nper, K, n, p[0], p[1], p[2]), jobs):
            _add_parts(out, parts, n)
    return out


# Large systems (tens of thousands of atom pairs): the per-pair table sums are copy-bound numpy
# work that threads do not speed up, so they run in a pool of spawned processes that map the
# tables from POSIX shared memory. The work is cut into a fixed number of chunks, whatever the
# core count, so the partial sums are added in the same order on every machine.
_POOL_MIN_JOBS = 20000
_POOL_CHUNKS = 64
_W = {}   # worker-side state (set by _w_init in each spawned process)


def _w_init(shm_name, shape, atom, box, off, nper, n, K):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)   # the creating process unlinks it
    _W.update(shm=shm, nper=nper, n=n, K=K,
              fs=FunctionSet(atom=atom, box=box, off=off,
                             val=np.ndarray(shape, dtype=np.float64, buffer=shm.buf)))


def _w_overlap(pairs):
    fs, nper, n = _W["fs"], _W["nper"], _W["n"]
    return [_pair_overlap(fs, fs, nper, nper, i, j, n) for (i, j, _) in pairs]


def _w_density(jobs):
    fs, nper, n, K = _W["fs"], _W["nper"], _W["n"], _W["K"]
    out = np.zeros((n, n, n))
    for (i, j, w) in jobs:
        _add_parts(out, _density_contrib(fs, nper, K, n, i, j, w), n)
    return out


def _pooled(fs, nper, n, K, fn, jobs):
    """fn over fixed chunks of jobs in spawned workers, results in chunk order; None (the caller
    uses threads) for small job lists, inside a daemonic pool worker, or when shared memory cannot
    hold the tables."""
    import multiprocessing as mp
    if len(jobs) < _POOL_MIN_JOBS or mp.current_process().daemon:   # pool workers cannot fork
        return None
    try:
        st = os.statvfs("/dev/shm")
        if st.f_bavail * st.f_frsize < 1.2 * fs.val.nbytes:
            return None
    except OSError:
        return None
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(create=True, size=max(8, fs.val.nbytes))
    try:
        np.ndarray(fs.val.shape, dtype=np.float64, buffer=shm.buf)[:] = fs.val
        step = -(-len(jobs) // _POOL_CHUNKS)
        chunks = [jobs[c:c + step] for c in range(0, len(jobs), step)]
        keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})   # one BLAS thread per worker process
        try:
            pool = mp.get_context("spawn").Pool(
                max(1, min(64, os.cpu_count() or 1)), initializer=_w_init,
                initargs=(shm.name, fs.val.shape, fs.atom, fs.box, fs.off, nper, n, K))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        with pool:
            return pool.map(fn, chunks, chunksize=1)
    finally:
        shm.close()
        shm.unlink()


def _spectral_projector(H, S, nkeep):
    eps, C = scipy.linalg.eigh(H, S)
    Ck = C[:, :nkeep]
    return eps, Ck @ Ck.T


def generate(recipe: Recipe) -> System:
    """Build one seeded synthetic system from a recipe."""
    ss = np.random.SeedSequence(recipe.seed)
    r_pos, r_wphi, r_wchi, r_hphi, r_hchi = (np.random.default_rng(s) for s in ss.spawn(5))
    cell = recipe.cell_ang * BOHR_PER_ANG
    n = int(recipe.ngrid)
    h = cell / n
    R = recipe.radius_ang * BOHR_PER_ANG
    if recipe.sphere_density > 0.0:
        pos = _rsa_sphere_positions(r_pos, recipe.natoms, cell, recipe.min_sep_ang * BOHR_PER_ANG,
                                    recipe.sphere_density / BOHR_PER_ANG ** 3, recipe.core_atoms)
    else:
        pos = _rsa_positions(r_pos, recipe.natoms, cell, recipe.min_sep_ang * BOHR_PER_ANG,
                             recipe.cluster_ang * BOHR_PER_ANG)
    width = (recipe.width_ang[0] * BOHR_PER_ANG, recipe.width_ang[1] * BOHR_PER_ANG)
    dtype = np.float32 if recipe.fast else np.float64
    par_phi, par_chi = {}, {}
    phi = _tabulate(r_wphi, pos, recipe.nphi, cell, n, R, width, dtype, par_phi)
    chi = _tabulate(r_wchi, pos, recipe.nchi, cell, n, R, width, dtype, par_chi)
    dV = h ** 3
    if recipe.fast:
        # large systems: the overlap sums factor along the axes (exact to double rounding, see
        # _separable_overlaps); the tables are kept in float32
        S_phi = _separable_overlaps(phi, recipe.nphi, pos, cell, n, dV, 2.0 * R, par_phi)
        S_chi = _separable_overlaps(chi, recipe.nchi, pos, cell, n, dV, 2.0 * R, par_chi)
    else:
        S_phi = _overlap_matrix(phi, recipe.nphi, pos, cell, n, dV, 2.0 * R)
        S_chi = _overlap_matrix(chi, recipe.nchi, pos, cell, n, dV, 2.0 * R)
    decay = recipe.h_decay_ang * BOHR_PER_ANG
    H_phi = _random_hamiltonian(r_hphi, pos, cell, recipe.nphi, 2.0 * R, recipe.h_sigma, decay)
    H_chi = _random_hamiltonian(r_hchi, pos, cell, recipe.nchi, 2.0 * R, recipe.h_sigma, decay)
    n_phi = recipe.natoms * recipe.nphi
    n_chi = recipe.natoms * recipe.nchi
    n_occ = n_phi // 2
    n_cond = n_chi // 2
    eps_v, P_v = _spectral_projector(H_phi, S_phi, n_occ)
    if recipe.fast:
        # one decomposition: shifting H^chi by s S^chi shifts every eigenvalue by s and keeps the
        # eigenvectors, so the projector onto the lowest n_cond states is that of H^chi itself
        eps_c, C = scipy.linalg.eigh(H_chi, S_chi)
        shift = recipe.gap_ev * HA_PER_EV - (eps_c[0] - eps_v[n_occ - 1])
        H_chi = H_chi + shift * S_chi
        P_c = C[:, :n_cond] @ C[:, :n_cond].T
        del C
        # ground-state density: superposition of the atoms' on-site valence densities
        n0 = 2.0 * _atomic_density(phi, recipe.nphi, P_v, n)
    else:
        eps_c = scipy.linalg.eigh(H_chi, S_chi, eigvals_only=True)
        shift = recipe.gap_ev * HA_PER_EV - (eps_c[0] - eps_v[n_occ - 1])
        H_chi = H_chi + shift * S_chi
        _, P_c = _spectral_projector(H_chi, S_chi, n_cond)
        n0 = 2.0 * _density_on_grid(phi, recipe.nphi, P_v, pos, cell, n, 2.0 * R)
    return System(recipe=recipe, cell=cell, n=n, pos=pos, phi=phi, chi=chi,
                  S_phi=S_phi, S_chi=S_chi, H_phi=H_phi, H_chi=H_chi, P_v=P_v, P_c=P_c,
                  n0=n0, kernel_cutoff=recipe.kernel_cutoff_ang * BOHR_PER_ANG,
                  n_occ=n_occ, n_cond=n_cond,
                  density_kernel_cutoff=recipe.density_kernel_cutoff_ang * BOHR_PER_ANG)


@dataclasses.dataclass
class JointInputs:
    """Raw inputs of the joint unoccupied representation {varphi} = {phi} (+) {chi}: the joint
    function set (per atom its phi, then its chi), its overlap and Hamiltonian, the columns
    S^{varphi phi} of the overlap that belong to phi, and the valence side (H^phi shifted so that
    its unoccupied part lies `gap` above the valence states, P^v unchanged). The conduction
    projector of that representation is not made here: it is the method's own step."""
    funcs: FunctionSet
    S_joint: np.ndarray
    H_joint: np.ndarray
    S_joint_phi: np.ndarray
    H_phi: np.ndarray
    phi_cols: np.ndarray   # int64 [N_phi]: joint index of each phi function


def joint_inputs(sys: System, seed: int, cross_sigma=0.02, chi_shift_ev=4.0) -> JointInputs:
    """Joint-representation inputs from a generated system: per atom its nphi phi and nchi chi
    functions; the joint overlap from the tables; the joint Hamiltonian with the phi block the
    valence Hamiltonian (unoccupied part lifted by the system's gap), the chi block the
    conduction Hamiltonian lifted by chi_shift_ev * S^chi, and random cross blocks of std
    cross_sigma Ha decaying with distance like the other blocks."""
    r = sys.recipe
    nphi, nchi = r.nphi, r.nchi
    nper = nphi + nchi
    na = sys.natoms
    e3 = int(sys.phi.off[1] - sys.phi.off[0])
    if int(sys.chi.off[1] - sys.chi.off[0]) != e3:
        raise ValueError("phi and chi boxes differ in size")
    nfun = na * nper
    atom = np.repeat(np.arange(na, dtype=np.int32), nper)
    box = np.zeros((nfun, 6), dtype=np.int32)
    off = np.arange(nfun + 1, dtype=np.int64) * e3
    val = np.empty(int(off[-1]))
    phi_cols = np.zeros(na * nphi, dtype=np.int64)
    chi_cols = np.zeros(na * nchi, dtype=np.int64)
    for a in range(na):
        for q in range(nphi):
            f, g = a * nper + q, a * nphi + q
            box[f] = sys.phi.box[g]
            val[off[f]:off[f + 1]] = sys.phi.val[sys.phi.off[g]:sys.phi.off[g + 1]]
            phi_cols[g] = f
        for q in range(nchi):
            f, g = a * nper + nphi + q, a * nchi + q
            box[f] = sys.chi.box[g]
            val[off[f]:off[f + 1]] = sys.chi.val[sys.chi.off[g]:sys.chi.off[g + 1]]
            chi_cols[g] = f
    funcs = FunctionSet(atom=atom, box=box, off=off, val=val)
    R = r.radius_ang * BOHR_PER_ANG
    S = _overlap_matrix(funcs, nper, sys.pos, sys.cell, sys.n, sys.dV, 2.0 * R)
    # valence Hamiltonian with its unoccupied part lifted: P^v stays its spectral projector
    gap = r.gap_ev * HA_PER_EV
    Sv = sys.S_phi
    Hv = sys.H_phi + gap * (Sv - Sv @ sys.P_v @ Sv)
    rng = np.random.default_rng(seed)
    H = _random_hamiltonian(rng, sys.pos, sys.cell, nper, 2.0 * R, cross_sigma, r.h_decay_ang * BOHR_PER_ANG)
    H[np.ix_(phi_cols, phi_cols)] = Hv
    H[np.ix_(chi_cols, chi_cols)] = sys.H_chi + chi_shift_ev * HA_PER_EV * sys.S_chi
    H = 0.5 * (H + H.T)
    return JointInputs(funcs=funcs, S_joint=S, H_joint=H, S_joint_phi=S[:, phi_cols], H_phi=Hv, phi_cols=phi_cols)


def with_joint(sys: System, ji: JointInputs, P_c: np.ndarray) -> System:
    """The system in the joint representation: chi := {varphi}, with the conduction projector
    P_c of that representation (from the method, Eq. proj) supplied by the caller."""
    n_cond = int(round(np.trace(P_c @ ji.S_joint)))
    return dataclasses.replace(sys, chi=ji.funcs, S_chi=ji.S_joint, H_chi=ji.H_joint, H_phi=ji.H_phi, P_c=P_c,
                               n_cond=n_cond)


def smooth_grid(n: int) -> int:
    """The smallest 2/3/5-smooth integer >= n (FFT-friendly grid sizes)."""
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 1


def small_density_recipe(natoms: int, seed: int) -> Recipe:
    """The small workload's recipe (4 phi + 4 chi per atom, 7 A radius, 1/3 A grid) at its atom
    density (8 atoms per (16 A)^3), the cubic cell grown with the atom count; the grid is the next
    2/3/5-smooth size (the learned preconditioner's training and evaluation systems)."""
    cell = 16.0 * (natoms / 8.0) ** (1.0 / 3.0)
    n = smooth_grid(int(math.ceil(cell * 3.0)))
    return Recipe(natoms=natoms, cell_ang=cell, ngrid=n, nphi=4, nchi=4, radius_ang=7.0, seed=seed)


def batch_recipes(nsys: int, seed: int, n_min=20, n_max=300, density=0.1, radius=7.0, h=0.25, k_max=8):
    """Uneven systems for a batched launch: atom counts log-uniform in [n_min, n_max], atoms in a
    cube at `density` atoms / A^3, the cell the cube plus 2R + 1 A of vacuum rounded up to a
    2/3/5-smooth grid of spacing h, 4 phi + 4 chi (s, p) per atom of radius R, states uniform in
    1..k_max. Returns [(Recipe, k)]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nsys):
        natoms = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        side = (natoms / density) ** (1.0 / 3.0)
        n = smooth_grid(int(math.ceil((side + 2.0 * radius + 1.0) / h)))
        k = int(rng.integers(1, k_max + 1))
        # the generator's fast path (float32 tables, factored overlap sums) where the boxes are at
        # most half the cell; the small systems take the plain path
        T = 2 * box_half_width(radius, h) + 1
        out.append((Recipe(natoms=natoms, cell_ang=n * h, ngrid=n, nphi=4, nchi=4, radius_ang=radius,
                           cluster_ang=side, seed=1000 * seed + i, fast=2 * T <= n), k))
    return out


def initial_guess(sys: System, k: int, seed: int):
    """Random starting vectors (paper Sec. II B: CG starts from a random vector).

    Returns one float64 array [k, N_chi, N_phi] of N(0,1) draws. Masking to the kernel pattern,
    projection and orthonormalisation are the solver's job, not the generator's.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7919]))
    nc, nv = sys.chi.nfun, sys.phi.nfun
    return rng.standard_normal((k, nc, nv))


def random_kernels(sys: System, k: int, seed: int):
    """Random (P^p, P^q) batches [k, N_chi, N_phi] for operator tests (not projected)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 104729]))
    nc, nv = sys.chi.nfun, sys.phi.nfun
    return (rng.standard_normal((k, nc, nv)), rng.standard_normal((k, nc, nv)))


def mlp_init(n_in: int, width: int, n_out: int, seed: int):
    """Initial parameters of the atom-block network (in -> width -> width -> out), float32, in
    the order W1 [n_in][width], b1, W2 [width][width], b2, W3 [width][n_out], b3. Weights are
    uniform in +-sqrt(6 / fan_in) (He et al. 2015), the output layer scaled by 0.1; biases 0."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 15485863]))
    parts = []
    for fi, fo, scale in ((n_in, width, 1.0), (width, width, 1.0), (width, n_out, 0.1)):
        lim = np.sqrt(6.0 / fi)
        parts.append(scale * rng.uniform(-lim, lim, size=fi * fo))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def minibatch_order(n: int, steps: int, batch: int, seed: int):
    """Sample indices of `steps` minibatches of `batch` rows drawn from n rows: a fresh random
    permutation per epoch, concatenated; int64 [steps * batch]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 32452843]))
    need = steps * batch
    out = []
    have = 0
    while have < need:
        p = rng.permutation(n)
        out.append(p)
        have += n
    return np.concatenate(out)[:need].astype(np.int64)


def fingerprint(sys: System) -> str:
    """Short hash of the generated arrays, for checking two machines built the same system."""
    hsh = hashlib.sha256()
    for a in (sys.pos, sys.S_phi, sys.S_chi, sys.H_phi, sys.H_chi, sys.P_v, sys.P_c, sys.n0):
        hsh.update(np.ascontiguousarray(a).tobytes())
    hsh.update(sys.phi.val[::97].tobytes())
    hsh.update(sys.chi.val[::97].tobytes())
    return hsh.hexdigest()[:16]
