"""Real-space grid operations on localised functions tabulated in periodic boxes.

* ``response_density``: rho(r) = sum_ab chi_a(r) P_ab phi_b(r) (Sec. II C, the response density
  in the mixed chi/phi representation; Sec. III A uses it for rho^q).
* ``potential_integrals``: V_ab = dV sum_r chi_a(r) V(r) phi_b(r), the matrix
  <chi_a|V_SCF^(1)|phi_b> of Eq. operator_TDA / operator_RPA.
* ``full_grid``: every function scattered onto the whole grid (used by the dense oracle and by
  the brute-force pins of the box code).

Functions that share a box (consecutive, same origin and extent) are handled together. Sums run
over the common points of two boxes only, found axis by axis on the periodic grid; no blocking or
reordering beyond that.
"""
import numpy as np


class BoxedSet:
    """A set of functions in periodic boxes, grouped by identical boxes."""

    def __init__(self, fs, n):
        self.n = n
        self.nfun = fs.nfun
        self.groups = []   # (f0, f1, origin[3], values[nf, ex, ey, ez], lo[3], hi[3])
        f = 0
        while f < fs.nfun:
            g = f + 1
            while g < fs.nfun and np.array_equal(fs.box[g], fs.box[f]):
                g += 1
            ex, ey, ez = (int(v) for v in fs.box[f, 3:])
            vals = fs.val[fs.off[f]:fs.off[g]].reshape(g - f, ex, ey, ez)
            nzx = np.nonzero(np.any(vals != 0.0, axis=(0, 2, 3)))[0]
            nzy = np.nonzero(np.any(vals != 0.0, axis=(0, 1, 3)))[0]
            nzz = np.nonzero(np.any(vals != 0.0, axis=(0, 1, 2)))[0]
            if nzx.size == 0:
                lo = np.zeros(3, dtype=np.int64)
                hi = np.zeros(3, dtype=np.int64)
            else:
                lo = np.array([nzx[0], nzy[0], nzz[0]], dtype=np.int64)
                hi = np.array([nzx[-1] + 1, nzy[-1] + 1, nzz[-1] + 1], dtype=np.int64)
            self.groups.append((f, g, fs.box[f, :3].astype(np.int64), vals, lo, hi))
            f = g


def _runs(sa, la, sb, lb, n):
    """Common points of wrapped ranges [sa, sa+la) and [sb, sb+lb) (mod n), as runs
    (offset in a, offset in b, length)."""
    if la <= 0 or lb <= 0:
        return []
    shift = (sb - sa) % n
    out = []
    if shift < la:
        out.append((shift, 0, min(la, shift + lb) - shift))
    if shift + lb > n:
        ln = min(la, shift + lb - n)
        if ln > 0:
            out.append((0, n - shift, ln))
    return out


def _common(ga, gb, n):
    """Yield (slice_a, slice_b, gx, gy, gz) blocks of points common to the supports of two groups."""
    _, _, oa, _, loa, hia = ga
    _, _, ob, _, lob, hib = gb
    per_axis = []
    for ax in range(3):
        sa = int(oa[ax] + loa[ax])
        sb = int(ob[ax] + lob[ax])
        runs = _runs(sa, int(hia[ax] - loa[ax]), sb, int(hib[ax] - lob[ax]), n)
        if not runs:
            return
        per_axis.append([(int(loa[ax]) + ra, int(lob[ax]) + rb, ln, (sa + ra + np.arange(ln)) % n)
                         for (ra, rb, ln) in runs])
    for (ax, bx, lx, gx) in per_axis[0]:
        for (ay, by, ly, gy) in per_axis[1]:
            for (az, bz, lz, gz) in per_axis[2]:
                sa = (slice(None), slice(ax, ax + lx), slice(ay, ay + ly), slice(az, az + lz))
                sb = (slice(None), slice(bx, bx + lx), slice(by, by + ly), slice(bz, bz + lz))
                yield sa, sb, gx, gy, gz


def response_density(chi: BoxedSet, phi: BoxedSet, P):
    """rho_s(r) = sum_ab chi_a(r) P_s[a, b] phi_b(r) for a batch P[s, a, b]; returns [s, n, n, n]."""
    n = chi.n
    P = np.asarray(P)
    k = P.shape[0]
    rho = np.zeros((k, n, n, n))
    for ga in chi.groups:
        fa0, fa1, _, va, _, _ = ga
        for gb in phi.groups:
            fb0, fb1, _, vb, _, _ = gb
            Pab = P[:, fa0:fa1, fb0:fb1]
            if not np.any(Pab):
                continue
            for sa, sb, gx, gy, gz in _common(ga, gb, n):
                xa = va[sa]
                xb = vb[sb]
                shp = xa.shape[1:]
                xa = xa.reshape(xa.shape[0], -1)
                xb = xb.reshape(xb.shape[0], -1)
                # sum_a chi_a(r) * (sum_b P_ab phi_b(r))
                contrib = np.einsum("ar,sar->sr", xa, Pab @ xb).reshape((k,) + shp)
                rho[np.ix_(np.arange(k), gx, gy, gz)] += contrib
    return rho


def potential_integrals(chi: BoxedSet, phi: BoxedSet, V, dV):
    """V_s[a, b] = dV sum_r chi_a(r) V_s(r) phi_b(r) for potentials V[s, n, n, n]."""
    n = chi.n
    V = np.asarray(V)
    k = V.shape[0]
    out = np.zeros((k, chi.nfun, phi.nfun))
    for ga in chi.groups:
        fa0, fa1, _, va, _, _ = ga
        for gb in phi.groups:
            fb0, fb1, _, vb, _, _ = gb
            for sa, sb, gx, gy, gz in _common(ga, gb, n):
                xa = va[sa].reshape(fa1 - fa0, -1)
                xb = vb[sb].reshape(fb1 - fb0, -1)
                vsub = V[np.ix_(np.arange(k), gx, gy, gz)].reshape(k, -1)
                out[:, fa0:fa1, fb0:fb1] += dV * np.einsum("ar,sr,br->sab", xa, vsub, xb)
    return out


def full_grid(fs, n):
    """Scatter every function of a set onto the whole periodic grid: [nfun, n, n, n]."""
    out = np.zeros((fs.nfun, n, n, n))
    for f in range(fs.nfun):
        ox, oy, oz, ex, ey, ez = (int(v) for v in fs.box[f])
        vals = fs.val[fs.off[f]:fs.off[f + 1]].reshape(ex, ey, ez)
        gx = (ox + np.arange(ex)) % n
        gy = (oy + np.arange(ey)) % n
        gz = (oz + np.arange(ez)) % n
        out[f][np.ix_(gx, gy, gz)] += vals
    return out


def _inside(g, p, n):
    """Box offsets of grid point p in group g, or None when p is outside its nonzero support."""
    _, _, org, _, lo, hi = g
    off = (np.asarray(p, dtype=np.int64) - org) % n
    if np.all(off >= lo) and np.all(off < hi):
        return off
    return None


def values_at(bs: BoxedSet, p):
    """All function values of a set at one grid point p = (ix, iy, iz): a dense vector [nfun]."""
    out = np.zeros(bs.nfun)
    for g in bs.groups:
        off = _inside(g, p, bs.n)
        if off is not None:
            f0, f1, _, vals, _, _ = g
            out[f0:f1] = vals[:, off[0], off[1], off[2]]
    return out


def density_at(chi: BoxedSet, phi: BoxedSet, P, points):
    """rho_s(r) = sum_ab chi_a(r) P_s[a, b] phi_b(r) at the given grid points only: [s, npoints].
    The same definition as response_density, evaluated point by point (for workloads whose full
    grid is too large for the oracle)."""
    P = np.asarray(P)
    out = np.zeros((P.shape[0], len(points)))
    for i, p in enumerate(points):
        xc = values_at(chi, p)
        xp = values_at(phi, p)
        a = np.nonzero(xc)[0]
        b = np.nonzero(xp)[0]
        if a.size and b.size:
            out[:, i] = np.einsum("a,sab,b->s", xc[a], P[:, a][:, :, b], xp[b])
    return out


def integrals_at(chi: BoxedSet, phi: BoxedSet, V, dV, pairs):
    """V_s[a, b] = dV sum_r chi_a(r) V_s(r) phi_b(r) for the listed (a, b) pairs only: [s, npairs].
    The same sums as potential_integrals, over the common support of the two functions."""
    n = chi.n
    V = np.asarray(V)
    k = V.shape[0]

    def group_of(bs, f):
        for g in bs.groups:
            if g[0] <= f < g[1]:
                return g
        raise IndexError(f)

    out = np.zeros((k, len(pairs)))
    for i, (a, b) in enumerate(pairs):
        ga, gb = group_of(chi, a), group_of(phi, b)
        for sa, sb, gx, gy, gz in _common(ga, gb, n):
            xa = ga[3][a - ga[0]][sa[1:]].reshape(-1)
            xb = gb[3][b - gb[0]][sb[1:]].reshape(-1)
            vsub = V[np.ix_(np.arange(k), gx, gy, gz)].reshape(k, -1)
            out[:, i] += dV * (vsub @ (xa * xb))
    return out
