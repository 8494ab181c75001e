"""Argument marshalling of the Python binding, without a GPU: the atom-blocked (tddft_bsr) form of
a dense matrix holds exactly its nonzero atom blocks, in row-major order of (row atom, column
atom), and rebuilds the matrix; for uniform and for uneven function counts per atom."""
import numpy as np

from paper_1507_08157_gb300 import tddft


def _rebuild(row_ptr, col, blk_off, val, rc, cc):
    r0 = np.concatenate([[0], np.cumsum(rc)])
    c0 = np.concatenate([[0], np.cumsum(cc)])
    M = np.zeros((r0[-1], c0[-1]))
    for I in range(len(rc)):
        for b in range(row_ptr[I], row_ptr[I + 1]):
            J = col[b]
            assert blk_off[b + 1] - blk_off[b] == rc[I] * cc[J]
            M[r0[I]:r0[I + 1], c0[J]:c0[J + 1]] = val[blk_off[b]:blk_off[b + 1]].reshape(rc[I], cc[J])
        cols = col[row_ptr[I]:row_ptr[I + 1]]
        assert np.all(np.diff(cols) > 0)
    return M


def _case(rc, cc, seed):
    rng = np.random.default_rng(seed)
    na = len(rc)
    ra = np.repeat(np.arange(na), rc)
    ca = np.repeat(np.arange(na), cc)
    M = rng.standard_normal((ra.size, ca.size))
    keep = rng.random((na, na)) < 0.5
    M *= keep[ra][:, ca]
    return M, ra, ca, keep


def test_atom_bsr_uniform_counts():
    rc, cc = np.full(5, 9), np.full(5, 4)
    M, ra, ca, keep = _case(rc, cc, 1)
    rp, col, bo, val = tddft.atom_bsr(M, ra, ca, 5)
    assert rp[-1] == keep.sum()
    assert np.array_equal(_rebuild(rp, col, bo, val, rc, cc), M)


def test_atom_bsr_uneven_counts():
    rc, cc = np.array([3, 1, 4, 2]), np.array([2, 5, 1, 3])
    M, ra, ca, keep = _case(rc, cc, 2)
    rp, col, bo, val = tddft.atom_bsr(M, ra, ca, 4)
    assert rp[-1] == keep.sum()
    assert np.array_equal(_rebuild(rp, col, bo, val, rc, cc), M)
