"""ctypes binding of libtddft (include/tddft.h): argument marshalling only.

Every computation runs in the CUDA library. Arrays may be numpy (host) or torch CUDA float64
tensors (device); the library tells them apart. If the library has not been built this module
raises at load time: there is no CPU path.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

from .synthetic import System

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtddft.so")

OK, E_INVALID, E_NOMEM, E_CUDA, E_NOT_CONVERGED, E_BREAKDOWN, E_TIMEOUT, E_PAIRING = range(8)
FP64, MIXED = 0, 1
NOALLOC_MAX_STATES = 64        # TDDFT_NOALLOC_MAX_STATES of the header
MODE = {"full": 0, "tda": 1, "d_only": 2}
PRECOND = {"none": 0, "iter": 1, "learned": 2, "exact": 3}
FXC = {"none": 0, "lda": 1}

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)


class _Funcs(ctypes.Structure):
    _fields_ = [("nfun", ctypes.c_int32), ("atom", c_int32_p), ("box", c_int32_p),
                ("off", c_int64_p), ("val", c_double_p), ("val32", ctypes.POINTER(ctypes.c_float))]


class _System(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_double), ("n", ctypes.c_int32), ("natoms", ctypes.c_int32),
                ("pos", c_double_p), ("phi", _Funcs), ("chi", _Funcs),
                ("S_chi", c_double_p), ("S_phi", c_double_p), ("H_chi", c_double_p),
                ("H_phi", c_double_p), ("P_v", c_double_p), ("P_c", c_double_p),
                ("n0", c_double_p), ("fxc_kind", ctypes.c_int32),
                ("kernel_cutoff", ctypes.c_double)]


class _Bsr(ctypes.Structure):
    _fields_ = [("row_ptr", c_int64_p), ("col_idx", c_int32_p), ("blk_off", c_int64_p), ("val", c_double_p)]


class _SparseSystem(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_double), ("n", ctypes.c_int32), ("natoms", ctypes.c_int32),
                ("pos", c_double_p), ("phi", _Funcs), ("chi", _Funcs),
                ("S_chi", _Bsr), ("H_chi", _Bsr), ("P_c", _Bsr),
                ("S_phi", _Bsr), ("H_phi", _Bsr), ("P_v", _Bsr),
                ("n0", c_double_p), ("fxc_kind", ctypes.c_int32),
                ("kernel_cutoff", ctypes.c_double), ("density_kernel_cutoff", ctypes.c_double)]


class TuningEntry(ctypes.Structure):
    _fields_ = [("stage", ctypes.c_char * 32), ("kind", ctypes.c_int32), ("chi_chunk", ctypes.c_int32),
                ("phi_chunk", ctypes.c_int32), ("chosen", ctypes.c_int32), ("ms", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("precond_maxit", ctypes.c_int32),
                ("precond_tol", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("reapply_every", ctypes.c_int32),
                ("restart_every", ctypes.c_int32), ("precond_adaptive", ctypes.c_int32),
                ("spin_limit_cycles", ctypes.c_int64)]


class StageStats(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


SYMBOLS = sorted(["tddft_default_options", "tddft_create", "tddft_destroy", "tddft_last_error",
                  "tddft_dims", "tddft_apply", "tddft_response_density", "tddft_response_density_noalloc",
                  "tddft_response_potential",
                  "tddft_potential_integrals", "tddft_fxc", "tddft_state_create",
                  "tddft_state_destroy", "tddft_pcg_step", "tddft_solve", "tddft_state_get",
                  "tddft_subspace", "tddft_pattern", "tddft_profile", "tddft_profile_read",
                  "tddft_work", "tddft_mlp_create", "tddft_mlp_destroy", "tddft_mlp_last_error",
                  "tddft_mlp_size", "tddft_mlp_set", "tddft_mlp_get", "tddft_mlp_forward",
                  "tddft_mlp_loss_grad", "tddft_mlp_train", "tddft_learned_dims", "tddft_set_mlp",
                  "tddft_samples", "tddft_state_stats", "tddft_state_export",
                  "tddft_state_import", "tddft_create_batch", "tddft_solve_batch",
                  "tddft_oscillator_strengths", "tddft_spectrum", "tddft_joint_projector",
                  "tddft_wait_check", "tddft_create_sparse", "tddft_kernel_pattern",
                  "tddft_autotune"])

_lib = None
_live = weakref.WeakSet()      # open contexts and states, closed before interpreter shutdown
_closed_all = False


@atexit.register
def _close_all():
    global _closed_all
    for obj in [o for o in list(_live) if isinstance(o, State)]:
        obj.close()
    for obj in list(_live):
        obj.close()
    _closed_all = True


def load(path: str = LIB_PATH):
    """Load libtddft.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1507_08157_gb300.build`")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.tddft_default_options.argtypes = [ctypes.POINTER(_Options)]
    lib.tddft_default_options.restype = None
    lib.tddft_create.argtypes = [ctypes.POINTER(_System), ctypes.POINTER(_Options), vp, ctypes.POINTER(vp)]
    lib.tddft_create_sparse.argtypes = [ctypes.POINTER(_SparseSystem), ctypes.POINTER(_Options), vp,
                                        ctypes.POINTER(vp)]
    lib.tddft_kernel_pattern.argtypes = [vp, c_int64_p, c_int64_p, c_int64_p, c_int32_p, c_int64_p]
    lib.tddft_destroy.argtypes = [vp]
    lib.tddft_destroy.restype = None
    lib.tddft_last_error.argtypes = [vp]
    lib.tddft_last_error.restype = ctypes.c_char_p
    lib.tddft_dims.argtypes = [vp, c_int32_p, c_int32_p, c_int32_p]
    lib.tddft_apply.argtypes = [vp, ctypes.c_int32, vp, vp, vp, vp]
    for name in ("tddft_response_density", "tddft_response_potential", "tddft_potential_integrals"):
        getattr(lib, name).argtypes = [vp, ctypes.c_int32, vp, vp]
    lib.tddft_fxc.argtypes = [vp, vp]
    lib.tddft_autotune.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(TuningEntry), ctypes.c_int32, c_int32_p]
    lib.tddft_autotune.restype = ctypes.c_int
    lib.tddft_wait_check.argtypes = [vp]
    lib.tddft_wait_check.restype = ctypes.c_int
    lib.tddft_response_density_noalloc.argtypes = [vp, ctypes.c_int32, vp, vp]
    lib.tddft_response_density_noalloc.restype = ctypes.c_int
    lib.tddft_state_create.argtypes = [vp, ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.tddft_state_destroy.argtypes = [vp]
    lib.tddft_state_destroy.restype = None
    lib.tddft_pcg_step.argtypes = [vp, vp, vp, vp]
    lib.tddft_solve.argtypes = [vp, vp, vp, vp, c_int32_p]
    lib.tddft_state_get.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.tddft_subspace.argtypes = [vp, vp, vp, vp]
    lib.tddft_pattern.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
    lib.tddft_profile.argtypes = [vp, ctypes.c_int32]
    lib.tddft_profile_read.argtypes = [vp, ctypes.POINTER(StageStats), ctypes.c_int32, c_int32_p]
    lib.tddft_work.argtypes = [vp, c_double_p, c_double_p]
    i64 = ctypes.c_int64
    lib.tddft_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)]
    lib.tddft_mlp_destroy.argtypes = [vp]
    lib.tddft_mlp_destroy.restype = None
    lib.tddft_mlp_last_error.argtypes = [vp]
    lib.tddft_mlp_last_error.restype = ctypes.c_char_p
    lib.tddft_mlp_size.argtypes = [vp]
    lib.tddft_mlp_size.restype = i64
    lib.tddft_mlp_set.argtypes = [vp, vp]
    lib.tddft_mlp_get.argtypes = [vp, vp]
    lib.tddft_mlp_forward.argtypes = [vp, i64, vp, vp]
    lib.tddft_mlp_loss_grad.argtypes = [vp, i64, vp, vp, vp, c_double_p, vp]
    lib.tddft_mlp_train.argtypes = [vp, i64, vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, vp,
                                    c_double_p, c_double_p]
    lib.tddft_learned_dims.argtypes = [vp, c_int32_p, c_int32_p]
    lib.tddft_set_mlp.argtypes = [vp, vp]
    lib.tddft_samples.argtypes = [vp, vp, i64, vp, vp, vp, ctypes.POINTER(i64)]
    lib.tddft_state_stats.argtypes = [vp, c_int32_p, c_int32_p, ctypes.POINTER(i64)]
    lib.tddft_state_export.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.tddft_state_import.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.tddft_oscillator_strengths.argtypes = [vp, vp, vp, vp, vp]
    lib.tddft_joint_projector.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp]
    lib.tddft_spectrum.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_double, ctypes.c_int32, vp, vp]
    lib.tddft_create_batch.argtypes = [ctypes.POINTER(_System), ctypes.c_int32, ctypes.POINTER(_Options), vp,
                                       ctypes.POINTER(vp)]
    lib.tddft_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_int32,
                                      vp, vp, c_int32_p, c_int32_p]
    for name in ("tddft_create", "tddft_create_sparse", "tddft_kernel_pattern", "tddft_dims", "tddft_apply",
                 "tddft_response_density",
                 "tddft_response_potential", "tddft_potential_integrals", "tddft_fxc",
                 "tddft_state_create", "tddft_pcg_step", "tddft_solve", "tddft_state_get",
                 "tddft_subspace", "tddft_pattern", "tddft_profile", "tddft_profile_read",
                 "tddft_work", "tddft_mlp_create", "tddft_mlp_set", "tddft_mlp_get", "tddft_mlp_forward",
                 "tddft_mlp_loss_grad", "tddft_mlp_train", "tddft_learned_dims", "tddft_set_mlp",
                 "tddft_samples", "tddft_state_stats", "tddft_state_export",
                 "tddft_state_import", "tddft_create_batch", "tddft_solve_batch",
                 "tddft_oscillator_strengths", "tddft_spectrum", "tddft_joint_projector"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class TddftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tddft status {status}: {msg}")
        self.status = status


def _ptr(a):
    """Address of a numpy array or a torch tensor (must be float64 and contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(type(a))


def _options(precision="fp64", mode="full", precond="iter", precond_tol=1e-4, precond_maxit=50,
             tol=1e-6, max_iter=500, reapply_every=10, restart_every=10, precond_adaptive=False,
             spin_limit_cycles=0):
    o = _Options()
    load().tddft_default_options(ctypes.byref(o))
    o.precision = FP64 if precision == "fp64" else MIXED
    o.mode = MODE[mode]
    o.precond = PRECOND[precond]
    o.precond_tol = precond_tol
    o.precond_maxit = precond_maxit
    o.tol = tol
    o.max_iter = max_iter
    o.reapply_every = reapply_every
    o.restart_every = restart_every
    o.precond_adaptive = 1 if precond_adaptive else 0
    o.spin_limit_cycles = int(spin_limit_cycles)
    return o


def _marshal(sys: System, fxc="lda", matrices=True):
    """The tddft_system view of a System; `keep` holds the arrays it points into (matrices=False:
    only the geometry, functions and n0)."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt)))

    def funcs(fs):
        f = _Funcs()
        f.nfun = fs.nfun
        f.atom = arr(fs.atom, np.int32)
        f.box = arr(fs.box, np.int32)
        f.off = arr(fs.off, np.int64)
        if fs.val.dtype == np.float32:
            f.val32 = arr(fs.val, np.float32)     # float32 tables pass as they are
        else:
            f.val = arr(fs.val, np.float64)
        return f

    s = _System()
    s.cell = sys.cell
    s.n = sys.n
    s.natoms = sys.natoms
    s.pos = arr(sys.pos, np.float64)
    s.phi = funcs(sys.phi)
    s.chi = funcs(sys.chi)
    if matrices:
        s.S_chi = arr(sys.S_chi, np.float64)
        s.S_phi = arr(sys.S_phi, np.float64)
        s.H_chi = arr(sys.H_chi, np.float64)
        s.H_phi = arr(sys.H_phi, np.float64)
        s.P_v = arr(sys.P_v, np.float64)
        s.P_c = arr(sys.P_c, np.float64)
    s.n0 = arr(sys.n0, np.float64)
    s.fxc_kind = FXC[fxc]
    s.kernel_cutoff = sys.kernel_cutoff
    return s, keep


def atom_counts(atom, natoms):
    """Functions per atom of a set grouped by atom."""
    return np.bincount(np.asarray(atom, dtype=np.int64), minlength=natoms)


def atom_bsr(M, row_atom, col_atom, natoms):
    """The atom-blocked form (tddft_bsr) of a dense matrix whose rows and columns are functions
    grouped by atom: blocks with a nonzero entry, in row-major order of (row atom, column atom).
    Returns (row_ptr int64 [natoms+1], col_idx int32 [nnzb], blk_off int64 [nnzb+1], val float64)."""
    M = np.asarray(M, dtype=np.float64)
    rc, cc = atom_counts(row_atom, natoms), atom_counts(col_atom, natoms)
    r0 = np.concatenate([[0], np.cumsum(rc)])
    c0 = np.concatenate([[0], np.cumsum(cc)])
    if np.all(rc == rc[0]) and np.all(cc == cc[0]) and rc[0] > 0 and cc[0] > 0:
        nr, nc = int(rc[0]), int(cc[0])
        blocks = M.reshape(natoms, nr, natoms, nc).transpose(0, 2, 1, 3)
        keep = np.any(blocks != 0.0, axis=(2, 3))
        I, J = np.nonzero(keep)
        val = np.ascontiguousarray(blocks[I, J]).ravel()
        sizes = np.full(I.size, nr * nc, dtype=np.int64)
    else:
        I, J, parts = [], [], []
        for a in range(natoms):
            for b in range(natoms):
                blk = M[r0[a]:r0[a + 1], c0[b]:c0[b + 1]]
                if blk.size and np.any(blk != 0.0):
                    I.append(a)
                    J.append(b)
                    parts.append(blk.ravel())
        I, J = np.array(I, dtype=np.int64), np.array(J, dtype=np.int64)
        val = np.concatenate(parts) if parts else np.zeros(0)
        sizes = rc[I] * cc[J]
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(I, minlength=natoms))]).astype(np.int64)
    blk_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return row_ptr, J.astype(np.int32), blk_off, val


def _marshal_sparse(sys: System, fxc="lda"):
    """The tddft_sparse_system view of a System (matrices in atom-blocked form)."""
    base, keep = _marshal(sys, fxc, matrices=False)

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt)))

    def bsr(M, ra, ca):
        rp, ci, bo, v = atom_bsr(M, ra, ca, sys.natoms)
        b = _Bsr()
        b.row_ptr, b.col_idx, b.blk_off, b.val = arr(rp, np.int64), arr(ci, np.int32), arr(bo, np.int64), arr(v, np.float64)
        return b

    s = _SparseSystem()
    s.cell, s.n, s.natoms, s.pos, s.phi, s.chi = base.cell, base.n, base.natoms, base.pos, base.phi, base.chi
    ca, pa = sys.chi.atom, sys.phi.atom
    s.S_chi, s.H_chi, s.P_c = bsr(sys.S_chi, ca, ca), bsr(sys.H_chi, ca, ca), bsr(sys.P_c, ca, ca)
    s.S_phi, s.H_phi, s.P_v = bsr(sys.S_phi, pa, pa), bsr(sys.H_phi, pa, pa), bsr(sys.P_v, pa, pa)
    s.n0, s.fxc_kind = base.n0, base.fxc_kind
    s.kernel_cutoff = sys.kernel_cutoff
    s.density_kernel_cutoff = getattr(sys, "density_kernel_cutoff", 0.0)
    return s, keep


def joint_projector(S_joint, S_joint_phi, P_v, stream=None):
    """P^c of the joint representation (Eq. proj) on the device (tddft_joint_projector)."""
    lib = load()
    S = np.ascontiguousarray(S_joint, dtype=np.float64)
    Sjp = np.ascontiguousarray(S_joint_phi, dtype=np.float64)
    Pv = np.ascontiguousarray(P_v, dtype=np.float64)
    out = np.empty_like(S)
    rc = lib.tddft_joint_projector(ctypes.c_void_p(stream) if stream is not None else None, S.shape[0], Pv.shape[0],
                                   S.ctypes.data, Sjp.ctypes.data, Pv.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise TddftError(rc, "tddft_joint_projector failed (see stderr)")
    return out


def create_batch(systems, fxc="lda", stream=None, **opts):
    """Contexts for several systems at once (tddft_create_batch): each owns its own stream."""
    lib = load()
    n = len(systems)
    views = [_marshal(sy_, fxc) for sy_ in systems]
    arr = (_System * n)(*[v[0] for v in views])
    out = (ctypes.c_void_p * n)()
    options = _options(**opts)
    st = ctypes.c_void_p(stream) if stream is not None else None
    rc = lib.tddft_create_batch(arr, n, ctypes.byref(options), st, out)
    if rc != OK:
        raise TddftError(rc, "tddft_create_batch failed (see stderr)")
    return [Context(sy_, _handle=ctypes.c_void_p(out[i]), **opts) for i, sy_ in enumerate(systems)]


def solve_batch(states, nthreads=0):
    """tddft_solve_batch over states of distinct contexts. Returns per system (omega, resid),
    the iteration counts and the statuses."""
    lib = load()
    n = len(states)
    ks = [s_.k for s_ in states]
    om, res = np.zeros(sum(ks)), np.zeros(sum(ks))
    it = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    cs = (ctypes.c_void_p * n)(*[s_.ctx._ctx.value for s_ in states])
    ss = (ctypes.c_void_p * n)(*[s_._st.value for s_ in states])
    rc = lib.tddft_solve_batch(cs, ss, n, nthreads, om.ctypes.data, res.ctypes.data,
                               it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc == E_INVALID:
        raise TddftError(rc, "tddft_solve_batch: bad arguments")
    off = np.concatenate([[0], np.cumsum(ks)])
    return ([(om[off[i]:off[i + 1]], res[off[i]:off[i + 1]]) for i in range(n)], it, status)


class Context:
    """One system on the GPU (tddft_create). Keyword options follow tddft_options."""

    def __init__(self, sys: System, fxc="lda", stream=None, _handle=None, sparse=False, **opts):
        """sparse=True: the truncated (linear-scaling) form (tddft_create_sparse); every chi x phi
        array then has the shape [k][nnz] of the kernel pattern (see to_pattern / from_pattern)."""
        lib = load()
        self._lib = lib
        self.sys = sys
        self.sparse = bool(sparse)
        self.options = _options(**opts)
        if _handle is None:
            ctx = ctypes.c_void_p()
            st = ctypes.c_void_p(stream) if stream is not None else None
            if self.sparse:
                s, keep = _marshal_sparse(sys, fxc)
                rc = lib.tddft_create_sparse(ctypes.byref(s), ctypes.byref(self.options), st, ctypes.byref(ctx))
            else:
                s, keep = _marshal(sys, fxc)
                rc = lib.tddft_create(ctypes.byref(s), ctypes.byref(self.options), st, ctypes.byref(ctx))
            if rc != OK:
                raise TddftError(rc, "tddft_create failed (see stderr)")
        else:
            ctx = _handle
        self._ctx = ctx
        self.nc, self.nv, self.n = sys.chi.nfun, sys.phi.nfun, sys.n
        self.natoms = sys.natoms
        self._states = weakref.WeakSet()
        _live.add(self)
        if self.sparse:
            self._pattern_arrays()

    def _pattern_arrays(self):
        nnzb, nnz = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.tddft_kernel_pattern(self._ctx, ctypes.byref(nnzb), ctypes.byref(nnz), None, None, None))
        self.nnz = int(nnz.value)
        self.kp_row_ptr = np.zeros(self.natoms + 1, dtype=np.int64)
        self.kp_col = np.zeros(int(nnzb.value), dtype=np.int32)
        self.kp_blk_off = np.zeros(int(nnzb.value) + 1, dtype=np.int64)
        self._check(self._lib.tddft_kernel_pattern(
            self._ctx, None, None, self.kp_row_ptr.ctypes.data_as(c_int64_p),
            self.kp_col.ctypes.data_as(c_int32_p), self.kp_blk_off.ctypes.data_as(c_int64_p)))
        # (row, column) of every pattern value in the dense chi x phi matrix
        rc = atom_counts(self.sys.chi.atom, self.natoms)
        cc = atom_counts(self.sys.phi.atom, self.natoms)
        r0 = np.concatenate([[0], np.cumsum(rc)])
        c0 = np.concatenate([[0], np.cumsum(cc)])
        rows, cols = [], []
        for I in range(self.natoms):
            for b in range(self.kp_row_ptr[I], self.kp_row_ptr[I + 1]):
                J = int(self.kp_col[b])
                rr, cc_ = np.meshgrid(np.arange(r0[I], r0[I + 1]), np.arange(c0[J], c0[J + 1]), indexing="ij")
                rows.append(rr.ravel())
                cols.append(cc_.ravel())
        self.kp_rows = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
        self.kp_cols = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)

    def to_pattern(self, X):
        """Dense [k][N_chi][N_phi] -> [k][nnz]: the kernel pattern's entries in the boundary order."""
        X = np.asarray(X, dtype=np.float64)
        return np.ascontiguousarray(X[:, self.kp_rows, self.kp_cols])

    def from_pattern(self, x):
        """[k][nnz] -> dense [k][N_chi][N_phi] (zero off the pattern)."""
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros((x.shape[0], self.nc, self.nv))
        out[:, self.kp_rows, self.kp_cols] = x
        return out

    def _kshape(self, k):
        return (k, self.nnz) if self.sparse else (k, self.nc, self.nv)

    def close(self):
        if getattr(self, "_ctx", None):
            for st in list(getattr(self, "_states", ())):
                st.close()
            self._lib.tddft_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise TddftError(rc, self._lib.tddft_last_error(self._ctx).decode())

    def last_error(self):
        """The message of the context's last failed call (tddft_last_error)."""
        return self._lib.tddft_last_error(self._ctx).decode()

    def _out(self, like, shape):
        if like is not None and hasattr(like, "data_ptr"):
            import torch
            return torch.empty(shape, dtype=torch.float64, device=like.device)
        return np.empty(shape)

    # -- Eq. operator_RPA --------------------------------------------------------------------------
    def apply(self, Pp, Pq, fp=None, fq=None):
        k = Pp.shape[0]
        shape = self._kshape(k)
        fp = self._out(Pp, shape) if fp is None else fp
        fq = self._out(Pp, shape) if fq is None else fq
        self._check(self._lib.tddft_apply(self._ctx, k, _ptr(Pp), _ptr(Pq), _ptr(fp), _ptr(fq)))
        return fp, fq

    def response_density(self, P):
        out = self._out(P, (P.shape[0], self.n, self.n, self.n))
        self._check(self._lib.tddft_response_density(self._ctx, P.shape[0], _ptr(P), _ptr(out)))
        return out

    def response_density_noalloc(self, P, rho):
        """rho = density of P through the allocation-free entry point; P [k][N_chi][N_phi] and
        rho [k][n][n][n] are contiguous float32 CUDA tensors owned by the caller."""
        import torch
        for a in (P, rho):
            if not (a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()):
                raise ValueError("P and rho must be contiguous float32 CUDA tensors")
        k = P.shape[0]
        if tuple(P.shape[1:]) != (self.nc, self.nv) or tuple(rho.shape) != (k, self.n, self.n, self.n):
            raise ValueError("P must be [k][N_chi][N_phi] and rho [k][n][n][n]")
        self._check(self._lib.tddft_response_density_noalloc(self._ctx, k, P.data_ptr(), rho.data_ptr()))
        return rho

    def response_potential(self, rho):
        out = self._out(rho, rho.shape)
        self._check(self._lib.tddft_response_potential(self._ctx, rho.shape[0], _ptr(rho), _ptr(out)))
        return out

    def potential_integrals(self, V):
        out = self._out(V, self._kshape(V.shape[0]))
        self._check(self._lib.tddft_potential_integrals(self._ctx, V.shape[0], _ptr(V), _ptr(out)))
        return out

    def autotune(self, k):
        """tddft_autotune: time the candidate unit cuts of the grid kernels for k states and keep the
        fastest; returns one dict per candidate."""
        buf = (TuningEntry * 64)()
        n = ctypes.c_int32(0)
        self._check(self._lib.tddft_autotune(self._ctx, k, buf, 64, ctypes.byref(n)))
        return [{"stage": buf[i].stage.decode(), "kind": "units" if buf[i].kind else "per-tile",
                 "chi_chunk": buf[i].chi_chunk, "phi_chunk": buf[i].phi_chunk, "ms": buf[i].ms,
                 "chosen": bool(buf[i].chosen)} for i in range(min(n.value, 64))]

    def wait_check(self):
        """Status of tddft_wait_check: a kernel whose bounded wait must expire (E_TIMEOUT expected)."""
        return int(self._lib.tddft_wait_check(self._ctx))

    def fxc(self):
        out = np.empty((self.n, self.n, self.n))
        self._check(self._lib.tddft_fxc(self._ctx, _ptr(out)))
        return out

    def pattern(self):
        m = np.empty((self.natoms, self.natoms), dtype=np.uint8)
        self._check(self._lib.tddft_pattern(self._ctx, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
        return m

    def state(self, Y0):
        return State(self, Y0)

    def spectrum(self, omega, f, E, gamma):
        """S(E) = sum_i f_i (gamma / pi) / ((E - omega_i)^2 + gamma^2) on the device (tddft_spectrum)."""
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        E = np.ascontiguousarray(E, dtype=np.float64)
        S = np.empty_like(E)
        self._check(self._lib.tddft_spectrum(self._ctx, omega.size, omega.ctypes.data, f.ctypes.data, gamma,
                                             E.size, E.ctypes.data, S.ctypes.data))
        return S

    def import_state(self, blob):
        """A state resumed from the bytes of State.export (tddft_state_import)."""
        return State(self, None, blob=bytes(blob))

    def profile(self, enable=True):
        self._check(self._lib.tddft_profile(self._ctx, 1 if enable else 0))

    def profile_read(self):
        """Per-stage {name: (launches, ms, flops, bytes)} since profiling was enabled."""
        buf = (StageStats * 16)()
        n = ctypes.c_int32(0)
        self._check(self._lib.tddft_profile_read(self._ctx, buf, 16, ctypes.byref(n)))
        return {buf[i].name.decode(): (int(buf[i].launches), buf[i].ms, buf[i].flops, buf[i].bytes)
                for i in range(n.value)}

    # -- learned atom-block preconditioner ---------------------------------------------------------
    def learned_dims(self):
        """(n_b, n_f): block and feature lengths of the learned preconditioner's rows."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.tddft_learned_dims(self._ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_mlp(self, mlp):
        """Bind the model used by precond="learned" (None unbinds)."""
        self._mlp = mlp
        self._check(self._lib.tddft_set_mlp(self._ctx, mlp._m if mlp is not None else None))

    def samples(self, state):
        """Training rows (X, T, w) at the state's iterate, as float32 CUDA tensors."""
        import torch
        n_b, n_f = self.learned_dims()
        rows = state.k * self.natoms ** 2
        X = torch.empty((rows, n_b + n_f), dtype=torch.float32, device="cuda")
        T = torch.empty((rows, n_b), dtype=torch.float32, device="cuda")
        w = torch.empty((rows,), dtype=torch.float32, device="cuda")
        cnt = ctypes.c_int64(0)
        self._check(self._lib.tddft_samples(self._ctx, state._st, rows, X.data_ptr(), T.data_ptr(),
                                            w.data_ptr(), ctypes.byref(cnt)))
        return X, T, w

    def work(self):
        """(pair_points, table_values): algorithmic work of the grid contractions."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.tddft_work(self._ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value


class State:
    """Trial pairs of the PCG solver (tddft_state_create)."""

    def __init__(self, ctx: Context, Y0, blob=None):
        self.ctx = ctx
        st = ctypes.c_void_p()
        if blob is not None:
            buf = ctypes.create_string_buffer(blob, len(blob))
            ctx._check(ctx._lib.tddft_state_import(ctx._ctx, buf, len(blob), ctypes.byref(st)))
            self.k = int(np.frombuffer(blob, dtype=np.int32, count=1, offset=16)[0])
        else:
            self.k = Y0.shape[0]
            Y0 = np.ascontiguousarray(Y0, dtype=np.float64) if isinstance(Y0, np.ndarray) else Y0
            ctx._check(ctx._lib.tddft_state_create(ctx._ctx, self.k, _ptr(Y0), ctypes.byref(st)))
        self._st = st
        ctx._states.add(self)
        _live.add(self)

    def close(self):
        if getattr(self, "_st", None):
            if getattr(self.ctx, "_ctx", None):
                self.ctx._lib.tddft_state_destroy(self._st)
            self._st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self):
        om, res = np.empty(self.k), np.empty(self.k)
        self.ctx._check(self.ctx._lib.tddft_pcg_step(self.ctx._ctx, self._st, _ptr(om), _ptr(res)))
        return om, res

    def solve(self):
        """Returns (omega, resid, iters, status); status is OK, NOT_CONVERGED or PAIRING."""
        om, res = np.empty(self.k), np.empty(self.k)
        it = ctypes.c_int32(0)
        rc = self.ctx._lib.tddft_solve(self.ctx._ctx, self._st, _ptr(om), _ptr(res), ctypes.byref(it))
        if rc not in (OK, E_NOT_CONVERGED, E_PAIRING):
            self.ctx._check(rc)
        return om, res, int(it.value), rc

    def get(self):
        shape = self.ctx._kshape(self.k)
        out = {name: np.empty(shape) for name in ("Pp", "Pq", "fp", "fq", "Lp", "Lq")}
        self.ctx._check(self.ctx._lib.tddft_state_get(
            self.ctx._ctx, self._st, *(_ptr(out[n]) for n in ("Pp", "Pq", "fp", "fq", "Lp", "Lq"))))
        return out

    def oscillator_strengths(self):
        """(omega [k], f [k], mu [k, 3]) of the current Ritz pairs (tddft_oscillator_strengths)."""
        om, f, mu = np.empty(self.k), np.empty(self.k), np.empty((self.k, 3))
        self.ctx._check(self.ctx._lib.tddft_oscillator_strengths(self.ctx._ctx, self._st, om.ctypes.data,
                                                                 f.ctypes.data, mu.ctypes.data))
        return om, f, mu

    def export(self):
        """The state as checkpoint bytes (tddft_state_export)."""
        n = ctypes.c_size_t(0)
        self.ctx._check(self.ctx._lib.tddft_state_export(self.ctx._ctx, self._st, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self.ctx._check(self.ctx._lib.tddft_state_export(self.ctx._ctx, self._st, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def stats(self):
        """(PCG steps, preconditioner fallbacks (learned to CG, truncated-form CG to the gradient),
        inner CG iterations)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self.ctx._check(self.ctx._lib.tddft_state_stats(self._st, ctypes.byref(a), ctypes.byref(b),
                                                        ctypes.byref(c)))
        return a.value, b.value, c.value

    def subspace(self):
        om, pr = np.empty(self.k), np.empty(2 * self.k)
        self.ctx._check(self.ctx._lib.tddft_subspace(self.ctx._ctx, self._st, _ptr(om), _ptr(pr)))
        return om, pr.reshape(self.k, 2)


class Mlp:
    """The model of the learned preconditioner (tddft_mlp_*): features (n_f) -> width -> width ->
    an n_b x n_b map A, applied to the block part of each row. Rows and targets are float32 CUDA
    tensors; parameters move as float32 numpy vectors."""

    def __init__(self, n_block, n_feat, width):
        lib = load()
        self._lib = lib
        m = ctypes.c_void_p()
        rc = lib.tddft_mlp_create(n_block, n_feat, width, ctypes.byref(m))
        if rc != OK:
            raise TddftError(rc, "tddft_mlp_create failed")
        self._m = m
        self.n_block, self.n_feat, self.width = n_block, n_feat, width
        self.n_in = n_block + n_feat
        self.size = int(lib.tddft_mlp_size(m))
        _live.add(self)

    def close(self):
        if getattr(self, "_m", None):
            self._lib.tddft_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise TddftError(rc, self._lib.tddft_mlp_last_error(self._m).decode())

    @staticmethod
    def _dev(a, cols):
        import torch
        if not (a.is_cuda and a.dtype == torch.float32 and a.is_contiguous() and a.shape[1] == cols):
            raise ValueError(f"expected a contiguous float32 CUDA tensor with {cols} columns")
        return a.data_ptr()

    def set(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        if theta.size != self.size:
            raise ValueError("parameter vector has the wrong length")
        self._check(self._lib.tddft_mlp_set(self._m, theta.ctypes.data))

    def get(self):
        out = np.empty(self.size, dtype=np.float32)
        self._check(self._lib.tddft_mlp_get(self._m, out.ctypes.data))
        return out

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], self.n_block), dtype=torch.float32, device=X.device)
        self._check(self._lib.tddft_mlp_forward(self._m, X.shape[0], self._dev(X, self.n_in), Y.data_ptr()))
        return Y

    @staticmethod
    def _weights(w, n):
        import torch
        if w is None:
            return None
        if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous() and w.numel() == n):
            raise ValueError("row weights must be a contiguous float32 CUDA tensor of n entries")
        return w.data_ptr()

    def loss_grad(self, X, T, w=None):
        loss = ctypes.c_double()
        g = np.empty(self.size, dtype=np.float32)
        self._check(self._lib.tddft_mlp_loss_grad(self._m, X.shape[0], self._dev(X, self.n_in),
                                                  self._dev(T, self.n_block), self._weights(w, X.shape[0]),
                                                  ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, X, T, steps, batch, lr, order, w=None):
        order = np.ascontiguousarray(order, dtype=np.int64)
        if order.size < steps * batch:
            raise ValueError("order holds fewer than steps * batch indices")
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.tddft_mlp_train(self._m, X.shape[0], self._dev(X, self.n_in),
                                              self._dev(T, self.n_block), self._weights(w, X.shape[0]), steps,
                                              batch, lr, order.ctypes.data, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value
