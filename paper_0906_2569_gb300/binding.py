"""ctypes binding of libhpsi's C ABI (include/hpsi.h), with the same names.

Argument marshalling only: every step of H|psi> and of the Davidson solver runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (complex128); host arrays are numpy.  If the
library is missing, ``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhpsi.so")

HPSI_OK, HPSI_EINVAL, HPSI_ENOMEM, HPSI_ECUDA = 0, -1, -2, -3
HPSI_ENOTCONV, HPSI_ESINGULAR, HPSI_ETIMEOUT, HPSI_ENODEV = -4, -5, -6, -7
HPSI_FP64, HPSI_MIXED = 0, 1
HPSI_OPT_PRECOND_TAU, HPSI_OPT_PRECOND_SHIFT, HPSI_OPT_KERNEL_TIMING, HPSI_OPT_NL_TERMS = 1, 2, 3, 4
HPSI_OPT_LOCAL_PATH, HPSI_OPT_TC_KSPLIT, HPSI_OPT_FINAL_FP64, HPSI_OPT_BASIS, HPSI_OPT_AUTOTUNE = 5, 6, 7, 8, 9
HPSI_OPT_EIGENSOLVER, HPSI_OPT_FP32_GEMM = 10, 11
HPSI_OPT_LOCKING, HPSI_OPT_LOCK_BATCH, HPSI_OPT_LOCK_BASIS, HPSI_OPT_THICK_RESTART = 12, 13, 14, 15
HPSI_OPT_RITZ_SPLIT, HPSI_OPT_REORTH_TEST, HPSI_OPT_CG_TMIN = 16, 17, 18
HPSI_OPT_SCF_NMIX, HPSI_OPT_SCF_BETA, HPSI_OPT_SCF_DAVIDSON_TOL, HPSI_OPT_GAMMA_GEMM = 19, 20, 21, 22
HPSI_OPT_EIGH_DF = 23
HPSI_OPT_PERSISTENT = 24
HPSI_OPT_BATCH_NL = 25
KERNELS = ("inv_zy", "xvx_y", "fwd_z", "calbec", "dscale", "addvus", "split", "davidson", "eigh", "tridiag", "gamma", "scf", "fock",
           "batch")
HPSI_K_AT_FP64 = 16   # added to a class: only its launches made while H was applied in float64
STATUS_NAMES = {0: "HPSI_OK", -1: "HPSI_EINVAL", -2: "HPSI_ENOMEM", -3: "HPSI_ECUDA", -4: "HPSI_ENOTCONV",
                -5: "HPSI_ESINGULAR", -6: "HPSI_ETIMEOUT", -7: "HPSI_ENODEV"}

EXPORTS = ("hpsi_gsphere", "hpsi_setup", "hpsi_setup_cells", "hpsi_nprob", "hpsi_npw", "hpsi_nproj", "hpsi_apply",
           "hpsi_apply_batch", "hpsi_apply_noalloc", "hpsi_apply_gamma", "davidson_solve", "davidson_solve_gamma", "hpsi_scf", "hpsi_fock_apply", "hpsi_eigh_lowest_sym", "cg_solve", "hpsi_eigh_lowest", "hpsi_set_option", "hpsi_kernel_stats", "hpsi_sync", "hpsi_selftest_timeout", "hpsi_last_error",
           "hpsi_destroy")

_lib = None


class HpsiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _declare(lib):
    P, I, D, V = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.hpsi_gsphere.argtypes = [P(D), D, P(D), P(I), P(ctypes.c_int32), I]
    lib.hpsi_gsphere.restype = I
    lib.hpsi_setup.argtypes = [P(V), P(D), D, I, P(D), P(I), P(D), I, P(D), P(D), I, V]
    lib.hpsi_setup.restype = I
    lib.hpsi_setup_cells.argtypes = [P(V), I, P(D), P(D), P(I), P(P(D)), P(I), P(P(D)), P(P(D)), I, V]
    lib.hpsi_setup_cells.restype = I
    for f in (lib.hpsi_nprob,):
        f.argtypes = [V]
        f.restype = I
    for f in (lib.hpsi_npw, lib.hpsi_nproj):
        f.argtypes = [V, I]
        f.restype = I
    lib.hpsi_apply.argtypes = [V, I, V, V, I]
    lib.hpsi_apply.restype = I
    lib.hpsi_apply_noalloc.argtypes = [V, I, V, V, I]
    lib.hpsi_apply_noalloc.restype = I
    lib.hpsi_apply_batch.argtypes = [V, I, P(I), P(I), P(V), P(V)]
    lib.hpsi_apply_batch.restype = I
    lib.hpsi_apply_gamma.argtypes = [V, I, V, V, I]
    lib.hpsi_apply_gamma.restype = I
    lib.davidson_solve.argtypes = [V, I, I, D, I, V, P(D), P(I), P(D)]
    lib.davidson_solve_gamma.argtypes = [V, I, I, D, I, V, P(D), P(I), P(D)]
    lib.davidson_solve_gamma.restype = I
    lib.hpsi_scf.argtypes = [V, I, I, I, D, I, V, P(D), P(D), P(D), P(I), P(D)]
    lib.hpsi_scf.restype = I
    lib.hpsi_fock_apply.argtypes = [V, I, I, V, V, V, I, D, P(D)]
    lib.hpsi_fock_apply.restype = I
    lib.cg_solve.argtypes = [V, I, I, D, I, V, P(D), P(I), P(D)]
    lib.davidson_solve.restype = I
    lib.hpsi_eigh_lowest.argtypes = [V, I, V, I, I, V, V]
    lib.hpsi_eigh_lowest.restype = I
    lib.hpsi_eigh_lowest_sym.argtypes = [V, I, V, I, I, V, V]
    lib.hpsi_eigh_lowest_sym.restype = I
    lib.hpsi_set_option.argtypes = [V, I, D]
    lib.hpsi_set_option.restype = I
    lib.hpsi_kernel_stats.argtypes = [V, I, P(ctypes.c_longlong), P(D), I]
    lib.hpsi_kernel_stats.restype = I
    lib.hpsi_sync.argtypes = [V]
    lib.hpsi_sync.restype = I
    lib.hpsi_selftest_timeout.argtypes = [V]
    lib.hpsi_selftest_timeout.restype = I
    lib.hpsi_last_error.argtypes = [V]
    lib.hpsi_last_error.restype = ctypes.c_char_p
    lib.hpsi_destroy.argtypes = [V]
    lib.hpsi_destroy.restype = None
    return lib


def load(path: str | None = None):
    """Open libhpsi.so (built by ``paper_0906_2569_gb300.build``).  Raises if it is absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libhpsi.so not found at {p}: run paper_0906_2569_gb300.build.build() first "
                           "(there is no CPU fallback)")
    lib = _declare(ctypes.CDLL(p))
    if path is None:
        _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(lib, ctx, rc: int, what: str):
    if rc != HPSI_OK:
        msg = lib.hpsi_last_error(ctx)
        raise HpsiError(rc, f"{what}: {msg.decode() if msg else ''}")


def _ptr(x) -> int:
    """Address of a torch tensor (device or host) or a numpy array; the library reads and writes
    dense row-major blocks, so anything else is refused."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("libhpsi needs C-contiguous tensors")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("libhpsi needs C-contiguous arrays")
    return x.ctypes.data


def hpsi_gsphere(cell, ecut: float, k) -> np.ndarray:
    """Miller indices of the sphere, int32 [npw, 3], in the library's documented order."""
    lib = load()
    cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(3))
    npw = ctypes.c_int(0)
    _check(lib, None, lib.hpsi_gsphere(_dp(cell), float(ecut), _dp(k), ctypes.byref(npw), None, 0), "hpsi_gsphere")
    out = np.zeros((npw.value, 3), dtype=np.int32)
    _check(lib, None, lib.hpsi_gsphere(_dp(cell), float(ecut), _dp(k), ctypes.byref(npw),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), npw.value), "hpsi_gsphere")
    return out


class Context:
    """An hpsi_ctx: the operator for one cell and its k-points, or for a set of cells."""

    def __init__(self, handle, lib):
        self.handle = handle
        self.lib = lib

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hpsi_destroy(self.handle)
            self.handle = None

    def nprob(self) -> int:
        return self.lib.hpsi_nprob(self.handle)

    def npw(self, ik: int = 0) -> int:
        return self.lib.hpsi_npw(self.handle, ik)

    def nproj(self, ik: int = 0) -> int:
        return self.lib.hpsi_nproj(self.handle, ik)

    def last_error(self) -> str:
        return self.lib.hpsi_last_error(self.handle).decode()


def hpsi_setup(cell, ecut: float, kpts, fft, vloc_r, beta, dmat, precision: int = HPSI_FP64, stream=None) -> Context:
    """hpsi_setup(): ``beta`` is a list over k-points of complex128 [P][npw(k)] arrays (or None)."""
    lib = load()
    cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
    kpts = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
    fft_a = np.ascontiguousarray(np.asarray(fft, dtype=np.int32).reshape(3))
    v = np.ascontiguousarray(np.asarray(vloc_r, dtype=np.float64))
    nproj = 0 if beta is None or len(beta) == 0 else int(np.asarray(beta[0]).shape[0])
    if nproj:
        bcat = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.complex128).reshape(-1) for b in beta]))
        d = np.ascontiguousarray(np.asarray(dmat, dtype=np.complex128))
        bptr = bcat.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        dptr = d.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        bptr = dptr = None
    h = ctypes.c_void_p()
    rc = lib.hpsi_setup(ctypes.byref(h), _dp(cell), float(ecut), len(kpts), _dp(kpts),
                        fft_a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(v), nproj, bptr, dptr, int(precision),
                        ctypes.c_void_p(stream))
    _check(lib, None, rc, "hpsi_setup")
    return Context(h, lib)


def hpsi_setup_cells(cells, ecuts, ffts, vlocs, betas, dmats, precision: int = HPSI_FP64, stream=None) -> Context:
    """hpsi_setup_cells(): per-cell lists of lattice, cutoff, box, V(r), beta [P][npw], D."""
    lib = load()
    n = len(cells)
    ca = np.ascontiguousarray(np.asarray(cells, dtype=np.float64).reshape(n, 9))
    ea = np.ascontiguousarray(np.asarray(ecuts, dtype=np.float64).reshape(n))
    fa = np.ascontiguousarray(np.asarray(ffts, dtype=np.int32).reshape(n, 3))
    keep = []
    DP = ctypes.POINTER(ctypes.c_double)
    vp = (DP * n)()
    bp = (DP * n)()
    dp = (DP * n)()
    npj = np.zeros(n, dtype=np.int32)
    for i in range(n):
        v = np.ascontiguousarray(np.asarray(vlocs[i], dtype=np.float64))
        keep.append(v)
        vp[i] = _dp(v)
        b = betas[i]
        if b is not None and len(b):
            b = np.ascontiguousarray(np.asarray(b, dtype=np.complex128))
            d = np.ascontiguousarray(np.asarray(dmats[i], dtype=np.complex128))
            keep += [b, d]
            npj[i] = b.shape[0]
            bp[i] = b.view(np.float64).ctypes.data_as(DP)
            dp[i] = d.view(np.float64).ctypes.data_as(DP)
    h = ctypes.c_void_p()
    rc = lib.hpsi_setup_cells(ctypes.byref(h), n, _dp(ca), _dp(ea), fa.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              vp, npj.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), bp, dp, int(precision),
                              ctypes.c_void_p(stream))
    _check(lib, None, rc, "hpsi_setup_cells")
    return Context(h, lib)


def hpsi_apply(ctx: Context, ik: int, psi_in, hpsi_out, nbnd: int | None = None) -> None:
    """hpsi_apply(): device tensors (asynchronous) or host arrays / pinned tensors (synchronous)."""
    nb = int(psi_in.shape[0]) if nbnd is None else int(nbnd)
    rc = ctx.lib.hpsi_apply(ctx.handle, int(ik), ctypes.c_void_p(_ptr(psi_in)), ctypes.c_void_p(_ptr(hpsi_out)), nb)
    _check(ctx.lib, ctx.handle, rc, "hpsi_apply")


def hpsi_apply_noalloc(ctx: Context, ik: int, psi_in, hpsi_out, nbnd: int | None = None) -> None:
    """hpsi_apply_noalloc(): device tensors only; intermediates in the library's fixed array."""
    nb = int(psi_in.shape[0]) if nbnd is None else int(nbnd)
    rc = ctx.lib.hpsi_apply_noalloc(ctx.handle, int(ik), ctypes.c_void_p(_ptr(psi_in)),
                                    ctypes.c_void_p(_ptr(hpsi_out)), nb)
    _check(ctx.lib, ctx.handle, rc, "hpsi_apply_noalloc")


def hpsi_apply_gamma(ctx: Context, ik: int, psi_in, hpsi_out, nbnd: int | None = None) -> None:
    """hpsi_apply_gamma(): half-sphere complex128 [nbnd][(npw+1)//2], device or host, as hpsi_apply."""
    nb = int(psi_in.shape[0]) if nbnd is None else int(nbnd)
    rc = ctx.lib.hpsi_apply_gamma(ctx.handle, int(ik), ctypes.c_void_p(_ptr(psi_in)), ctypes.c_void_p(_ptr(hpsi_out)),
                                  nb)
    _check(ctx.lib, ctx.handle, rc, "hpsi_apply_gamma")


def hpsi_apply_batch(ctx: Context, probs, psi_list, hpsi_list) -> None:
    """hpsi_apply_batch(): lists of problem indices and device tensors [nbnd_i][npw_i]."""
    n = len(probs)
    pa = np.ascontiguousarray(np.asarray(probs, dtype=np.int32))
    nb = np.ascontiguousarray(np.asarray([int(x.shape[0]) for x in psi_list], dtype=np.int32))
    pin = (ctypes.c_void_p * n)(*[_ptr(x) for x in psi_list])
    pout = (ctypes.c_void_p * n)(*[_ptr(x) for x in hpsi_list])
    rc = ctx.lib.hpsi_apply_batch(ctx.handle, n, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), pin, pout)
    _check(ctx.lib, ctx.handle, rc, "hpsi_apply_batch")


def hpsi_eigh_lowest(ctx: Context, a_colmajor, n: int, lda: int, nwant: int, w_out, v_out) -> None:
    """hpsi_eigh_lowest(): device tensors; a_colmajor holds the matrix column-major (row i of the
    tensor is column i), only its upper triangle is read; v_out [nwant][n] receives one
    eigenvector per row, w_out [nwant] the eigenvalues ascending."""
    rc = ctx.lib.hpsi_eigh_lowest(ctx.handle, int(n), ctypes.c_void_p(_ptr(a_colmajor)), int(lda), int(nwant),
                                  ctypes.c_void_p(_ptr(w_out)), ctypes.c_void_p(_ptr(v_out)))
    _check(ctx.lib, ctx.handle, rc, "hpsi_eigh_lowest")


def hpsi_eigh_lowest_sym(ctx: Context, a_colmajor, n: int, lda: int, nwant: int, w_out, v_out) -> None:
    """hpsi_eigh_lowest_sym(): device float64 tensors, layouts as hpsi_eigh_lowest."""
    rc = ctx.lib.hpsi_eigh_lowest_sym(ctx.handle, int(n), ctypes.c_void_p(_ptr(a_colmajor)), int(lda), int(nwant),
                                      ctypes.c_void_p(_ptr(w_out)), ctypes.c_void_p(_ptr(v_out)))
    _check(ctx.lib, ctx.handle, rc, "hpsi_eigh_lowest_sym")


def hpsi_set_option(ctx: Context, option: int, value: float) -> None:
    """hpsi_set_option(): Davidson preconditioner options."""
    _check(ctx.lib, ctx.handle, ctx.lib.hpsi_set_option(ctx.handle, int(option), float(value)), "hpsi_set_option")


def hpsi_sync(ctx: Context) -> None:
    """hpsi_sync(): wait for the context's stream; raises on a device-side timeout."""
    _check(ctx.lib, ctx.handle, ctx.lib.hpsi_sync(ctx.handle), "hpsi_sync")


def hpsi_selftest_timeout(ctx: Context) -> None:
    """hpsi_selftest_timeout(): queue the bounded-wait self-test (the next hpsi_sync raises ETIMEOUT)."""
    _check(ctx.lib, ctx.handle, ctx.lib.hpsi_selftest_timeout(ctx.handle), "hpsi_selftest_timeout")


def hpsi_kernel_stats(ctx: Context, kernel: int, reset: bool = False):
    """hpsi_kernel_stats(): (launches, total ms) of a kernel class; -1 all classes, -2 band-applications."""
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    _check(ctx.lib, ctx.handle, ctx.lib.hpsi_kernel_stats(ctx.handle, int(kernel), ctypes.byref(n), ctypes.byref(ms),
                                                          int(bool(reset))), "hpsi_kernel_stats")
    return n.value, ms.value


def davidson_solve(ctx: Context, ik: int, psi_inout, tol: float, maxiter: int, raise_on_notconv: bool = True):
    """davidson_solve(): returns (eigenvalues, iterations, residual norms, status)."""
    nbnd = int(psi_inout.shape[0])
    eig = np.zeros(nbnd)
    res = np.zeros(nbnd)
    it = ctypes.c_int(0)
    rc = ctx.lib.davidson_solve(ctx.handle, int(ik), nbnd, float(tol), int(maxiter), ctypes.c_void_p(_ptr(psi_inout)),
                                _dp(eig), ctypes.byref(it), _dp(res))
    if rc != HPSI_ENOTCONV or raise_on_notconv:
        _check(ctx.lib, ctx.handle, rc, "davidson_solve")
    return eig, it.value, res, rc


def davidson_solve_gamma(ctx: Context, ik: int, psi_inout, tol: float, maxiter: int, raise_on_notconv: bool = True):
    """davidson_solve_gamma(): half-sphere coefficients in and out; returns (eigenvalues, iterations,
    residual norms, status)."""
    nbnd = int(psi_inout.shape[0])
    eig = np.zeros(nbnd)
    res = np.zeros(nbnd)
    it = ctypes.c_int(0)
    rc = ctx.lib.davidson_solve_gamma(ctx.handle, int(ik), nbnd, float(tol), int(maxiter),
                                      ctypes.c_void_p(_ptr(psi_inout)), _dp(eig), ctypes.byref(it), _dp(res))
    if rc != HPSI_ENOTCONV or raise_on_notconv:
        _check(ctx.lib, ctx.handle, rc, "davidson_solve_gamma")
    return eig, it.value, res, rc


def hpsi_scf(ctx: Context, ik: int, nocc: int, psi_inout, rho, tol: float, maxiter: int,
             raise_on_notconv: bool = True):
    """hpsi_scf(): rho (float64 [n1][n2][n3], C order) is overwritten by the converged input density;
    returns (eigenvalues, (E, E_HWF), iterations, scf-norm history, status)."""
    nbnd = int(psi_inout.shape[0])
    assert rho.dtype == np.float64 and rho.flags.c_contiguous
    eig = np.zeros(nbnd)
    en = np.zeros(2)
    hist = np.zeros(int(maxiter))
    it = ctypes.c_int(0)
    rc = ctx.lib.hpsi_scf(ctx.handle, int(ik), int(nocc), nbnd, float(tol), int(maxiter),
                          ctypes.c_void_p(_ptr(psi_inout)), _dp(rho), _dp(eig), _dp(en), ctypes.byref(it), _dp(hist))
    if rc != HPSI_ENOTCONV or raise_on_notconv:
        _check(ctx.lib, ctx.handle, rc, "hpsi_scf")
    return eig, (float(en[0]), float(en[1])), it.value, hist[:it.value], rc


def hpsi_fock_apply(ctx: Context, ik: int, occ, psi_in, vx_out, alpha: float = 1.0, energy: bool = False):
    """hpsi_fock_apply(): device tensors; returns E_x = Re sum_b <psi_b|V_x psi_b> when energy is set."""
    ex = ctypes.c_double(0.0)
    rc = ctx.lib.hpsi_fock_apply(ctx.handle, int(ik), int(occ.shape[0]), ctypes.c_void_p(_ptr(occ)),
                                 ctypes.c_void_p(_ptr(psi_in)), ctypes.c_void_p(_ptr(vx_out)), int(psi_in.shape[0]),
                                 float(alpha), ctypes.byref(ex) if energy else None)
    _check(ctx.lib, ctx.handle, rc, "hpsi_fock_apply")
    return ex.value if energy else None


def cg_solve(ctx: Context, ik: int, psi_inout, tol: float, maxiter: int, raise_on_notconv: bool = True):
    """cg_solve(): returns (eigenvalues in the order found, total CG steps, residual norms, status)."""
    nbnd = int(psi_inout.shape[0])
    eig = np.zeros(nbnd)
    res = np.zeros(nbnd)
    it = ctypes.c_int(0)
    rc = ctx.lib.cg_solve(ctx.handle, int(ik), nbnd, float(tol), int(maxiter), ctypes.c_void_p(_ptr(psi_inout)),
                          _dp(eig), ctypes.byref(it), _dp(res))
    if rc != HPSI_ENOTCONV or raise_on_notconv:
        _check(ctx.lib, ctx.handle, rc, "cg_solve")
    return eig, it.value, res, rc
