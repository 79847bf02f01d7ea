"""GB300 engine for state-averaged PNO-EOM-CCSD (arXiv:1802.06738).

A thin ctypes binding over ``libpnoeom.so`` (C ABI in ``include/pnoeom.h``).
Every step of setup, sigma and the Davidson solve runs inside the library on
the GPU; this module only marshals arguments.  ``build()`` compiles the CUDA
sources in-tree for sm_103a.  Importing never falls back to anything: when
the library is missing the entry points raise.
"""
from __future__ import annotations

import ctypes
import os

from .build import build, LIB_PATH  # noqa: F401

OK = 0
ERR_INVALID_ARG, ERR_NOMEM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
HOST, DEVICE = 0, 1
FP64, FP32, BF16 = 0, 1, 2


# kernel classes of the sigma program reported by pno_sigma_timing
SIGMA_CLASSES = 6


class PnoeomError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pnoeom error {code}: {msg}")
        self.code = code


class System(ctypes.Structure):
    _fields_ = [("o", ctypes.c_int), ("v", ctypes.c_int), ("naux", ctypes.c_int),
                ("eps", ctypes.c_void_p), ("B", ctypes.c_void_p), ("t1", ctypes.c_void_p),
                ("t2", ctypes.c_void_p), ("mem_space", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("t_pno", ctypes.c_double), ("t_osv", ctypes.c_double),
                ("nroots_sa", ctypes.c_int), ("nroots_solve", ctypes.c_int),
                ("precision", ctypes.c_int), ("refine_fp64", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("max_subspace", ctypes.c_int),
                ("res_tol", ctypes.c_double), ("e_tol", ctypes.c_double),
                ("state_specific", ctypes.c_int), ("t_pno_gs", ctypes.c_double)]


def make_opts(t_pno=1e-7, t_osv=-1.0, nroots=3, nroots_solve=None, precision=FP64, refine_fp64=0,
              max_iter=100, max_subspace=0, res_tol=1e-7, e_tol=1e-10, state_specific=0, t_pno_gs=0.0):
    """pnoeom_opts.  state_specific = k >= 1: PNOs from CIS root k's density alone (1-based);
    t_pno_gs > 0: T2 truncated to ground-state PNOs at that threshold."""
    return Opts(t_pno, t_osv, nroots, nroots if nroots_solve is None else nroots_solve,
                precision, refine_fp64, max_iter, max_subspace, res_tol, e_tol, state_specific, t_pno_gs)


_lib = None
EXPORTS = ["pnoeom_create", "pnoeom_destroy", "pnoeom_last_error", "pno_build", "pno_destroy",
           "pno_query", "pno_get_basis", "sigma", "davidson_solve", "pno_get_eigenvectors",
           "pno_get_cis", "pno_get_occupations", "pno_get_cis_vectors", "pnoeom_small_eig", "pno_build_seconds",
           "pno_set_timing", "pno_sigma_timing", "sigma_noalloc", "pno_autotune_info", "pno_tc_mma_flops",
           "pnoeom_batch_create", "pnoeom_batch_destroy", "pnoeom_batch_sigma", "pnoeom_batch_solve",
           "pnoeom_server_create", "pnoeom_server_destroy", "pnoeom_server_submit", "pnoeom_server_poll",
           "pnoeom_server_wait", "pnoeom_server_stats", "pnoeom_gemm_tf32x3", "pnoeom_device_status",
           "pno_solve_stats", "pnoeom_selftest_bounded_wait", "pnoeom_inject_alloc_failure",
           "pnoeom_alloc_live_bytes", "pnoeom_measure_peaks", "pno_solve_lowprec_energies"]


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PnoeomError(ERR_UNSUPPORTED, f"{LIB_PATH} not built; call paper_1802_06738_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
        L.pnoeom_create.argtypes = [ctypes.POINTER(vp), i, ctypes.c_size_t]
        L.pnoeom_destroy.argtypes = [vp]; L.pnoeom_destroy.restype = None
        L.pnoeom_last_error.argtypes = []; L.pnoeom_last_error.restype = ctypes.c_char_p
        L.pno_build.argtypes = [vp, ctypes.POINTER(System), ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
        L.pno_destroy.argtypes = [vp]; L.pno_destroy.restype = None
        L.pno_query.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
        L.pno_get_basis.argtypes = [vp, i, dp, dp]
        L.sigma.argtypes = [vp, vp, i, vp, vp, i, vp]
        L.sigma_noalloc.argtypes = [vp, vp, i, vp, vp, i, vp]
        L.pno_autotune_info.argtypes = [vp, i, ip, ip, dp, ip]
        L.pno_tc_mma_flops.argtypes = [vp, dp]
        L.pnoeom_batch_create.argtypes = [vp, ctypes.POINTER(vp), i, vp, ctypes.POINTER(vp)]
        L.pnoeom_batch_destroy.argtypes = [vp]; L.pnoeom_batch_destroy.restype = None
        L.pnoeom_batch_sigma.argtypes = [vp, vp, ip, ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]
        L.pnoeom_batch_solve.argtypes = [vp, vp, ctypes.POINTER(Opts), vp, dp, dp, ip, ip]
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.pnoeom_server_create.argtypes = [vp, ctypes.c_size_t, i, ctypes.POINTER(vp)]
        L.pnoeom_server_destroy.argtypes = [vp]; L.pnoeom_server_destroy.restype = None
        L.pnoeom_server_submit.argtypes = [vp, ctypes.POINTER(System), ctypes.POINTER(Opts), i64p]
        L.pnoeom_server_poll.argtypes = [vp, ctypes.c_int64, ip, dp, dp, ip, i64p, dp]
        L.pnoeom_server_wait.argtypes = [vp, ctypes.c_int64, d]
        L.pnoeom_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ip, ip, i64p, i64p, i64p]
        L.davidson_solve.argtypes = [vp, vp, ctypes.POINTER(Opts), vp, dp, dp, ip]
        L.pno_get_eigenvectors.argtypes = [vp, dp]
        L.pno_solve_stats.argtypes = [vp, i64p, i64p]
        L.pno_solve_lowprec_energies.argtypes = [vp, i, i, dp, ip]
        L.pno_get_cis.argtypes = [vp, dp]
        L.pno_get_occupations.argtypes = [vp, dp]
        L.pno_get_cis_vectors.argtypes = [vp, dp]
        L.pnoeom_small_eig.argtypes = [i, dp, dp, dp, dp]
        L.pnoeom_gemm_tf32x3.argtypes = [vp, vp, vp, vp, i, i, i, ctypes.c_float, vp]
        L.pnoeom_device_status.argtypes = [vp, i, ip]
        L.pno_build_seconds.argtypes = [vp]; L.pno_build_seconds.restype = d
        L.pnoeom_selftest_bounded_wait.argtypes = [vp, ctypes.c_longlong, vp, ip]
        L.pnoeom_inject_alloc_failure.argtypes = [ctypes.c_longlong]
        L.pnoeom_alloc_live_bytes.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        L.pnoeom_measure_peaks.argtypes = [vp, vp, dp, i]
        L.pno_set_timing.argtypes = [vp, i]
        L.pno_sigma_timing.argtypes = [vp, i, i, i, ctypes.POINTER(ctypes.c_char_p), ip, dp, dp, dp]
        _lib = L
    return _lib


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise PnoeomError(rc, lib().pnoeom_last_error().decode())
    return rc


def _dptr(a):
    import numpy as np
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pnoeom_small_eig(A):
    """Eigenvalues (complex) and unit right eigenvectors (columns) of a small
    dense matrix, computed by the library's host routine."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    wr, wi, VR = np.zeros(n), np.zeros(n), np.zeros((n, n))
    _check(lib().pnoeom_small_eig(n, _dptr(A), _dptr(wr), _dptr(wi), _dptr(VR)))
    return wr + 1j * wi, VR


class Context:
    """pnoeom_create / pnoeom_destroy."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        h = ctypes.c_void_p()
        _check(lib().pnoeom_create(ctypes.byref(h), device, hbm_budget_bytes))
        self.h = h

    def close(self):
        if self.h:
            lib().pnoeom_destroy(self.h)
            self.h = None

    def gemm_tf32x3(self, A, B, C, alpha=1.0, stream=None):
        """C += alpha * A @ B for row-major FP32 CUDA tensors (pnoeom_gemm_tf32x3)."""
        M, K = A.shape
        N = B.shape[1]
        _check(lib().pnoeom_gemm_tf32x3(self.h, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                        ctypes.c_void_p(C.data_ptr()), M, N, K, alpha, _stream_ptr(stream)))

    def measure_peaks(self, stream=None):
        """dict of the device's peak rates measured by the library's microbenchmarks
        (pnoeom_measure_peaks)."""
        import numpy as np
        out = np.zeros(8)
        _check(lib().pnoeom_measure_peaks(self.h, _stream_ptr(stream), _dptr(out), 8))
        keys = ["fp32_fma_tflops", "fp64_fma_tflops", "tc_bf16_tflops", "tc_tf32_tflops", "cublas_dgemm_tflops",
                "cublas_dgemm_emulated_tflops", "dgemm_emulated_max_rel_err", "sm_count"]
        return dict(zip(keys, map(float, out)))

    def device_status(self, clear=True):
        """Status word of the tensor-core kernels (0: every bounded wait completed)."""
        v = ctypes.c_int()
        _check(lib().pnoeom_device_status(self.h, 1 if clear else 0, ctypes.byref(v)))
        return v.value

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    return None if stream is None else ctypes.c_void_p(stream)


class PNO:
    """A built system: pno_build / pno_query / sigma / davidson_solve."""

    def __init__(self, ctx, eps, B, o, t1=None, t2=None, opts=None, stream=None, device_inputs=False):
        import numpy as np
        self.ctx = ctx
        self.opts = opts if opts is not None else make_opts()
        nmo = len(eps) if not device_inputs else int(eps.numel())
        v = nmo - o
        naux = B.shape[0]
        if device_inputs:   # torch tensors on the GPU
            self._keep = (eps, B, t1, t2)
            ptr = lambda x: None if x is None else x.data_ptr()
            sysd = System(o, v, naux, ptr(eps), ptr(B), ptr(t1), ptr(t2), DEVICE)
        else:
            eps = np.ascontiguousarray(eps, dtype=np.float64)
            B = np.ascontiguousarray(B, dtype=np.float64)
            t1 = None if t1 is None else np.ascontiguousarray(t1, dtype=np.float64)
            t2 = None if t2 is None else np.ascontiguousarray(t2, dtype=np.float64)
            self._keep = (eps, B, t1, t2)
            ptr = lambda x: None if x is None else x.ctypes.data
            sysd = System(o, v, naux, ptr(eps), ptr(B), ptr(t1), ptr(t2), HOST)
        h = ctypes.c_void_p()
        _check(lib().pno_build(ctx.h, ctypes.byref(sysd), ctypes.byref(self.opts), _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.o, self.v, self.naux = o, v, naux
        npairs = ctypes.c_int()
        nij = ctypes.POINTER(ctypes.c_int)()
        ni = ctypes.POINTER(ctypes.c_int)()
        L = ctypes.c_size_t()
        fp = ctypes.c_size_t()
        _check(lib().pno_query(h, ctypes.byref(npairs), ctypes.byref(nij), ctypes.byref(ni), ctypes.byref(L), ctypes.byref(fp)))
        self.npairs = npairs.value
        self.n_ij = np.array([nij[k] for k in range(self.npairs)], dtype=np.int64)
        self.n_i = np.array([ni[k] for k in range(o)], dtype=np.int64)
        self.length = L.value
        self.footprint = fp.value
        self.build_seconds = lib().pno_build_seconds(h)
        self.off_i = np.concatenate([[0], np.cumsum(self.n_i)])
        self.off_ij = self.off_i[-1] + np.concatenate([[0], np.cumsum(self.n_ij ** 2)])
        self.pairs = [(i, j) for i in range(o) for j in range(i, o)]

    def close(self):
        if getattr(self, "h", None):
            lib().pno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def basis(self, pair):
        """(U, fbar) of stored pair index ``pair`` (or OSV i when pair = -i-1)."""
        import numpy as np
        n = int(self.n_ij[pair]) if pair >= 0 else int(self.n_i[-pair - 1])
        U = np.zeros((self.v, n)); fb = np.zeros(n)
        _check(lib().pno_get_basis(self.h, pair, _dptr(U), _dptr(fb)))
        return U, fb

    def cis_energies(self):
        import numpy as np
        w = np.zeros(self.opts.nroots_sa)
        _check(lib().pno_get_cis(self.h, _dptr(w)))
        return w

    def cis_vectors(self):
        import numpy as np
        b = np.zeros((self.opts.nroots_sa, self.o, self.v))
        _check(lib().pno_get_cis_vectors(self.h, _dptr(b)))
        return b

    def occupations(self):
        """Eigenvalues of every state-averaged pair density, [npairs, v]."""
        import numpy as np
        occ = np.zeros((self.npairs, self.v))
        _check(lib().pno_get_occupations(self.h, _dptr(occ)))
        return occ

    def sigma(self, r, out, precision=FP64, stream=None):
        """sigma for a batch of packed vectors: r, out are CUDA tensors of shape
        (nvec, length), float64 (FP64) or float32 (FP32 and BF16)."""
        nvec = r.shape[0] if r.dim() == 2 else 1
        _check(lib().sigma(self.ctx.h, self.h, nvec, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                           precision, _stream_ptr(stream)))
        return out

    def davidson_solve(self, opts=None, stream=None):
        """(energies, residual norms, iterations, converged) of the Davidson solve."""
        import numpy as np
        opts = opts if opts is not None else self.opts
        n = opts.nroots_solve
        e, rn, it = np.zeros(n), np.zeros(n), ctypes.c_int()
        rc = _check(lib().davidson_solve(self.ctx.h, self.h, ctypes.byref(opts), _stream_ptr(stream), _dptr(e), _dptr(rn),
                                         ctypes.byref(it)), allow=(ERR_NOT_CONVERGED,))
        return e, rn, it.value, rc == OK

    def autotune_info(self):
        """Candidates [(group size, vectors per CTA, summed ms of the small-block launches)] and the index
        of the candidate fastest over all launches together (each launch keeps its own fastest)."""
        import numpy as np
        gs = (ctypes.c_int * 64)()
        rp = (ctypes.c_int * 64)()
        ms = np.zeros(64)
        ch = ctypes.c_int()
        _check(lib().pno_autotune_info(self.h, 64, gs, rp, _dptr(ms), ctypes.byref(ch)))
        n = sum(1 for k in range(64) if gs[k] > 0)
        return [(gs[k], rp[k], float(ms[k])) for k in range(n)], ch.value

    def set_timing(self, enable=True):
        _check(lib().pno_set_timing(self.h, 1 if enable else 0))

    def sigma_timing(self, nvec, precision=FP64):
        """Per kernel class: dict(name, launches, ms, bytes, flops) of the recorded sigma calls."""
        out = []
        for k in range(SIGMA_CLASSES):
            nm, n = ctypes.c_char_p(), ctypes.c_int()
            ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _check(lib().pno_sigma_timing(self.h, k, nvec, precision, ctypes.byref(nm), ctypes.byref(n), ctypes.byref(ms),
                                          ctypes.byref(by), ctypes.byref(fl)))
            out.append(dict(name=nm.value.decode(), launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value))
        return out

    def tc_mma_flops(self):
        """Executed MMA flops of the tensor-core sandwich kernel per vector (padding included)."""
        x = ctypes.c_double()
        _check(lib().pno_tc_mma_flops(self.h, ctypes.byref(x)))
        return x.value

    def solve_stats(self):
        """dict(fp32, fp64): sigma evaluations of the last davidson_solve, by precision."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pno_solve_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return dict(fp32=a.value, fp64=b.value)

    def lowprec_energies(self, phase=FP32):
        """Ritz values of the last solve when its BF16 (phase=BF16) or FP32 (phase=FP32)
        phase handed over to the next precision (or [])."""
        import numpy as np
        n = ctypes.c_int()
        _check(lib().pno_solve_lowprec_energies(self.h, phase, 0, None, ctypes.byref(n)))
        e = np.zeros(max(1, n.value))
        _check(lib().pno_solve_lowprec_energies(self.h, phase, n.value, _dptr(e), ctypes.byref(n)))
        return e[:n.value]

    def eigenvectors(self):
        import numpy as np
        X = np.zeros((self.opts.nroots_solve, self.length))
        _check(lib().pno_get_eigenvectors(self.h, _dptr(X)))
        return X


class Batch:
    """pnoeom_batch_*: several built systems evaluated in one launch sequence."""

    def __init__(self, ctx, pnos, stream=None):
        self.ctx, self.pnos = ctx, list(pnos)
        arr = (ctypes.c_void_p * len(self.pnos))(*[p.h.value for p in self.pnos])
        h = ctypes.c_void_p()
        _check(lib().pnoeom_batch_create(ctx.h, arr, len(self.pnos), _stream_ptr(stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pnoeom_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sigma(self, rs, outs, precision=FP64, stream=None):
        """rs, outs: per member a CUDA tensor (nvec_k, length_k) or None."""
        n = len(self.pnos)
        nv = (ctypes.c_int * n)(*[0 if r is None else (r.shape[0] if r.dim() == 2 else 1) for r in rs])
        rp = (ctypes.c_void_p * n)(*[0 if r is None else r.data_ptr() for r in rs])
        op = (ctypes.c_void_p * n)(*[0 if o is None else o.data_ptr() for o in outs])
        _check(lib().pnoeom_batch_sigma(self.ctx.h, self.h, nv, rp, op, precision, _stream_ptr(stream)))

    def solve(self, opts, stream=None):
        """(energies [n, nroots], residual norms, iterations [n], converged [n])."""
        import numpy as np
        n, nr = len(self.pnos), opts.nroots_solve
        e, rn = np.zeros((n, nr)), np.zeros((n, nr))
        it, cv = (ctypes.c_int * n)(), (ctypes.c_int * n)()
        _check(lib().pnoeom_batch_solve(self.ctx.h, self.h, ctypes.byref(opts), _stream_ptr(stream), _dptr(e), _dptr(rn),
                                        it, cv), allow=(ERR_NOT_CONVERGED,))
        return e, rn, list(it), [bool(x) for x in cv]


QUEUED, BUILDING, RUNNING, DONE, FAILED = 0, 1, 2, 3, 4


class Server:
    """pnoeom_server_*: continuous-batching request loop (native threads)."""

    def __init__(self, ctx, hbm_budget_bytes=0, max_active=16):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(lib().pnoeom_server_create(ctx.h, hbm_budget_bytes, max_active, ctypes.byref(h)))
        self.h = h
        self.nroots = {}

    def close(self):
        if getattr(self, "h", None):
            lib().pnoeom_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, eps, B, o, opts, t1=None, t2=None):
        import numpy as np
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        t1 = None if t1 is None else np.ascontiguousarray(t1, dtype=np.float64)
        t2 = None if t2 is None else np.ascontiguousarray(t2, dtype=np.float64)
        ptr = lambda x: None if x is None else x.ctypes.data
        sysd = System(o, len(eps) - o, B.shape[0], ptr(eps), ptr(B), ptr(t1), ptr(t2), HOST)
        rid = ctypes.c_int64()
        _check(lib().pnoeom_server_submit(self.h, ctypes.byref(sysd), ctypes.byref(opts), ctypes.byref(rid)))
        self.nroots[rid.value] = opts.nroots_solve
        return rid.value

    def poll(self, rid):
        """dict(status, energies, res_norms, iters, sigma_evals, times, error)."""
        import numpy as np
        n = self.nroots.get(rid, 16)
        st, it, se = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        e, rn, tm = np.full(n, np.nan), np.full(n, np.nan), np.zeros(4)
        rc = lib().pnoeom_server_poll(self.h, rid, ctypes.byref(st), _dptr(e), _dptr(rn), ctypes.byref(it),
                                      ctypes.byref(se), _dptr(tm))
        err = None if rc == OK else (rc, lib().pnoeom_last_error().decode())
        if rc != OK and st.value != FAILED:
            raise PnoeomError(rc, err[1])
        return dict(status=st.value, energies=e, res_norms=rn, iters=it.value, sigma_evals=se.value, times=tm, error=err)

    def wait(self, rid, timeout_s=600.0):
        return lib().pnoeom_server_wait(self.h, rid, timeout_s)

    def stats(self):
        ub, q, r = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        ro, me, se = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().pnoeom_server_stats(self.h, ctypes.byref(ub), ctypes.byref(q), ctypes.byref(r), ctypes.byref(ro),
                                         ctypes.byref(me), ctypes.byref(se)))
        return dict(used_bytes=ub.value, queued=q.value, running=r.value, rounds=ro.value, merges=me.value,
                    sigma_evals=se.value)
