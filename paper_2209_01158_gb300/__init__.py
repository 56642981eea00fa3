"""GB300 (sm_103a) decoupled multicontinuum time stepping.

Python binding of libmc.so (include/mc.h): the functions below carry the C
names and only marshal arguments; every step of the method runs in the CUDA
kernels of the library. Host arrays may be numpy float64 arrays or CPU torch
float64 tensors (pinned tensors give asynchronous-capable copies); streams may
be given as a torch.cuda.Stream or a raw cudaStream_t integer.
"""

import ctypes as C

import numpy as np

from . import _native as N
from ._native import (MC_SCHEME_COUPLED, MC_SCHEME_D, MC_SCHEME_L, MC_SCHEME_U,
                      MC_PREC_FP64, MC_PREC_FP32_IR, MC_PREC_BF16T_IR, MC_MAX_CONTINUA)

SCHEMES = {"coupled": MC_SCHEME_COUPLED, "D": MC_SCHEME_D, "L": MC_SCHEME_L, "U": MC_SCHEME_U}


class MCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


def _lib():
    return N.load()


def _check(st, ctx=None):
    if st != N.MC_OK:
        lib = _lib()
        msg = lib.mc_last_error(ctx).decode() if ctx is not None else lib.mc_last_error(None).decode()
        raise MCError(st, msg or lib.mc_status_string(st).decode())


def _dptr(x, n=None, writable=False):
    """(double*, keepalive) for a host array: numpy float64 or CPU torch float64."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if x.is_cuda:
            raise ValueError("host buffer expected, got a CUDA tensor")
        if str(x.dtype) != "torch.float64" or not x.is_contiguous():
            raise ValueError("torch host buffers must be contiguous float64")
        if n is not None and x.numel() != n:
            raise ValueError("buffer has %d values, need %d" % (x.numel(), n))
        return C.cast(C.c_void_p(x.data_ptr()), N.dp), x
    a = np.asarray(x)
    if writable:
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("output arrays must be C-contiguous float64")
    else:
        a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("array has %d values, need %d" % (a.size, n))
    return a.ctypes.data_as(N.dp), a


def _dptr_list(xs, n, writable=False):
    ptrs, keep = [], []
    for x in xs:
        p, k = _dptr(x, n, writable)
        ptrs.append(p)
        keep.append(k)
    arr = (N.dp * len(ptrs))(*ptrs)
    return arr, keep


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def mc_default_opts():
    o = N.mc_opts()
    _check(_lib().mc_default_opts(C.byref(o)))
    return o


def mc_setup(nx, ny, k, c, sigma=None, sigma_cell=None, tau=1.0, opts=None, stream=None):
    """Returns an opaque context handle (c_void_p). sigma: L x L array or None;
    sigma_cell: dict {(a, b): array} (a < b) or a list in pair order or None."""
    L = len(k)
    n = int(nx) * int(ny)
    kk, keep_k = _dptr_list(k, n)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    if cc.size != L:
        raise ValueError("c needs L values")
    sg = None
    if sigma is not None:
        sg = np.ascontiguousarray(sigma, dtype=np.float64).reshape(L, L)
    sc_arr = None
    keep_sc = []
    if sigma_cell:
        pairs = [(a, b) for a in range(L) for b in range(a + 1, L)]
        if isinstance(sigma_cell, dict):
            seq = [sigma_cell.get(pq) for pq in pairs]
        else:
            seq = list(sigma_cell)
        ptrs = []
        for v in seq:
            if v is None:
                ptrs.append(N.dp())
            else:
                p, kp = _dptr(v, n)
                ptrs.append(p)
                keep_sc.append(kp)
        sc_arr = (N.dp * len(ptrs))(*ptrs)
    g = N.mc_grid(int(nx), int(ny))
    out = C.c_void_p()
    st = _lib().mc_setup(C.byref(g), L, kk, cc.ctypes.data_as(N.dp),
                         sg.ctypes.data_as(N.dp) if sg is not None else None,
                         sc_arr, float(tau), C.byref(opts) if opts is not None else None,
                         _stream_handle(stream), C.byref(out))
    _check(st)
    return out


def mc_set_opts(ctx, opts):
    _check(_lib().mc_set_opts(ctx, C.byref(opts)), ctx)


def mc_set_source(ctx, alpha, F, n=None):
    p, keep = _dptr(F, n)
    _check(_lib().mc_set_source(ctx, int(alpha), p), ctx)


def mc_set_well(ctx, alpha, W, pw, n=None):
    """Implicit well term of continuum alpha (W = q_w |cell| per cell, p_w per
    cell); W=None removes it."""
    if W is None:
        _check(_lib().mc_set_well(ctx, int(alpha), None, None), ctx)
        return
    pw = np.broadcast_to(np.asarray(pw, dtype=np.float64), np.shape(W))
    w, keep_w = _dptr(np.ascontiguousarray(np.ravel(W), dtype=np.float64), n)
    q, keep_q = _dptr(np.ascontiguousarray(np.ravel(pw), dtype=np.float64), n)
    _check(_lib().mc_set_well(ctx, int(alpha), w, q), ctx)


def mc_set_state(ctx, p, n=None):
    arr, keep = _dptr_list(p, n)
    _check(_lib().mc_set_state(ctx, arr), ctx)


def mc_get_state(ctx, out):
    """Fill the L preallocated host buffers `out` with the state."""
    arr, keep = _dptr_list(out, None, writable=True)
    _check(_lib().mc_get_state(ctx, arr), ctx)
    return out


def mc_state_device(ctx, alpha):
    ptr = C.c_void_p()
    _check(_lib().mc_state_device(ctx, int(alpha), C.byref(ptr)), ctx)
    return ptr.value


def _stats_dict(s, L):
    return {
        "steps_done": s.steps_done, "status": s.status,
        "iters": [int(s.iters[a]) for a in range(L)],
        "max_iters": [int(s.max_iters[a]) for a in range(L)],
        "ir_sweeps": int(s.ir_sweeps),
        "rel_residual": [float(s.rel_residual[a]) for a in range(L)],
        "mass_defect": float(s.mass_defect),
    }


def mc_step_decoupled(ctx, scheme, nsteps, L=MC_MAX_CONTINUA, check=True):
    s = N.mc_stats()
    st = _lib().mc_step_decoupled(ctx, int(scheme), int(nsteps), C.byref(s))
    d = _stats_dict(s, L)
    d["return"] = st
    if check:
        _check(st, ctx)
    return d


def mc_step_coupled(ctx, nsteps, L=MC_MAX_CONTINUA, check=True):
    s = N.mc_stats()
    st = _lib().mc_step_coupled(ctx, int(nsteps), C.byref(s))
    d = _stats_dict(s, L)
    d["return"] = st
    if check:
        _check(st, ctx)
    return d


def mc_get_coefficients(ctx, alpha, n):
    TE, TN, dg = np.empty(n), np.empty(n), np.empty(n)
    _check(_lib().mc_get_coefficients(ctx, int(alpha), TE.ctypes.data_as(N.dp),
                                      TN.ctypes.data_as(N.dp), dg.ctypes.data_as(N.dp)), ctx)
    return TE, TN, dg


def mc_apply(ctx, scheme, x, n):
    xs, kx = _dptr_list(x, n)
    ys = [np.empty(n) for _ in x]
    yy, ky = _dptr_list(ys, n, writable=True)
    _check(_lib().mc_apply(ctx, int(scheme), xs, yy), ctx)
    return ys


def mc_rhs_decoupled(ctx, L, n):
    bs = [np.empty(n) for _ in range(L)]
    bb, kb = _dptr_list(bs, n, writable=True)
    _check(_lib().mc_rhs_decoupled(ctx, bb), ctx)
    return bs


def mc_device_bytes(ctx):
    v = C.c_int64()
    _check(_lib().mc_device_bytes(ctx, C.byref(v)), ctx)
    return v.value


def _dev_ptr(x):
    if hasattr(x, "data_ptr"):
        if not x.is_cuda or str(x.dtype) != "torch.float64" or not x.is_contiguous():
            raise ValueError("device buffers must be contiguous CUDA float64 tensors")
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(int(x))


def mc_step_single_noalloc(nx, ny, k, c, tau, F, p, nsteps, rtol=1e-12, max_iter=100000,
                           stream=None, check=True):
    """Single-continuum steps with no device allocation (see include/mc.h).
    k, F, p: CUDA float64 tensors (or raw device pointers) of nx*ny values;
    p is updated in place."""
    s = N.mc_stats()
    st = _lib().mc_step_single_noalloc(int(nx), int(ny), _dev_ptr(k), float(c), float(tau),
                                       _dev_ptr(F), _dev_ptr(p), int(nsteps), float(rtol),
                                       int(max_iter), _stream_handle(stream), C.byref(s))
    d = _stats_dict(s, 1)
    d["return"] = st
    if check and st != N.MC_OK:
        raise MCError(st, _lib().mc_status_string(st).decode())
    return d


def mc_fp64_fma_rate(stream=None):
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    v = C.c_double()
    st = _lib().mc_fp64_fma_rate(_stream_handle(stream), C.byref(v))
    if st != N.MC_OK:
        raise MCError(st, _lib().mc_status_string(st).decode())
    return v.value


def mc_destroy(ctx):
    if ctx:
        _lib().mc_destroy(ctx)


class NLMC:
    """Owning wrapper of an mc_nlmc built on a Context (which must stay open).

    support: None, or a list of L entries, each None or a boolean nx*ny mask
    of the cells where that continuum lives (mc_nlmc_build_ex);
    conservative: set MC_NLMC_CONSERVATIVE."""

    def __init__(self, ctx, ncx, ncy, layers, basis_rtol=1e-12, basis_max_iter=50000,
                 support=None, conservative=False):
        self.ctx = ctx
        self.ncx, self.ncy, self.L = int(ncx), int(ncy), ctx.L
        self.n = self.L * self.ncx * self.ncy
        h = C.c_void_p()
        sup_arr, keep = None, []
        if support is not None:
            ptrs = []
            for s in support:
                if s is None:
                    ptrs.append(None)
                    continue
                a = np.ascontiguousarray(np.ravel(s), dtype=np.uint8)
                if a.size != ctx.n:
                    raise ValueError("support mask needs nx*ny values")
                keep.append(a)
                ptrs.append(a.ctypes.data_as(C.c_void_p))
            sup_arr = (C.c_void_p * len(ptrs))(*ptrs)
        flags = N.MC_NLMC_CONSERVATIVE if conservative else 0
        st = _lib().mc_nlmc_build_ex(ctx.handle, int(ncx), int(ncy), int(layers), float(basis_rtol),
                                     int(basis_max_iter), sup_arr, int(flags), C.byref(h))
        _check(st, ctx.handle)
        self._h = h

    def active(self):
        out = np.empty(self.n, dtype=np.uint8)
        _check(_lib().mc_nlmc_active(self._h, out.ctypes.data_as(C.POINTER(C.c_uint8))))
        return out.astype(bool)

    def step(self, scheme="D", nsteps=1):
        sc = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        s = N.mc_stats()
        st = _lib().mc_nlmc_step(self._h, int(sc), int(nsteps), C.byref(s))
        _check(st, self.ctx.handle)
        return {"steps_done": s.steps_done}

    def get_state(self):
        out = np.empty(self.n)
        _check(_lib().mc_nlmc_get_state(self._h, out.ctypes.data_as(N.dp)))
        return out

    def set_state(self, pbar):
        a = np.ascontiguousarray(pbar, dtype=np.float64)
        _check(_lib().mc_nlmc_set_state(self._h, a.ctypes.data_as(N.dp)))

    def operator(self):
        A = np.empty((self.n, self.n))
        m = np.empty(self.n)
        f = np.empty(self.n)
        _check(_lib().mc_nlmc_get_operator(self._h, A.ctypes.data_as(N.dp), m.ctypes.data_as(N.dp),
                                           f.ctypes.data_as(N.dp)))
        return A, m, f

    def basis(self, block, beta):
        out = np.empty(self.L * self.ctx.n)
        _check(_lib().mc_nlmc_get_basis(self._h, int(block), int(beta), out.ctypes.data_as(N.dp)))
        return out

    def info(self):
        v = (C.c_int64 * 5)()
        _check(_lib().mc_nlmc_info(self._h, v))
        return {"Nc": v[0], "L": v[1], "basis_iters": v[2], "basis_iters_max": v[3],
                "device_bytes": v[4]}

    def close(self):
        if getattr(self, "_h", None):
            _lib().mc_nlmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owning wrapper around an mc_ctx for one workload on one stream."""

    def __init__(self, nx, ny, k, c, sigma=None, sigma_cell=None, tau=1.0, opts=None,
                 stream=None):
        self.nx, self.ny, self.L = int(nx), int(ny), len(k)
        self.n = self.nx * self.ny
        self._ctx = mc_setup(nx, ny, k, c, sigma, sigma_cell, tau, opts, stream)

    @classmethod
    def from_workload(cls, w, opts=None, stream=None):
        ctx = cls(w.nx, w.ny, [np.ravel(x) for x in w.k], w.c, w.sigma,
                  {kk: np.ravel(v) for kk, v in w.sigma_cell.items()} or None,
                  w.tau, opts, stream)
        for a in range(w.L):
            ctx.set_source(a, w.F[a])
        for a, (W, pw) in (getattr(w, "wells", None) or {}).items():
            ctx.set_well(a, W, pw)
        ctx.set_state(w.p0)
        return ctx

    @property
    def handle(self):
        return self._ctx

    def set_opts(self, opts):
        mc_set_opts(self._ctx, opts)

    def set_source(self, alpha, F):
        mc_set_source(self._ctx, alpha, np.ravel(F) if not hasattr(F, "data_ptr") else F, self.n)

    def set_well(self, alpha, W, pw):
        mc_set_well(self._ctx, alpha, W, pw, self.n)

    def set_state(self, p):
        mc_set_state(self._ctx, [np.ravel(x) if not hasattr(x, "data_ptr") else x for x in p],
                     self.n)

    def get_state(self, out=None):
        if out is None:
            out = [np.empty(self.n) for _ in range(self.L)]
        return mc_get_state(self._ctx, out)

    def step_decoupled(self, scheme="D", nsteps=1, check=True):
        sc = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        return mc_step_decoupled(self._ctx, sc, nsteps, self.L, check)

    def step_coupled(self, nsteps=1, check=True):
        return mc_step_coupled(self._ctx, nsteps, self.L, check)

    def step(self, scheme, nsteps=1, check=True):
        if scheme == "coupled" or scheme == MC_SCHEME_COUPLED:
            return self.step_coupled(nsteps, check)
        return self.step_decoupled(scheme, nsteps, check)

    def coefficients(self, alpha):
        return mc_get_coefficients(self._ctx, alpha, self.n)

    def apply(self, scheme, x):
        sc = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        return mc_apply(self._ctx, sc, [np.ravel(v) for v in x], self.n)

    def rhs_decoupled(self):
        return mc_rhs_decoupled(self._ctx, self.L, self.n)

    def state_device(self, alpha):
        return mc_state_device(self._ctx, alpha)

    def device_bytes(self):
        return mc_device_bytes(self._ctx)

    def close(self):
        if getattr(self, "_ctx", None):
            mc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper of an mc_batch over a list of Context objects (which must
    stay open while the batch lives)."""

    def __init__(self, contexts, opts, team=None):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.handle.value for c in self.contexts])
        h = C.c_void_p()
        st = _lib().mc_batch_create(arr, len(self.contexts), C.byref(opts), C.byref(h))
        if st != N.MC_OK:
            raise MCError(st, _lib().mc_batch_last_error(None).decode())
        self._h = h
        if team is not None:
            self.set_team(team)

    def _check(self, st):
        if st != N.MC_OK:
            raise MCError(st, _lib().mc_batch_last_error(self._h).decode())

    def set_team(self, team):
        self._check(_lib().mc_batch_set_team(self._h, int(team)))

    def step(self, scheme="D", nsteps=1, check=True):
        sc = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        s = N.mc_stats()
        st = _lib().mc_batch_step(self._h, int(sc), int(nsteps), C.byref(s))
        d = _stats_dict(s, MC_MAX_CONTINUA)
        d["return"] = st
        if check:
            self._check(st)
        return d

    def instance_stats(self, i):
        s = N.mc_stats()
        self._check(_lib().mc_batch_instance_stats(self._h, int(i), C.byref(s)))
        return _stats_dict(s, self.contexts[i].L)

    def autotune(self, scheme="D", candidates=None, cache_path=None):
        sc = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        cand = None
        n = 0
        ms = None
        if candidates is not None:
            n = len(candidates)
            cand = (C.c_int32 * n)(*[int(x) for x in candidates])
            ms = np.full(n, -1.0)
        best = C.c_int32()
        self._check(_lib().mc_batch_autotune(
            self._h, int(sc), cand, n, cache_path.encode() if cache_path else None,
            C.byref(best), ms.ctypes.data_as(N.dp) if ms is not None else None))
        return best.value, (list(ms) if ms is not None else None)

    def info(self):
        v = (C.c_int64 * 9)()
        self._check(_lib().mc_batch_info(self._h, v))
        return {"n": v[0], "team": v[1], "teams": v[2], "ctas": v[3], "graph": v[4],
                "from_cache": v[5], "continuum_cells": v[6], "device_bytes": v[7],
                "fp64_instances": v[8]}

    def close(self):
        if getattr(self, "_h", None):
            _lib().mc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Fracture:
    """Owning wrapper of an mc_frac: a fracture continuum on its own 1-D mesh
    attached to a Context (which must stay open) holding the matrix continua.

    segments: (S, 4) array of (x0, y0, x1, y1); kf, cf: fracture
    permeability and capacity; sigma_f: exchange coefficient with each matrix
    continuum."""

    def __init__(self, ctx, segments, kf, cf, sigma_f):
        self.ctx = ctx
        self.L = ctx.L
        seg = np.ascontiguousarray(np.asarray(segments, dtype=np.float64).reshape(-1, 4))
        sf = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma_f, dtype=np.float64), (ctx.L,)))
        h = C.c_void_p()
        st = _lib().mc_frac_create(ctx.handle, int(seg.shape[0]), seg.ctypes.data_as(N.dp), float(kf),
                                   float(cf), sf.ctypes.data_as(N.dp), C.byref(h))
        _check(st, ctx.handle)
        self._h = h
        self.P = self.info()["pieces"]

    @classmethod
    def from_workload(cls, ctx, w):
        """Attach w.frac to ctx: point sources go to the piece whose midpoint
        is nearest to the point, wells q_w |piece| to the pieces whose
        midpoints lie in a well box; the initial fracture state is w.frac.p0."""
        fr = w.frac
        f = cls(ctx, fr.segments, fr.kf, fr.cf, fr.sigma_f)
        ln, mid, _ = f.pieces()
        if fr.sources:
            F = np.zeros(f.P)
            for (x, y, v) in fr.sources:
                F[int(np.argmin((mid[:, 0] - x) ** 2 + (mid[:, 1] - y) ** 2))] += v
            f.set_source(F)
        if fr.well_boxes:
            W = np.zeros(f.P)
            for (x0, x1, y0, y1) in fr.well_boxes:
                inb = ((mid[:, 0] >= x0) & (mid[:, 0] <= x1) & (mid[:, 1] >= y0) & (mid[:, 1] <= y1))
                W[inb] = fr.qw * ln[inb]
            f.set_well(W, np.full(f.P, fr.pw))
        f.set_state(None, np.full(f.P, fr.p0))
        return f

    def info(self):
        v = (C.c_int64 * 5)()
        _check(_lib().mc_frac_info(self._h, v), self.ctx.handle)
        return {"pieces": v[0], "junctions": v[1], "entries": v[2], "host_cells": v[3],
                "device_bytes": v[4]}

    def pieces(self):
        ln = np.empty(self.P)
        mid = np.empty(2 * self.P)
        host = np.empty(self.P, dtype=np.int32)
        _check(_lib().mc_frac_pieces(self._h, ln.ctypes.data_as(N.dp), mid.ctypes.data_as(N.dp),
                                     host.ctypes.data_as(C.POINTER(C.c_int32))), self.ctx.handle)
        return ln, mid.reshape(-1, 2), host

    def set_source(self, Ff):
        p, keep = _dptr(Ff, self.P)
        _check(_lib().mc_frac_set_source(self._h, p), self.ctx.handle)

    def set_well(self, Wf, pwf):
        if Wf is None:
            _check(_lib().mc_frac_set_well(self._h, None, None), self.ctx.handle)
            return
        w, kw = _dptr(Wf, self.P)
        q, kq = _dptr(pwf, self.P)
        _check(_lib().mc_frac_set_well(self._h, w, q), self.ctx.handle)

    def set_state(self, pm=None, pf=None):
        arr, keep = (None, None)
        if pm is not None:
            arr, keep = _dptr_list([np.ravel(x) if not hasattr(x, "data_ptr") else x for x in pm],
                                   self.ctx.n)
        pp, kp = (None, None)
        if pf is not None:
            pp, kp = _dptr(pf, self.P)
        _check(_lib().mc_frac_set_state(self._h, arr, pp), self.ctx.handle)

    def get_state(self):
        pm = [np.empty(self.ctx.n) for _ in range(self.L)]
        pf = np.empty(self.P)
        arr, keep = _dptr_list(pm, self.ctx.n, writable=True)
        _check(_lib().mc_frac_get_state(self._h, arr, pf.ctypes.data_as(N.dp)), self.ctx.handle)
        return pm, pf

    def step(self, scheme="D", nsteps=1, check=True):
        sc = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        s = N.mc_stats()
        st = _lib().mc_frac_step(self._h, int(sc), int(nsteps), C.byref(s))
        d = _stats_dict(s, MC_MAX_CONTINUA)
        d["return"] = st
        if check:
            _check(st, self.ctx.handle)
        return d

    def close(self):
        if getattr(self, "_h", None):
            _lib().mc_frac_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
