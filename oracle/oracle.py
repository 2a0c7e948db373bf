"""ctypes binding of the CGKS-5 CPU oracle (test infrastructure only)."""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgks_oracle.c")
_SO = os.path.join(_HERE, "libcgks_oracle.so")


def build_oracle(force=False):
    """Compile the oracle with gcc (-O2, OpenMP, strict IEEE arithmetic)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "cgks_oracle.h"))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class _Desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("nodes", C.POINTER(C.c_double)),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("gamma", C.c_double),
                ("mu", C.c_double), ("prandtl", C.c_double), ("tau_mode", C.c_int),
                ("cfl", C.c_double), ("dt_fixed", C.c_double), ("linear", C.c_int),
                ("c_chi", C.c_double), ("bc", C.c_int * 6), ("bc_state", (C.c_double * 5) * 6)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(_SO)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Desc)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_nfields.argtypes = [C.c_void_p]
        L.orc_ncells.restype = C.c_long
        L.orc_ncells.argtypes = [C.c_void_p]
        L.orc_set_state.argtypes = [C.c_void_p, dp, C.c_double]
        L.orc_get_state.argtypes = [C.c_void_p, dp, dp]
        L.orc_num_init_points.restype = C.c_long
        L.orc_num_init_points.argtypes = [C.c_void_p]
        L.orc_init_points.argtypes = [C.c_void_p, dp]
        L.orc_init_from_prims.argtypes = [C.c_void_p, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_compute_dt.restype = C.c_double
        L.orc_compute_dt.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_step_dt.argtypes = [C.c_void_p, C.c_double]
        L.orc_get_chi.argtypes = [C.c_void_p, dp]
        L.orc_positivity_fallbacks.restype = C.c_long
        L.orc_positivity_fallbacks.argtypes = [C.c_void_p]
        L.orc_get_metrics.argtypes = [C.c_void_p, dp, dp]
        fp = C.POINTER(C.c_float)
        L.orc_set_selector.argtypes = [C.c_void_p, fp, C.c_float, C.c_float]
        L.orc_selector_stats.argtypes = [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_long), dp]
        L.orc_selector_features.argtypes = [C.c_void_p, fp]
        L.orc_selector_logits.argtypes = [fp, fp, C.c_long, fp]
        L.orc_basis_size.argtypes = [C.c_int]
        L.orc_data_size.argtypes = [C.c_int]
        L.orc_recon_matrix.argtypes = [C.c_int, dp, ip]
        L.orc_recon_reference.argtypes = [C.c_int, dp, C.c_int, C.c_double, dp, dp]
        L.orc_recon_coeffs.argtypes = [C.c_int, dp, dp]
        L.orc_gram.argtypes = [C.c_int, dp, dp]
        L.orc_linear_sub.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_gks_point.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                    C.c_double, dp, dp, dp, dp, dp]
        L.orc_moments_u.argtypes = [C.c_double, C.c_double, dp, dp, dp]
        L.orc_micro_slope.argtypes = [C.c_int, C.c_double, dp, dp, dp]
        L.orc_s2o4_stage1.restype = C.c_double
        L.orc_s2o4_stage1.argtypes = [C.c_double] * 4
        L.orc_s2o4_stage2.restype = C.c_double
        L.orc_s2o4_stage2.argtypes = [C.c_double] * 5
        _lib = L
    return _lib


def set_threads(n):
    """Threads of the oracle's OpenMP loops from now on (n <= 0: unchanged);
    returns the number in use.  Results do not depend on it."""
    return lib().orc_set_threads(int(n))


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle:
    """One oracle mesh + state.  Arguments mirror the library's mesh descriptor."""

    def __init__(self, dim, n, lo=(0, 0, 0), hi=(1, 1, 1), nodes=None, gamma=1.4, mu=0.0,
                 prandtl=1.0, tau_mode=0, cfl=0.5, dt_fixed=0.0, linear=False, c_chi=100.0, bc=None,
                 bc_state=None):
        L = lib()
        d = _Desc()
        d.dim = dim
        nn = list(n) + [1] * (3 - len(n))
        for i in range(3):
            d.n[i] = int(nn[i])
            d.lo[i] = float(lo[i]) if i < len(lo) else 0.0
            d.hi[i] = float(hi[i]) if i < len(hi) else 1.0
        self._nodes = None
        if nodes is not None:
            self._nodes = np.ascontiguousarray(nodes, dtype=np.float64)
            d.nodes = _p(self._nodes)
        d.gamma, d.mu, d.prandtl, d.tau_mode = gamma, mu, prandtl, tau_mode
        d.cfl, d.dt_fixed, d.linear, d.c_chi = cfl, dt_fixed, int(linear), c_chi
        for f in range(6):
            d.bc[f] = int(bc[f]) if bc is not None and f < len(bc) else 0
            if bc_state is not None and f < len(bc_state) and bc_state[f] is not None:
                for v, q in enumerate(bc_state[f]):
                    d.bc_state[f][v] = float(q)
        self._h = L.orc_create(C.byref(d))
        if not self._h:
            raise RuntimeError("orc_create failed")
        self.dim, self.n = dim, tuple(int(x) for x in nn[:dim])
        self.nv = dim + 2
        self.nf = L.orc_nfields(self._h)
        self.ncell = L.orc_ncells(self._h)
        self.gamma = gamma

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    @property
    def state_shape(self):
        return (self.nf, self.nv) + tuple(reversed(self.n))

    def init_points(self):
        L = lib()
        npts = L.orc_num_init_points(self._h)
        pts = np.empty((npts, self.dim))
        L.orc_init_points(self._h, _p(pts))
        return pts

    def init_from_prims(self, prims):
        prims = np.ascontiguousarray(prims, dtype=np.float64)
        lib().orc_init_from_prims(self._h, _p(prims))

    def init(self, field_fn):
        """field_fn(*coords) -> list of primitive arrays (rho, U, V[, W], p)."""
        pts = self.init_points()
        prims = np.stack(field_fn(*[pts[:, d] for d in range(self.dim)]), axis=-1)
        self.init_from_prims(prims)

    def set_state(self, s, t=0.0):
        s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1)
        lib().orc_set_state(self._h, _p(s), t)

    def get_state(self):
        s = np.empty(self.state_shape)
        t = C.c_double(0)
        lib().orc_get_state(self._h, _p(s), C.byref(t))
        return s

    def time(self):
        s = np.empty(self.state_shape)
        t = C.c_double(0)
        lib().orc_get_state(self._h, _p(s), C.byref(t))
        return t.value

    def dt(self):
        return lib().orc_compute_dt(self._h)

    def step(self, nsteps=1):
        dt = C.c_double(0)
        rc = lib().orc_step(self._h, nsteps, C.byref(dt))
        if rc:
            raise RuntimeError("orc_step failed: %d" % rc)
        return dt.value

    def step_dt(self, dt):
        rc = lib().orc_step_dt(self._h, dt)
        if rc:
            raise RuntimeError("orc_step_dt failed: %d" % rc)

    def advance_to(self, t_end):
        """CFL steps, the last one shortened to land on t_end; returns the step count."""
        n = 0
        while True:
            t = self.time()
            if t >= t_end * (1 - 1e-14):
                return n
            dt = min(self.dt(), t_end - t)
            self.step_dt(dt)
            n += 1

    def chi(self):
        out = np.empty((self.nv,) + tuple(reversed(self.n)))
        lib().orc_get_chi(self._h, _p(out))
        return out

    def positivity_fallbacks(self):
        return lib().orc_positivity_fallbacks(self._h)

    def set_selector(self, params=None, thr_skip=0.0, thr_lo=0.0):
        """Learned selector on (params: SEL_NPARAM floats) or off (None)."""
        fp = C.POINTER(C.c_float)
        if params is None:
            lib().orc_set_selector(self._h, None, 0.0, 0.0)
            return
        self._sel = np.ascontiguousarray(params, dtype=np.float32)
        assert self._sel.size == selector_nparam()
        lib().orc_set_selector(self._h, self._sel.ctypes.data_as(fp), float(thr_skip), float(thr_lo))

    def selector_stats(self):
        a, b, m = C.c_long(0), C.c_long(0), C.c_double(0)
        lib().orc_selector_stats(self._h, C.byref(a), C.byref(b), C.byref(m))
        return a.value, b.value, m.value

    def selector_features(self):
        out = np.empty((self.ncell, 16), dtype=np.float32)
        lib().orc_selector_features(self._h, out.ctypes.data_as(C.POINTER(C.c_float)))
        return out

    def metrics(self):
        vol = np.empty(self.ncell)
        clo = np.empty((self.ncell, self.dim))
        lib().orc_get_metrics(self._h, _p(vol), _p(clo))
        return vol, clo


# ---- unit-level helpers ----
def recon_matrix(dim):
    L = lib()
    nb, nd = L.orc_basis_size(dim), L.orc_data_size(dim)
    M = np.empty((nb, nd))
    ex = np.empty((nb, 3), dtype=np.int32)
    L.orc_recon_matrix(dim, _p(M), ex.ctypes.data_as(C.POINTER(C.c_int)))
    return M, ex


def recon_reference(dim, data, linear=False, c_chi=100.0, low_order=False):
    """values and reference gradients at the face Gauss points of one cell;
    linear: chi = 1 (fifth order), low_order: chi = 0 (the weighted linear
    sub-stencils alone), neither: chi from the GENO path function"""
    L = lib()
    data = np.ascontiguousarray(data, dtype=np.float64)
    ngp = 2 * dim * (4 if dim == 3 else 2)
    out = np.empty((ngp, 1 + dim))
    chi = C.c_double(0)
    mode = 2 if low_order else (1 if linear else 0)
    L.orc_recon_reference(dim, _p(data), mode, c_chi, _p(out), C.byref(chi))
    return out, chi.value


def recon_coeffs(dim, data):
    L = lib()
    data = np.ascontiguousarray(data, dtype=np.float64)
    a = np.empty(L.orc_basis_size(dim))
    L.orc_recon_coeffs(dim, _p(data), _p(a))
    return a


def gram(dim):
    L = lib()
    nb = L.orc_basis_size(dim)
    gh, gl = np.empty((nb, nb)), np.empty((nb, nb))
    L.orc_gram(dim, _p(gh), _p(gl))
    return gh, gl


def linear_sub(dim, m, data):
    b = np.empty(dim)
    data = np.ascontiguousarray(data, dtype=np.float64)
    lib().orc_linear_sub(dim, m, _p(data), _p(b))
    return b


def gks_point(dim, WL, dWL, WR, dWR, dt, gamma=1.4, mu=0.0, prandtl=1.0, tau_mode=0):
    nv = dim + 2
    arr = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (WL, dWL, WR, dWR)]
    out = np.empty(6 * nv)
    rc = lib().orc_gks_point(dim, gamma, mu, prandtl, tau_mode, dt, *[_p(a) for a in arr], _p(out))
    if rc:
        raise RuntimeError("gks_point failed %d" % rc)
    return out.reshape(6, nv)


def moments_u(U, lam):
    f, p, n = np.empty(7), np.empty(7), np.empty(7)
    lib().orc_moments_u(U, lam, _p(f), _p(p), _p(n))
    return f, p, n


def micro_slope(dim, prim, b, gamma=1.4):
    a = np.empty(dim + 2)
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    lib().orc_micro_slope(dim, gamma, _p(prim), _p(b), _p(a))
    return a


def s2o4(Q, dt, L, Lt, Lt_star=None):
    lb = lib()
    qs = lb.orc_s2o4_stage1(Q, dt, L, Lt)
    if Lt_star is None:
        return qs
    return qs, lb.orc_s2o4_stage2(Q, dt, L, Lt, Lt_star)


def selector_nparam():
    return lib().orc_selector_nparam()


def selector_logits(params, feat):
    """BF16-emulated logits of the selector network for features [n][16]."""
    fp = C.POINTER(C.c_float)
    params = np.ascontiguousarray(params, dtype=np.float32)
    feat = np.ascontiguousarray(feat, dtype=np.float32)
    out = np.empty(feat.shape[0], dtype=np.float32)
    lib().orc_selector_logits(params.ctypes.data_as(fp), feat.ctypes.data_as(fp), feat.shape[0],
                              out.ctypes.data_as(fp))
    return out
