"""ctypes binding of libcgks.so with the C-ABI's names; marshalling only.

Every step of the scheme runs in the library's kernels.  Loading fails
loudly if the library is missing or was not built for this machine; there is
no CPU path.  PyTorch is used only for device buffers and the CUDA stream.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

STATUS_NAMES = {0: "CGKS_OK", -1: "CGKS_EINVAL", -2: "CGKS_ENOMEM", -3: "CGKS_ECUDA", -4: "CGKS_ENONPHYS",
                -5: "CGKS_ETIMEOUT", -6: "CGKS_ESTATE", -7: "CGKS_EUNSUPPORTED", -8: "CGKS_ETOOLARGE"}


class CgksError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__("%s (%d)%s" % (STATUS_NAMES.get(status, "?"), status, (": " + msg) if msg else ""))
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("nodes", C.POINTER(C.c_double)),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("bc", C.c_int * 6),
                ("bc_state", (C.c_double * 5) * 6),
                ("gamma", C.c_double), ("mu", C.c_double), ("prandtl", C.c_double),
                ("tau_mode", C.c_int), ("cfl", C.c_double), ("dt_fixed", C.c_double),
                ("linear", C.c_int), ("c_chi", C.c_double), ("precision", C.c_int),
                ("stream", C.c_void_p)]


# boundary kinds of MeshDesc.bc (CGKS_BC_* of include/cgks.h)
BC_PERIODIC, BC_OUTFLOW, BC_SLIP_WALL, BC_NOSLIP_WALL, BC_INFLOW = 0, 1, 2, 3, 4

SEL_NFEAT, SEL_NPARAM = 16, 2689


def _f32(t, n, what):
    """device pointer of a contiguous float32 CUDA tensor of n values on the
    current device (the library reads or writes exactly n)"""
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float32 CUDA tensor" % what)
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on another device than the current one" % what)
    check_size(t.numel(), n, what)
    return C.c_void_p(t.data_ptr())


def mlp_loss_grad(params, X, y, w, grad, stream=None):
    """Weighted BCE loss of the selector network and its gradient (into
    `grad`), all torch CUDA float32 tensors; returns the loss."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    N = int(X.shape[0])
    for t, n, what in ((params, SEL_NPARAM, "params"), (X, N * SEL_NFEAT, "X"), (y, N, "y"), (w, N, "w"),
                       (grad, SEL_NPARAM, "grad")):
        _f32(t, n, what)
    loss = C.c_float(0)
    status = lib().cgks_mlp_loss_grad(C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()),
                                      C.c_void_p(y.data_ptr()), C.c_void_p(w.data_ptr()), int(X.shape[0]),
                                      C.c_void_p(grad.data_ptr()), C.byref(loss), C.c_void_p(st.cuda_stream))
    if status:
        raise CgksError(status, "cgks_mlp_loss_grad")
    return loss.value


def mlp_logits(params, X, out=None, stream=None):
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    if out is None:
        out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    N = int(X.shape[0])
    for t, n, what in ((params, SEL_NPARAM, "params"), (X, N * SEL_NFEAT, "X"), (out, N, "out")):
        _f32(t, n, what)
    status = lib().cgks_mlp_logits(C.c_void_p(params.data_ptr()), C.c_void_p(X.data_ptr()), int(X.shape[0]),
                                   C.c_void_p(out.data_ptr()), C.c_void_p(st.cuda_stream))
    if status:
        raise CgksError(status, "cgks_mlp_logits")
    return out


def mlp_adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    for t, what in ((params, "params"), (grad, "grad"), (m, "m"), (v, "v")):
        _f32(t, SEL_NPARAM, what)
    status = lib().cgks_mlp_adam(C.c_void_p(params.data_ptr()), C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
                                 C.c_void_p(v.data_ptr()), int(step), float(lr), float(beta1), float(beta2),
                                 float(eps), C.c_void_p(st.cuda_stream))
    if status:
        raise CgksError(status, "cgks_mlp_adam")


class BatchTiles(C.Structure):
    _fields_ = [("tile_x", C.c_int), ("tile_y", C.c_int), ("recon_blocks", C.c_int), ("flux_blocks", C.c_int),
                ("update_blocks", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["cgks_create_mesh", "cgks_destroy", "cgks_num_vars", "cgks_num_fields", "cgks_num_cells",
           "cgks_flux_staging",
           "cgks_set_state", "cgks_get_state", "cgks_set_state_async", "cgks_get_state_async", "cgks_sync",
           "cgks_step", "cgks_compute_dt", "cgks_init_points_per_cell",
           "cgks_init_points", "cgks_init_from_prims", "cgks_get_chi", "cgks_profile_enable",
           "cgks_profile_read", "cgks_last_error", "cgks_compute_dt_noalloc", "cgks_batch_create",
           "cgks_batch_destroy", "cgks_batch_num_cases", "cgks_batch_num_cells", "cgks_batch_set_state",
           "cgks_batch_get_state", "cgks_batch_times", "cgks_batch_step", "cgks_batch_get_tiles",
           "cgks_batch_set_tiles", "cgks_batch_tune", "cgks_batch_last_error", "cgks_set_selector",
           "cgks_selector_stats", "cgks_selector_features", "cgks_batch_set_selector", "cgks_batch_selector_stats",
           "cgks_mlp_loss_grad", "cgks_mlp_logits", "cgks_mlp_adam", "cgks_diagnostics"]

_lib = None


def lib(build_if_missing=True):
    """Load libcgks.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libcgks.so is missing: build it with paper_2508_08965_gb300.build.build()")
    L = C.CDLL(path)
    vp, dp, lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_long)
    L.cgks_create_mesh.argtypes = [C.POINTER(MeshDesc), C.POINTER(vp)]
    L.cgks_destroy.argtypes = [vp]
    L.cgks_destroy.restype = None
    L.cgks_num_vars.argtypes = [vp]
    L.cgks_num_fields.argtypes = [vp]
    L.cgks_num_cells.argtypes = [vp]
    L.cgks_num_cells.restype = C.c_long
    L.cgks_flux_staging.argtypes = [vp]
    L.cgks_flux_staging.restype = C.c_int
    L.cgks_set_state.argtypes = [vp, vp, C.c_int, C.c_double]
    L.cgks_get_state.argtypes = [vp, vp, C.c_int, dp]
    L.cgks_set_state_async.argtypes = [vp, vp, C.c_int, C.c_double]
    L.cgks_get_state_async.argtypes = [vp, vp, C.c_int]
    L.cgks_sync.argtypes = [vp]
    L.cgks_step.argtypes = [vp, C.c_int, C.c_double, dp, dp]
    L.cgks_compute_dt.argtypes = [vp, dp]
    L.cgks_init_points_per_cell.argtypes = [vp]
    L.cgks_init_points.argtypes = [vp, C.c_long, C.c_long, vp]
    L.cgks_init_from_prims.argtypes = [vp, C.c_long, C.c_long, vp]
    L.cgks_get_chi.argtypes = [vp, vp, C.c_int]
    L.cgks_profile_enable.argtypes = [vp, C.c_int]
    L.cgks_profile_read.argtypes = [vp, C.POINTER(C.c_char_p), lp, dp, C.c_int]
    L.cgks_last_error.argtypes = [vp, C.c_char_p, C.c_size_t]
    L.cgks_compute_dt_noalloc.argtypes = [C.POINTER(MeshDesc), vp, dp]
    L.cgks_batch_create.argtypes = [C.POINTER(MeshDesc), C.c_int, vp, C.POINTER(vp)]
    L.cgks_batch_destroy.argtypes = [vp]
    L.cgks_batch_destroy.restype = None
    L.cgks_batch_num_cases.argtypes = [vp]
    L.cgks_batch_num_cells.argtypes = [vp]
    L.cgks_batch_num_cells.restype = C.c_long
    L.cgks_batch_set_state.argtypes = [vp, C.c_int, vp, C.c_int, C.c_double]
    L.cgks_batch_get_state.argtypes = [vp, C.c_int, vp, C.c_int, dp]
    L.cgks_batch_times.argtypes = [vp, dp, dp]
    L.cgks_batch_step.argtypes = [vp, C.c_int, C.c_int]
    L.cgks_batch_get_tiles.argtypes = [vp, C.POINTER(BatchTiles)]
    L.cgks_batch_set_tiles.argtypes = [vp, C.POINTER(BatchTiles)]
    L.cgks_batch_tune.argtypes = [vp, C.c_int, C.POINTER(BatchTiles), dp]
    L.cgks_batch_last_error.argtypes = [vp, C.c_char_p, C.c_size_t]
    fp = C.POINTER(C.c_float)
    ull = C.POINTER(C.c_ulonglong)
    L.cgks_diagnostics.argtypes = [vp, dp, dp]
    L.cgks_set_selector.argtypes = [vp, fp, C.c_float, C.c_float]
    L.cgks_selector_stats.argtypes = [vp, ull, ull]
    L.cgks_selector_features.argtypes = [vp, vp]
    L.cgks_batch_set_selector.argtypes = [vp, fp, C.c_float, C.c_float]
    L.cgks_batch_selector_stats.argtypes = [vp, ull, ull]
    L.cgks_mlp_loss_grad.argtypes = [vp, vp, vp, vp, C.c_long, vp, fp, vp]
    L.cgks_mlp_logits.argtypes = [vp, vp, C.c_long, vp, vp]
    L.cgks_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, vp]
    _lib = L
    return L


def _torch():
    import torch
    return torch


def make_desc(dim, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), nodes=None, gamma=1.4, mu=0.0, prandtl=1.0,
              tau_mode=0, cfl=0.5, dt_fixed=0.0, linear=False, c_chi=0.0, precision=0, bc=None, bc_state=None):
    """A cgks_mesh_desc (and the node array it points to, which the caller
    keeps alive until the library has copied it)."""
    d = MeshDesc()
    d.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for a in range(3):
        d.n[a] = int(nn[a])
        d.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        d.hi[a] = float(hi[a]) if a < len(hi) else 1.0
    keep = None
    if nodes is not None:
        keep = np.ascontiguousarray(nodes, dtype=np.float64)
        d.nodes = keep.ctypes.data_as(C.POINTER(C.c_double))
    d.gamma, d.mu, d.prandtl, d.tau_mode = gamma, mu, prandtl, tau_mode
    d.cfl, d.dt_fixed, d.linear, d.c_chi = cfl, dt_fixed, int(linear), c_chi
    for f in range(6):
        d.bc[f] = int(bc[f]) if bc is not None and f < len(bc) else BC_PERIODIC
        if bc_state is not None and f < len(bc_state) and bc_state[f] is not None:
            for v, q in enumerate(bc_state[f]):
                d.bc_state[f][v] = float(q)
    d.precision = int(precision)
    return d, keep


def check_size(n, want, what):
    if n != want:
        raise ValueError("%s holds %d values, the library reads or writes %d" % (what, n, want))


class Mesh:
    """One library context: a mesh, its device state and metrics.

    Arguments follow cgks_mesh_desc.  ``stream`` is a torch.cuda.Stream (or
    None for torch's current stream at construction time).  precision 0 is
    FP64 throughout; 1 runs reconstruction, interface flux and weights in
    FP32 with FP64 cell averages and metrics; 2 is FP64 with the interface
    flux solved in paired-FP32 arithmetic.  ``flux_staging`` says how the
    interface-flux kernel stages its inputs ("tma" or "cp.async";
    cgks_flux_staging).
    """

    def __init__(self, dim, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), nodes=None, gamma=1.4, mu=0.0,
                 prandtl=1.0, tau_mode=0, cfl=0.5, dt_fixed=0.0, linear=False, c_chi=0.0, stream=None,
                 precision=0, bc=None, bc_state=None):
        torch = _torch()
        L = lib()
        d, self._nodes = make_desc(dim, n, lo, hi, nodes, gamma, mu, prandtl, tau_mode, cfl, dt_fixed, linear, c_chi,
                                   precision, bc, bc_state)
        nn = list(n) + [1] * (3 - len(n))
        self.precision = int(precision)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d.stream = C.c_void_p(self.stream.cuda_stream)
        h = C.c_void_p()
        self._h = None
        self._pending = []  # host or device buffers of enqueued copies, kept alive until a sync
        self._check(L.cgks_create_mesh(C.byref(d), C.byref(h)))
        self._h = h
        self.dim = dim
        self.n = tuple(int(x) for x in nn[:dim])
        self.nv = L.cgks_num_vars(h)
        self.nf = L.cgks_num_fields(h)
        self.ncell = L.cgks_num_cells(h)
        self.flux_staging = "tma" if L.cgks_flux_staging(h) == 1 else "cp.async"
        self.lo, self.hi = tuple(lo[:dim]), tuple(hi[:dim])

    def _check(self, st):
        if st != 0:
            msg = ""
            if self._h:
                buf = C.create_string_buffer(512)
                lib().cgks_last_error(self._h, buf, 512)
                msg = buf.value.decode()
            raise CgksError(st, msg)

    def close(self):
        if self._h:
            if self._pending:
                lib().cgks_sync(self._h)
            lib().cgks_destroy(self._h)
            self._h = None
            self._pending = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def state_shape(self):
        return (self.nf, self.nv) + tuple(reversed(self.n))

    def set_state(self, s, t=0.0):
        """s: numpy array (host) or torch CUDA tensor of state_shape, float64."""
        torch = _torch()
        size = self.nf * self.nv * self.ncell
        if isinstance(s, torch.Tensor) and s.is_cuda:
            if s.dtype != torch.float64:
                raise ValueError("state must be float64")
            s = s.contiguous()
            check_size(s.numel(), size, "state")
            self._check(lib().cgks_set_state(self._h, C.c_void_p(s.data_ptr()), 1, float(t)))
            self._keep = s
        else:
            a = np.ascontiguousarray(s, dtype=np.float64)
            check_size(a.size, size, "state")
            self._check(lib().cgks_set_state(self._h, a.ctypes.data_as(C.c_void_p), 0, float(t)))

    def get_state(self, out=None):
        """Host numpy copy (or into `out`: a contiguous float64 torch CUDA
        tensor or writable numpy array of the state's size); returns (state, t)."""
        torch = _torch()
        t = C.c_double(0)
        size = self.nf * self.nv * self.ncell
        if out is None:
            out = np.empty(self.state_shape)
        p, dev, keep = self._buffer(out, True)
        check_size(keep.numel() if isinstance(keep, torch.Tensor) else keep.size, size, "output buffer")
        self._check(lib().cgks_get_state(self._h, C.c_void_p(p), dev, C.byref(t)))
        self._pending = []
        return out, t.value

    @staticmethod
    def _buffer(a, writable):
        """(pointer, is_device, keep-alive) of a torch tensor (CUDA on the
        current device, or CPU, best page-locked) or a numpy array, in the
        public layout, float64"""
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("state buffers are contiguous float64")
            if a.is_cuda and a.device.index != torch.cuda.current_device():
                raise ValueError("device buffer on another device than the current one")
            return a.data_ptr(), int(a.is_cuda), a
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise ValueError("state buffers are contiguous float64")
        if writable and not a.flags.writeable:
            raise ValueError("read-only output buffer")
        return a.ctypes.data, 0, a

    def set_state_async(self, s, t=0.0):
        """Enqueue the copy of state s in (no wait); s must stay valid and
        unchanged until sync() (or step(), get_state())."""
        p, dev, keep = self._buffer(s, False)
        n = keep.size if isinstance(keep, np.ndarray) else keep.numel()
        if n != self.nf * self.nv * self.ncell:
            raise ValueError("state of the wrong size")
        self._check(lib().cgks_set_state_async(self._h, C.c_void_p(p), dev, float(t)))
        self._pending.append(keep)

    def get_state_async(self, out):
        """Enqueue the copy of the state out into `out` (no wait); read it
        after sync()."""
        p, dev, keep = self._buffer(out, True)
        n = keep.size if isinstance(keep, np.ndarray) else keep.numel()
        if n != self.nf * self.nv * self.ncell:
            raise ValueError("output buffer of the wrong size")
        self._check(lib().cgks_get_state_async(self._h, C.c_void_p(p), dev))
        self._pending.append(keep)

    def sync(self):
        self._check(lib().cgks_sync(self._h))
        self._pending = []

    def step(self, nsteps=1, t_end=0.0):
        t, dt = C.c_double(0), C.c_double(0)
        self._check(lib().cgks_step(self._h, int(nsteps), float(t_end), C.byref(t), C.byref(dt)))
        self._pending = []
        return t.value, dt.value

    def advance_to(self, t_end, max_steps=10 ** 7):
        t, _ = self.step(max_steps, t_end)
        return t

    def compute_dt(self):
        dt = C.c_double(0)
        self._check(lib().cgks_compute_dt(self._h, C.byref(dt)))
        return dt.value

    def chi(self, out=None):
        """GENO weights of stage 1 of the last step, [v][cell] (host numpy, or
        into a torch CUDA float64 tensor `out`)."""
        if out is not None:
            torch = _torch()
            if not (isinstance(out, torch.Tensor) and out.is_cuda):
                raise ValueError("out must be a torch CUDA tensor")
            p, _, keep = self._buffer(out, True)
            check_size(keep.numel(), self.nv * self.ncell, "output buffer")
            self._check(lib().cgks_get_chi(self._h, C.c_void_p(p), 1))
            return out
        a = np.empty((self.nv,) + tuple(reversed(self.n)))
        self._check(lib().cgks_get_chi(self._h, a.ctypes.data_as(C.c_void_p), 0))
        return a

    def diagnostics(self):
        """(kinetic energy, enstrophy) volume averages of the current state."""
        ek, es = C.c_double(0), C.c_double(0)
        self._check(lib().cgks_diagnostics(self._h, C.byref(ek), C.byref(es)))
        return ek.value, es.value

    def set_selector(self, params=None, thr_skip=0.0, thr_lo=0.0):
        """Learned troubled-cell selector on (params: CGKS_SEL_NPARAM floats) or off (None)."""
        if params is None:
            self._check(lib().cgks_set_selector(self._h, None, 0.0, 0.0))
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == SEL_NPARAM
        self._check(lib().cgks_set_selector(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), float(thr_skip),
                                            float(thr_lo)))

    def selector_stats(self):
        a, b = C.c_ulonglong(0), C.c_ulonglong(0)
        self._check(lib().cgks_selector_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def selector_features(self, out=None):
        """Features of every cell of the current state: torch CUDA float32 [ncell][16]."""
        torch = _torch()
        if out is None:
            out = torch.empty((self.ncell, SEL_NFEAT), dtype=torch.float32, device="cuda")
        self._check(lib().cgks_selector_features(self._h, _f32(out, self.ncell * SEL_NFEAT, "out")))
        return out

    def init(self, field_fn, chunk_cells=1 << 18):
        """Initial data from a point function field_fn(*coords) -> [rho, U, V[, W], p]
        evaluated on the device (torch tensors), chunk by chunk."""
        torch = _torch()
        L = lib()
        npc = L.cgks_init_points_per_cell(self._h)
        with torch.cuda.stream(self.stream):
            for c0 in range(0, self.ncell, chunk_cells):
                nc = min(chunk_cells, self.ncell - c0)
                pts = torch.empty((nc * npc, self.dim), dtype=torch.float64, device="cuda")
                self._check(L.cgks_init_points(self._h, c0, nc, C.c_void_p(pts.data_ptr())))
                prims = torch.stack([torch.as_tensor(p, dtype=torch.float64, device="cuda").expand(nc * npc)
                                     for p in field_fn(*[pts[:, a] for a in range(self.dim)])], dim=-1).contiguous()
                self.stream.synchronize()
                self._check(L.cgks_init_from_prims(self._h, c0, nc, C.c_void_p(prims.data_ptr())))

    def profile(self, on=True):
        self._check(lib().cgks_profile_enable(self._h, int(on)))

    def profile_read(self):
        names = (C.c_char_p * 16)()
        launches = (C.c_long * 16)()
        ms = (C.c_double * 16)()
        n = lib().cgks_profile_read(self._h, names, launches, ms, 16)
        return {names[i].decode(): (launches[i], ms[i]) for i in range(n)}


def compute_dt_noalloc(state, dim, n, lo, hi, gamma=1.4, mu=0.0, cfl=0.5, dt_fixed=0.0, stream=None):
    """dt of a device state (contiguous torch CUDA float64 tensor, public
    layout, at least its averages) on a uniform box, without any device
    allocation by the library (for callers that cannot allocate: see
    cgks_compute_dt_noalloc in include/cgks.h).  The call runs on the state's
    device, on `stream` or that device's current stream.  Returns
    (status, dt); status 0 is CGKS_OK."""
    torch = _torch()
    if not (isinstance(state, torch.Tensor) and state.is_cuda and state.dtype == torch.float64
            and state.is_contiguous()):
        raise ValueError("state must be a contiguous float64 CUDA tensor")
    ncell = 1
    for a in range(dim):
        ncell *= int(n[a])
    if state.numel() < (dim + 2) * ncell:
        raise ValueError("state holds %d values; the averages of %d cells need %d"
                         % (state.numel(), ncell, (dim + 2) * ncell))
    with torch.cuda.device(state.device):
        return _compute_dt_noalloc(state, dim, n, lo, hi, gamma, mu, cfl, dt_fixed, stream)


def _compute_dt_noalloc(state, dim, n, lo, hi, gamma, mu, cfl, dt_fixed, stream):
    torch = _torch()
    d = MeshDesc()
    d.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for a in range(3):
        d.n[a] = int(nn[a])
        d.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        d.hi[a] = float(hi[a]) if a < len(hi) else 1.0
    d.gamma, d.mu, d.cfl, d.dt_fixed = gamma, mu, cfl, dt_fixed
    st = stream if stream is not None else torch.cuda.current_stream()
    d.stream = C.c_void_p(st.cuda_stream)
    dt = C.c_double(0.0)
    status = lib().cgks_compute_dt_noalloc(C.byref(d), C.c_void_p(state.data_ptr()), C.byref(dt))
    return status, dt.value


class Batch:
    """Many independent uniform-box meshes (cases) advanced together by the
    batched kernels: one launch per kernel and phase for all cases, and one
    CUDA graph launch per call of step().  ``cases`` is a list of dicts of
    Mesh's keyword arguments (dim, n, lo, hi, bc, gamma, mu, ...); all share
    dim and ``precision``.  ``stream``: a torch.cuda.Stream (a new one if
    None: graph capture needs a non-default stream)."""

    def __init__(self, cases, precision=0, stream=None):
        torch = _torch()
        L = lib()
        arr = (MeshDesc * len(cases))()
        for k, kw in enumerate(cases):
            kw = dict(kw)
            if kw.get("nodes") is not None:
                raise ValueError("batched cases are uniform boxes")
            d, _ = make_desc(precision=precision, **kw)
            arr[k] = d
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        self._h = None
        self._check(L.cgks_batch_create(arr, len(cases), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.ncase = len(cases)
        self.dims = [(kw["dim"], tuple(int(x) for x in kw["n"][:kw["dim"]])) for kw in cases]
        self.ncell = L.cgks_batch_num_cells(h)
        self.precision = int(precision)

    def _check(self, st):
        if st != 0:
            msg = ""
            if self._h:
                buf = C.create_string_buffer(512)
                lib().cgks_batch_last_error(self._h, buf, 512)
                msg = buf.value.decode()
            raise CgksError(st, msg)

    def close(self):
        if self._h:
            lib().cgks_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state_shape(self, k):
        dim, n = self.dims[k]
        nf = 1 + dim + dim * (4 if dim == 3 else 2)
        return (nf, dim + 2) + tuple(reversed(n))

    def set_state(self, k, s, t=0.0):
        """State of case k: numpy (host) or torch CUDA float64, that case's layout."""
        torch = _torch()
        if not 0 <= int(k) < self.ncase:
            raise IndexError("case %d of %d" % (k, self.ncase))
        size = int(np.prod(self.state_shape(k)))
        if isinstance(s, torch.Tensor) and s.is_cuda:
            if s.dtype != torch.float64:
                raise ValueError("state must be float64")
            if s.device.index != torch.cuda.current_device():
                raise ValueError("device buffer on another device than the current one")
            s = s.contiguous()
            check_size(s.numel(), size, "state")
            self._check(lib().cgks_batch_set_state(self._h, int(k), C.c_void_p(s.data_ptr()), 1, float(t)))
        else:
            a = np.ascontiguousarray(s, dtype=np.float64)
            check_size(a.size, size, "state")
            self._check(lib().cgks_batch_set_state(self._h, int(k), a.ctypes.data_as(C.c_void_p), 0, float(t)))

    def get_state(self, k):
        a = np.empty(self.state_shape(k))
        t = C.c_double(0)
        self._check(lib().cgks_batch_get_state(self._h, int(k), a.ctypes.data_as(C.c_void_p), 0, C.byref(t)))
        return a, t.value

    def times(self):
        t = np.empty(self.ncase)
        dt = np.empty(self.ncase)
        self._check(lib().cgks_batch_times(self._h, t.ctypes.data_as(C.POINTER(C.c_double)),
                                           dt.ctypes.data_as(C.POINTER(C.c_double))))
        return t, dt

    def step(self, nsteps=1, graph=True):
        self._check(lib().cgks_batch_step(self._h, int(nsteps), int(bool(graph))))

    def tiles(self):
        t = BatchTiles()
        self._check(lib().cgks_batch_get_tiles(self._h, C.byref(t)))
        return t.as_dict()

    def set_tiles(self, **kw):
        t = BatchTiles()
        self._check(lib().cgks_batch_get_tiles(self._h, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        self._check(lib().cgks_batch_set_tiles(self._h, C.byref(t)))

    def set_selector(self, params=None, thr_skip=0.0, thr_lo=0.0):
        if params is None:
            self._check(lib().cgks_batch_set_selector(self._h, None, 0.0, 0.0))
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(lib().cgks_batch_set_selector(self._h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                                  float(thr_skip), float(thr_lo)))

    def selector_stats(self):
        a, b = C.c_ulonglong(0), C.c_ulonglong(0)
        self._check(lib().cgks_batch_selector_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def tune(self, reps=3):
        """Run the library's autotuner; returns (chosen tiles, summed phase ms)."""
        t = BatchTiles()
        ms = C.c_double(0)
        self._check(lib().cgks_batch_tune(self._h, int(reps), C.byref(t), C.byref(ms)))
        return t.as_dict(), ms.value
