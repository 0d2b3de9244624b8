"""Python binding of the C ABI in ``include/fgi.h`` (argument marshalling only).

Every step of the computation runs in ``libfgi.so`` on the GPU; this module
only converts arrays and tensors to pointers.  PyTorch provides device
memory and streams.  There is no CPU fallback: if the library is missing,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfgi.so")

FGI_FP64, FGI_SPLIT_BF16, FGI_BF16 = 0, 1, 2
FGI_STATIC_SCRATCH_BYTES = 64 << 20          # include/fgi.h
PRECISIONS = {"fp64": FGI_FP64, "split_bf16": FGI_SPLIT_BF16, "bf16": FGI_BF16}
ERRORS = {-1: "FGI_ERR_ARG", -2: "FGI_ERR_STATE", -3: "FGI_ERR_CUDA", -4: "FGI_ERR_WORKSPACE",
          -5: "FGI_ERR_TIMEOUT", -6: "FGI_ERR_NONFINITE", -7: "FGI_ERR_UNSUPPORTED",
          -8: "FGI_ERR_NOMEM"}

SYMBOLS = ["fgi_create", "fgi_destroy", "fgi_last_error", "fgi_add_radial", "fgi_add_species",
           "fgi_set_systems", "fgi_set_grid", "fgi_plan", "fgi_set_precision", "fgi_get_sizes",
           "fgi_get_system", "fgi_get_pattern", "fgi_workspace_size", "fgi_integrate_h",
           "fgi_density", "fgi_adjoint", "fgi_trace", "fgi_sync", "fgi_profile",
           "fgi_profile_read", "fgi_integrate_h_static", "fgi_get_batch_work", "fgi_selftest_wait_timeout",
           "fgi_get_schedule"]
KERNEL_KINDS = {"basis": 0, "h": 1, "density": 2, "adjoint": 3, "other": 4}


class FGIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libfgi.so and declare every entry point's argument and result types.
    ImportError when the library is not built: there is no fallback."""
    if not os.path.exists(path):
        raise ImportError("libfgi.so is not built (run __graft_entry__.build()); "
                          "there is no fallback path")
    lib = C.CDLL(path)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "fgi_create": ([C.POINTER(P), I], I),
        "fgi_destroy": ([P], I),
        "fgi_last_error": ([P], C.c_char_p),
        "fgi_add_radial": ([P, I, D, I, P, C.POINTER(I)], I),
        "fgi_add_species": ([P, D, I, P, C.POINTER(I)], I),
        "fgi_set_systems": ([P, I, P, P, P], I),
        "fgi_set_grid": ([P, I64, P, P, I64, P, P], I),
        "fgi_plan": ([P, I, C.c_char_p], I),
        "fgi_set_precision": ([P, I], I),
        "fgi_get_sizes": ([P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)], I),
        "fgi_get_system": ([P, I, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)], I),
        "fgi_get_pattern": ([P, I, C.POINTER(I64), C.POINTER(P), C.POINTER(P)], I),
        "fgi_workspace_size": ([P, C.POINTER(C.c_size_t)], I),
        "fgi_integrate_h": ([P, P, P, I, P, C.c_size_t, P], I),
        "fgi_density": ([P, P, P, P, P, C.c_size_t, P], I),
        "fgi_adjoint": ([P, P, P, P, P, P, C.c_size_t, P], I),
        "fgi_trace": ([P, P, P, P, P], I),
        "fgi_sync": ([P, P], I),
        "fgi_profile": ([P, I], I),
        "fgi_profile_read": ([P, I, C.POINTER(I64), C.POINTER(D), C.POINTER(D), C.POINTER(D)], I),
        "fgi_integrate_h_static": ([P, P, P, I, P], I),
        "fgi_get_batch_work": ([P, I64, P, P], I),
        "fgi_selftest_wait_timeout": ([P, P], I),
        "fgi_get_schedule": ([P, I, C.POINTER(I64), C.POINTER(I64), P, P, P, P, P], I),
        "fgi_set_atom_grids": ([P, P, P, P, P, P], I),
        "fgi_hartree_workspace_size": ([P, C.POINTER(C.c_size_t)], I),
        "fgi_hartree": ([P, P, P, I, P, C.c_size_t, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = None


def lib() -> C.CDLL:
    """The process-wide handle of libfgi.so (loaded on first use)."""
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dev_f64(t, n, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be contiguous with %d elements" % (name, n))
    return t


class Context:
    """One library context: inputs, plan, and the compute calls."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        self._h = C.c_void_p()
        self.device = device
        rc = self._lib.fgi_create(C.byref(self._h), device)
        if rc != 0:
            raise FGIError(rc, "fgi_create(device=%d)" % device)
        self._keep = []
        self._ws = None

    def close(self):
        """Free the context and its device storage (fgi_destroy); idempotent."""
        if self._h:
            self._lib.fgi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise FGIError(rc, self._lib.fgi_last_error(self._h).decode())

    # ---- inputs
    def add_radial(self, l: int, h: float, coef) -> int:
        """Add a radial function u(r) as a uniform cubic spline: coef [n_knots-1][4]
        on the knots r_k = k h (u = c0 + t (c1 + t (c2 + t c3))).  Returns its id."""
        coef = _np(coef, np.float64)
        out = C.c_int()
        self._check(self._lib.fgi_add_radial(self._h, int(l), float(h), coef.shape[0] + 1, _ptr(coef),
                                             C.byref(out)))
        return out.value

    def add_species(self, Z: float, radial_ids) -> int:
        """Add a species: nuclear charge Z and its shells (radial ids, 2l+1
        functions each, m = -l..l).  Returns its id."""
        ids = _np(radial_ids, np.int32)
        out = C.c_int()
        self._check(self._lib.fgi_add_species(self._h, float(Z), len(ids), _ptr(ids), C.byref(out)))
        return out.value

    def set_systems(self, atom_off, species, xyz):
        """Independent systems: atom_off [n_sys+1] splits species [n_atoms] and
        xyz [n_atoms][3] (Bohr).  Invalidates the plan."""
        atom_off = _np(atom_off, np.int64)
        species = _np(species, np.int32)
        xyz = _np(xyz, np.float64)
        self._check(self._lib.fgi_set_systems(self._h, len(atom_off) - 1, _ptr(atom_off), _ptr(species),
                                              _ptr(xyz)))
        self._n_sys = len(atom_off) - 1
        self._xyz = xyz.reshape(-1, 3).copy()

    def positions(self):
        """The atom positions [n_atoms][3] (Bohr) given to set_systems: the
        geometry the plan and every H integration are for."""
        return self._xyz.copy()

    def set_grid(self, xyz, w, batch_off, batch_sys):
        """Grid points xyz [n_pts][3] and weights w, grouped in batches of
        consecutive points (batch_off [n_batch+1], at most 1024 points each),
        batch_sys [n_batch] the system of each batch.  Invalidates the plan."""
        xyz = _np(xyz, np.float64)
        w = _np(w, np.float64)
        batch_off = _np(batch_off, np.int64)
        batch_sys = _np(batch_sys, np.int32)
        self._check(self._lib.fgi_set_grid(self._h, len(w), _ptr(xyz), _ptr(w), len(batch_off) - 1,
                                           _ptr(batch_off), _ptr(batch_sys)))
        self._n_batch = len(batch_off) - 1

    def set_atom_grids(self, owner, shell, atom_rgrid):
        """The grid's atom-centred structure for the Hartree potential: owner
        atom and radial shell of every point, and per atom rows (r_min, ln q,
        n_rad) of its radial grid r_k = r_min exp(k ln q)."""
        owner = _np(owner, np.int32)
        shell = _np(shell, np.int32)
        rg = np.asarray(atom_rgrid, dtype=np.float64).reshape(-1, 3)
        r_min = np.ascontiguousarray(rg[:, 0])
        ln_q = np.ascontiguousarray(rg[:, 1])
        n_rad = np.ascontiguousarray(rg[:, 2].astype(np.int32))
        self._check(self._lib.fgi_set_atom_grids(self._h, _ptr(owner), _ptr(shell), _ptr(r_min), _ptr(ln_q),
                                                 _ptr(n_rad)))
        self._hws = None

    def hartree_workspace_size(self) -> int:
        out = C.c_size_t()
        self._check(self._lib.fgi_hartree_workspace_size(self._h, C.byref(out)))
        return out.value

    def hartree(self, n, l_max=4, vh=None, ws=None, stream=None):
        """The Hartree potential of the density n on the grid (device FP64
        [n_pts] in, a new or given [n_pts] tensor out), multipoles up to l_max."""
        if getattr(self, "_pending_grids", None) is not None:
            self.set_atom_grids(*self._pending_grids)
            self._pending_grids = None
        n_pts = self.sizes()[2]
        _dev_f64(n, n_pts, "n")
        if vh is None:
            vh = torch.empty(n_pts, dtype=torch.float64, device=n.device)
        _dev_f64(vh, n_pts, "vh")
        if ws is None:
            if getattr(self, "_hws", None) is None:
                self._hws = torch.empty(max(256, self.hartree_workspace_size()), dtype=torch.uint8,
                                        device=n.device)
            ws = self._hws
        self._check(self._lib.fgi_hartree(self._h, _ptr(n), _ptr(vh), int(l_max), _ptr(ws), ws.numel(),
                                          _stream(stream)))
        return vh

    def plan(self, precision="fp64", tune_path=None):
        """Build the plan (active functions, pattern, tile lists, device copies)
        for precision 'fp64', 'split_bf16' or 'bf16'; tune_path: optional
        settings file (see tune.py)."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._check(self._lib.fgi_plan(self._h, p, tune_path.encode() if tune_path else None))
        self._ws = None

    def set_precision(self, precision):
        """Switch the precision of later compute calls without re-planning."""
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._check(self._lib.fgi_set_precision(self._h, p))

    def load(self, problem, precision="fp64", tune_path=None):
        """Marshal a problem object (radials, species, systems, grid) and plan."""
        rid = [self.add_radial(r.l, r.h, r.coef) for r in problem.radials]
        for sp in problem.species:
            self.add_species(sp.Z, [rid[k] for k in sp.radial_ids])
        self.set_systems(problem.atom_off, problem.atom_species, problem.atom_xyz)
        self.set_grid(problem.pts, problem.w, problem.batch_off, problem.batch_sys)
        # the grid's atom-centred structure goes to the library at the first
        # Hartree call (the integration does not need it)
        self._pending_grids = ((problem.owner, problem.shell, problem.atom_rgrid)
                               if getattr(problem, "owner", None) is not None else None)
        self.plan(precision, tune_path)
        return self

    # ---- queries
    def sizes(self):
        """(n_fn, nnz, n_pts, n_atoms) over all systems."""
        v = [C.c_int64() for _ in range(4)]
        self._check(self._lib.fgi_get_sizes(self._h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)       # n_fn, nnz, n_pts, n_atoms

    def system(self, s: int):
        """(fn0, n_fn, val0, nnz) of system s: its first function and count, and
        its first stored value and count in the H / D arrays."""
        v = [C.c_int64() for _ in range(4)]
        self._check(self._lib.fgi_get_system(self._h, s, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)       # fn0, n_fn, val0, nnz

    def batch_work(self):
        """Per batch: points P_b (int64) and active functions n_b (int32)."""
        nb = getattr(self, "_n_batch", 0)
        pts = np.zeros(nb, np.int64)
        nfn = np.zeros(nb, np.int32)
        self._check(self._lib.fgi_get_batch_work(self._h, nb, _ptr(pts), _ptr(nfn)))
        return pts, nfn

    def schedule(self, which: str = "h"):
        """The tensor-core schedule of the H integration ("h") or the density
        ("density"): dict of sb_first_batch [n_super+1], sb_points, sb_fns,
        wave_first_sb [n_waves+1] and sb_rank (position in the wave's tile
        lists, -1 without tiles)."""
        w = {"h": 0, "density": 1}[which]
        ns, nw = C.c_int64(), C.c_int64()
        self._check(self._lib.fgi_get_schedule(self._h, w, C.byref(ns), C.byref(nw),
                                               None, None, None, None, None))
        out = dict(sb_first_batch=np.zeros(ns.value + 1, np.int64), sb_points=np.zeros(ns.value, np.int32),
                   sb_fns=np.zeros(ns.value, np.int32), wave_first_sb=np.zeros(nw.value + 1, np.int64),
                   sb_rank=np.zeros(ns.value, np.int32))
        self._check(self._lib.fgi_get_schedule(self._h, w, C.byref(ns), C.byref(nw), _ptr(out["sb_first_batch"]),
                                               _ptr(out["sb_points"]), _ptr(out["sb_fns"]),
                                               _ptr(out["wave_first_sb"]), _ptr(out["sb_rank"])))
        return out

    def pattern(self, s: int = 0):
        """CSR pattern of system s's stored upper triangle: (rowptr [n_fn+1]
        relative to val0, col [nnz] function index within the system)."""
        nnz = C.c_int64()
        rp = C.c_void_p()
        col = C.c_void_p()
        self._check(self._lib.fgi_get_pattern(self._h, s, C.byref(nnz), C.byref(rp), C.byref(col)))
        n_fn = self.system(s)[1]
        rowptr = np.ctypeslib.as_array(C.cast(rp, C.POINTER(C.c_int64)), shape=(n_fn + 1,)).copy()
        cols = (np.ctypeslib.as_array(C.cast(col, C.POINTER(C.c_int32)), shape=(nnz.value,)).copy()
                if nnz.value else np.zeros(0, np.int32))
        return rowptr, cols

    def workspace_size(self) -> int:
        """Bytes of device scratch the compute calls need (every precision)."""
        b = C.c_size_t()
        self._check(self._lib.fgi_workspace_size(self._h, C.byref(b)))
        return b.value

    def workspace(self):
        """A cached uint8 device buffer of at least workspace_size() bytes."""
        need = self.workspace_size()
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda:%d" % self.device)
        return self._ws

    # ---- compute
    def integrate_h(self, v, h=None, accumulate=False, ws=None, stream=None):
        """H values on the pattern: h (+)= sum_p w_p v_p phi_i phi_j for every
        stored (i, j).  v: CUDA float64 [n_pts]; h: CUDA float64 [nnz]
        (allocated when None); returns h.  Enqueued on `stream`; sync()
        reports device-side errors."""
        n_fn, nnz, n_pts, _ = self.sizes()
        v = _dev_f64(v, n_pts, "v")
        if h is None:
            h = torch.empty(nnz, dtype=torch.float64, device=v.device)
        _dev_f64(h, nnz, "h")
        ws = self.workspace() if ws is None else ws
        self._check(self._lib.fgi_integrate_h(self._h, _ptr(v), _ptr(h), int(bool(accumulate)), _ptr(ws),
                                              ws.numel() * ws.element_size(), _stream(stream)))
        return h

    def density(self, d, n=None, traces=None, ws=None, stream=None, with_traces=True):
        """n_p = sum_ij phi_i(r_p) D_ij phi_j(r_p) from the stored values d of the
        symmetric D (CUDA float64 [nnz]); returns (n [n_pts], traces [n_sys] =
        sum_p w_p n_p per system, or None without traces)."""
        n_fn, nnz, n_pts, _ = self.sizes()
        d = _dev_f64(d, nnz, "d")
        if n is None:
            n = torch.empty(n_pts, dtype=torch.float64, device=d.device)
        _dev_f64(n, n_pts, "n")
        n_sys = self.n_systems()
        if traces is None and with_traces:
            traces = torch.empty(n_sys, dtype=torch.float64, device=d.device)
        ws = self.workspace() if ws is None else ws
        self._check(self._lib.fgi_density(self._h, _ptr(d), _ptr(n), _ptr(traces), _ptr(ws),
                                          ws.numel() * ws.element_size(), _stream(stream)))
        return n, traces

    def adjoint(self, g, v, dv=None, dR=None, ws=None, stream=None):
        """Gradients of L = sum_k g_k h_k(v, R) (g: CUDA float64 [nnz], the
        gradient with respect to the stored H values): returns dv [n_pts] and
        dR [n_atoms][3], grid and weights held fixed.  FP64 path."""
        n_fn, nnz, n_pts, n_at = self.sizes()
        g = _dev_f64(g, nnz, "g")
        v = _dev_f64(v, n_pts, "v")
        if dv is None:
            dv = torch.empty(n_pts, dtype=torch.float64, device=g.device)
        if dR is None:
            dR = torch.empty((n_at, 3), dtype=torch.float64, device=g.device)
        ws = self.workspace() if ws is None else ws
        self._check(self._lib.fgi_adjoint(self._h, _ptr(g), _ptr(v), _ptr(dv), _ptr(dR), _ptr(ws),
                                          ws.numel() * ws.element_size(), _stream(stream)))
        return dv, dR

    def trace(self, a, b, out=None, stream=None):
        """tr(A B) per system, in FP64, from the stored upper-triangle values of
        two symmetric matrices on the pattern (e.g. tr(DS), tr(DH))."""
        _, nnz, _, _ = self.sizes()
        _dev_f64(a, nnz, "a")
        _dev_f64(b, nnz, "b")
        if out is None:
            out = torch.empty(self.n_systems(), dtype=torch.float64, device=a.device)
        self._check(self._lib.fgi_trace(self._h, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))
        return out

    def sync(self, stream=None):
        """Wait for the stream and raise FGIError for a device-side error
        (FGI_ERR_TIMEOUT, FGI_ERR_NONFINITE) recorded since the last sync."""
        self._check(self._lib.fgi_sync(self._h, _stream(stream)))

    def selftest_wait_timeout(self, stream=None):
        """Enqueue a bounded device wait that runs out (about 2 s); the next
        sync() raises FGIError with code FGI_ERR_TIMEOUT."""
        self._check(self._lib.fgi_selftest_wait_timeout(self._h, _stream(stream)))

    def profile(self, enable: bool = True):
        """Start (clearing the record) or stop timing every kernel launch with
        CUDA events; not inside stream capture."""
        self._check(self._lib.fgi_profile(self._h, int(bool(enable))))

    def profile_read(self, kind):
        """Launches, milliseconds, algorithmic flops and bytes recorded for a kernel
        class: 'basis', 'h', 'density', 'adjoint' or 'other'."""
        k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        n = C.c_int64()
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        self._check(self._lib.fgi_profile_read(self._h, k, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
        return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}

    def n_systems(self) -> int:
        """Number of systems given to set_systems."""
        n = getattr(self, "_n_sys", None)
        if n is None:                                   # context filled through the C ABI directly
            n = 0
            while self._lib.fgi_get_system(self._h, n, None, None, None, None) == 0:
                n += 1
            self._n_sys = n
        return n


class HIntegrate(torch.autograd.Function):
    """h = H(v, R) as a differentiable function of the potential on the grid
    and of the atom positions (at the planned geometry).  The backward pass
    calls the adjoint kernels, which recompute the basis per batch."""

    @staticmethod
    def forward(fctx, context: Context, v, R):
        """h = H(v, R) on the context's plan.  R must equal the planned atom
        positions: the plan (active functions, pattern) belongs to one
        geometry, so a moved R raises ValueError instead of returning H at
        the old positions; plan a new context for a new geometry."""
        planned = torch.as_tensor(context.positions(), dtype=torch.float64)
        Rc = R.detach().to("cpu", torch.float64).reshape(planned.shape)
        if not torch.equal(Rc, planned):
            raise ValueError("HIntegrate: R differs from the planned atom positions by up to %.3e Bohr; "
                             "plan a context for the new geometry" % float((Rc - planned).abs().max()))
        fctx.context = context
        fctx.save_for_backward(v)
        return context.integrate_h(v.detach().contiguous())

    @staticmethod
    def backward(fctx, g):
        """(None, dL/dv, dL/dR) from the adjoint kernels."""
        (v,) = fctx.saved_tensors
        dv, dR = fctx.context.adjoint(g.contiguous(), v.detach().contiguous())
        return None, dv, dR


def integrate(context: Context, v, R):
    """Differentiable h = H(v, R) (see HIntegrate)."""
    return HIntegrate.apply(context, v, R)
