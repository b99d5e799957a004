"""Python binding of libhsweep (include/hsweep.h): the sweeping preconditioner for the
2D Helmholtz equation with H-matrix Schur complements, on one GB300 GPU.

The functions below carry the C-ABI names and only marshal arguments (torch CUDA
tensors -> device pointers, the current torch stream -> cudaStream_t).  Every step of
the method runs in the CUDA kernels of libhsweep.so; there is no CPU fallback: if the
library is missing the import of this module fails.

Vectors are torch.complex128 CUDA tensors of shape (nrhs, n*n) (or (n*n,) for one),
node (i, j) at (j-1)*n + (i-1), row by row with x1 fastest (Section 2.1).
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsweep.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NUMERIC, ERR_NOT_CONVERGED, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED = 0, 1
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NUMERIC",
                -5: "ERR_NOT_CONVERGED", -6: "ERR_TIMEOUT"}

EXPORTED = ["hsweep_default_opts", "hsweep_setup", "hsweep_create", "hsweep_apply", "hsweep_matvec",
            "hsweep_boundary_rhs",
            "hsweep_solve", "hsweep_grad", "hsweep_status", "hsweep_info", "hsweep_layer_ranks",
            "hsweep_export_layer", "hsweep_import_layer", "hsweep_free", "hsweep_profile",
            "hsweep_stats", "hsweep_apply_noalloc", "hsweep_sweep_plan", "hsweep_philox4x32_10",
            "hsweep_rsvd_normals", "hsweep_strong_plan", "hsweep_setup_tuning", "hsweep_strong_export",
            "hsweep_set_stream"]
NOALLOC_SCRATCH_BYTES = 32 << 20


class hsweep_opts(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("r_max", ctypes.c_int), ("precision", ctypes.c_int),
                ("pml_C", ctypes.c_double), ("pml_form", ctypes.c_int), ("gmres_max_it", ctypes.c_int),
                ("refine_max", ctypes.c_int), ("team", ctypes.c_int), ("groups", ctypes.c_int),
                ("sweep_kernel", ctypes.c_int), ("sweep_tc", ctypes.c_int),
                ("sweep_dir", ctypes.c_int), ("pml_sides", ctypes.c_int),
                ("strong_rank", ctypes.c_int), ("rsvd_seed", ctypes.c_uint),
                ("team_threads", ctypes.c_int), ("core_kernel", ctypes.c_int), ("krylov_lowp", ctypes.c_int)]


class HSweepError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, STATUS_NAMES.get(code, "?"), code))
        self.code = code


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libhsweep.so not built: run paper_1007_4290_gb300/build.py "
                          "(or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "hsweep_default_opts": (I, [ctypes.POINTER(hsweep_opts)]),
        "hsweep_setup": (I, [P, D, I, I, D, ctypes.POINTER(hsweep_opts), P, ctypes.POINTER(P)]),
        "hsweep_create": (I, [P, D, I, I, D, ctypes.POINTER(hsweep_opts), P, ctypes.POINTER(P)]),
        "hsweep_apply": (I, [P, P, P, I]),
        "hsweep_matvec": (I, [P, P, P, I]),
        "hsweep_boundary_rhs": (I, [P, I, P, P, I]),
        "hsweep_solve": (I, [P, P, P, I, D, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "hsweep_grad": (I, [P, P, I, P, I, P, P, ctypes.POINTER(D), D]),
        "hsweep_status": (I, [P, ctypes.POINTER(I)]),
        "hsweep_info": (I, [P, ctypes.POINTER(LL)]),
        "hsweep_layer_ranks": (I, [P, I, ctypes.POINTER(I)]),
        "hsweep_export_layer": (I, [P, I, P, P, ctypes.POINTER(I)]),
        "hsweep_import_layer": (I, [P, I, P, P, ctypes.POINTER(I)]),
        "hsweep_free": (None, [P]),
        "hsweep_profile": (I, [P, I]),
        "hsweep_set_stream": (I, [P, P]),
        "hsweep_stats": (I, [P, I, ctypes.POINTER(LL), ctypes.POINTER(LL), ctypes.POINTER(D)]),
        "hsweep_apply_noalloc": (I, [P, P, P, I]),
        "hsweep_sweep_plan": (I, [P, I, ctypes.POINTER(LL)]),
        "hsweep_setup_tuning": (I, [P, ctypes.POINTER(D)]),
        "hsweep_philox4x32_10": (I, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.POINTER(ctypes.c_uint32)]),
        "hsweep_rsvd_normals": (I, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, I, I, P]),
        "hsweep_strong_plan": (I, [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I), P, P, P]),
        "hsweep_strong_export": (I, [P, I, P, ctypes.POINTER(LL), ctypes.POINTER(I), ctypes.POINTER(LL)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _check(code, where):
    if code != OK:
        raise HSweepError(code, where)


def _ptr(t, dtype):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor of dtype %s" % dtype)
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_opts(**kw):
    o = hsweep_opts()
    _check(_lib.hsweep_default_opts(ctypes.byref(o)), "hsweep_default_opts")
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def philox4x32_10(ctr, key):
    """The library's Philox4x32-10 block (hsweep_philox4x32_10) of four 32-bit counter words
    under two key words, as a list of four ints; host only."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    out = (ctypes.c_uint32 * 4)()
    _check(_lib.hsweep_philox4x32_10(c, k, out), "hsweep_philox4x32_10")
    return list(out)


def rsvd_normals(blk, m, seed, rows, P):
    """hsweep_rsvd_normals: the (rows, P) complex Gaussian test vectors of block `blk` of
    layer m (host only)."""
    import numpy as np
    out = np.zeros(2 * rows * P, np.float64)
    _check(_lib.hsweep_rsvd_normals(blk, m, seed, rows, P, out.ctypes.data_as(ctypes.c_void_p)),
           "hsweep_rsvd_normals")
    return out.view(np.complex128).reshape(P, rows).T


def strong_plan(n, leaf, R):
    """hsweep_strong_plan: (far (nfar, 8), near (nnear, 6), ranks) int arrays (host only)."""
    import numpy as np
    nf, nn = ctypes.c_int(), ctypes.c_int()
    _check(_lib.hsweep_strong_plan(n, leaf, R, ctypes.byref(nf), ctypes.byref(nn), None, None, None),
           "hsweep_strong_plan")
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    far = np.zeros((max(1, nf.value), 8), np.int32)
    near = np.zeros((max(1, nn.value), 6), np.int32)
    ranks = np.zeros(1 << (L + 1), np.int32)
    _check(_lib.hsweep_strong_plan(n, leaf, R, ctypes.byref(nf), ctypes.byref(nn),
                                   far.ctypes.data_as(ctypes.c_void_p), near.ctypes.data_as(ctypes.c_void_p),
                                   ranks.ctypes.data_as(ctypes.c_void_p)), "hsweep_strong_plan")
    return far[:nf.value], near[:nn.value], ranks


class Handle:
    """An hsweep handle; owns the factorisation.  Free with .free() (or on GC)."""

    def __init__(self, raw, n):
        self._h = raw
        self.n = n
        self.N = n * n

    @property
    def raw(self):
        if self._h is None:
            raise RuntimeError("handle already freed")
        return self._h

    def free(self):
        if self._h is not None:
            _lib.hsweep_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        out = (ctypes.c_longlong * 8)()
        _check(_lib.hsweep_info(self.raw, out), "hsweep_info")
        keys = ["n", "L", "leaf", "r_max", "precision", "nleaves", "entries", "bytes_per_entry"]
        return dict(zip(keys, list(out)))

    def status(self):
        layer = ctypes.c_int(-1)
        code = _lib.hsweep_status(self.raw, ctypes.byref(layer))
        return code, layer.value

    def set_stream(self, stream=None):
        """Enqueue the handle's later work on `stream` (a torch.cuda.Stream; None: the
        current torch stream).  Ordering against work already enqueued is the caller's."""
        s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(_lib.hsweep_set_stream(self.raw, ctypes.c_void_p(s)), "hsweep_set_stream")

    def profile(self, enable=True):
        _check(_lib.hsweep_profile(self.raw, 1 if enable else 0), "hsweep_profile")

    def stats(self, reset=False):
        """(kernel launches, timed sweep launches, summed sweep device ms) since the last reset."""
        a, b, ms = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
        _check(_lib.hsweep_stats(self.raw, 1 if reset else 0, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)),
               "hsweep_stats")
        return a.value, b.value, ms.value

    def sweep_plan(self, nrhs):
        out = (ctypes.c_longlong * 8)()
        _check(_lib.hsweep_sweep_plan(self.raw, nrhs, out), "hsweep_sweep_plan")
        keys = ["tma", "team_ctas", "rhs_per_team", "teams", "grid_or_threads", "smem", "record_bytes_max",
                "leaves_per_chunk"]
        return dict(zip(keys, list(out)))

    def setup_tuning(self):
        """The setup's choice of core-product kernel per kind of recompression launch
        (hsweep_setup_tuning): {"after_depth": mode, "per_layer": mode, "ms": [[cc, tc], [cc, tc]]},
        mode -1 not tuned, 0 CUDA cores, 1 tensor cores."""
        out = (ctypes.c_double * 6)()
        _check(_lib.hsweep_setup_tuning(self.raw, out), "hsweep_setup_tuning")
        v = list(out)
        return {"after_depth": int(v[0]), "per_layer": int(v[1]), "ms": [[v[2], v[3]], [v[4], v[5]]]}

    def layer_ranks(self, m):
        L = self.info()["L"]
        out = (ctypes.c_int * (1 << (L + 1)))()
        _check(_lib.hsweep_layer_ranks(self.raw, m, out), "hsweep_layer_ranks")
        return list(out)

    # -- compute ------------------------------------------------------------------------
    def apply(self, r, z=None):
        """z = M r (Algorithm 2.6)."""
        r2 = r.reshape(-1, self.N)
        if z is None:
            z = torch.empty_like(r2)
        _check(_lib.hsweep_apply(self.raw, _ptr(r2, torch.complex128), _ptr(z, torch.complex128),
                                 r2.shape[0]), "hsweep_apply")
        return z.reshape(r.shape)

    def matvec(self, x, y=None):
        """y = A x (Eq. helmd)."""
        x2 = x.reshape(-1, self.N)
        if y is None:
            y = torch.empty_like(x2)
        _check(_lib.hsweep_matvec(self.raw, _ptr(x2, torch.complex128), _ptr(y, torch.complex128),
                                  x2.shape[0]), "hsweep_matvec")
        return y.reshape(x.shape)

    def boundary_rhs(self, side, b, f):
        """f -= (edge coefficient) * b on the unknowns next to `side` (0: x1 = 0, 1: x1 = 1,
        2: x2 = 0, 3: x2 = 1): Dirichlet data b ((nrhs, n) complex128) moved into f
        ((nrhs, n*n) complex128, updated in place; Section 2.5)."""
        f2 = f.reshape(-1, self.N)
        b2 = b.reshape(f2.shape[0], -1).contiguous()
        _check(_lib.hsweep_boundary_rhs(self.raw, int(side), _ptr(b2, torch.complex128), _ptr(f2, torch.complex128),
                                        f2.shape[0]), "hsweep_boundary_rhs")
        return f

    def solve(self, f, tol, u=None, check=True):
        """GMRES on M A u = M f; returns (u, iterations per RHS, true relative residuals)."""
        f2 = f.reshape(-1, self.N)
        nrhs = f2.shape[0]
        if u is None:
            u = torch.zeros_like(f2)
        it = (ctypes.c_int * nrhs)()
        rr = (ctypes.c_double * nrhs)()
        code = _lib.hsweep_solve(self.raw, _ptr(f2, torch.complex128), _ptr(u, torch.complex128), nrhs,
                                 float(tol), it, rr)
        if check and code not in (OK,):
            raise HSweepError(code, "hsweep_solve")
        return u.reshape(f.shape), list(it), list(rr)

    def grad(self, f, rec_idx, d, tol):
        """Misfit and its gradient with respect to c: returns (J, grad (n*n,) float64)."""
        f2 = f.reshape(-1, self.N)
        g = torch.empty(self.N, dtype=torch.float64, device=f.device)
        J = ctypes.c_double(0.0)
        rec = rec_idx.to(device=f.device, dtype=torch.int32).contiguous()
        d2 = d.reshape(f2.shape[0], -1).contiguous()
        _check(_lib.hsweep_grad(self.raw, _ptr(f2, torch.complex128), f2.shape[0], _ptr(rec, torch.int32),
                                rec.numel(), _ptr(d2, torch.complex128), _ptr(g, torch.float64),
                                ctypes.byref(J), float(tol)), "hsweep_grad")
        return J.value, g

    # -- layer I/O (host, complex128) ---------------------------------------------------
    def _layer_sizes(self):
        inf = self.info()
        L, leaf, r_max = inf["L"], inf["leaf"], inf["r_max"]
        return (1 << L) * leaf * leaf, self.n * L * r_max, 1 << (L + 1)

    def export_layer(self, m):
        import numpy as np
        nl, nf, nn = self._layer_sizes()
        leaves = np.zeros(nl, np.complex128)
        fac = np.zeros(nf, np.complex128)
        ranks = (ctypes.c_int * nn)()
        _check(_lib.hsweep_export_layer(self.raw, m, leaves.ctypes.data_as(ctypes.c_void_p),
                                        fac.ctypes.data_as(ctypes.c_void_p), ranks), "hsweep_export_layer")
        return leaves, fac, np.array(list(ranks), dtype=np.int32)

    def strong_export(self, m):
        """Layer m in the strongly admissible format of the strong sweep: (records, recoff,
        rstride) as numpy arrays (hsweep_strong_export)."""
        import numpy as np
        nleaves = 1 << self.info()["L"]
        ne = ctypes.c_longlong(0)
        _check(_lib.hsweep_strong_export(self.raw, m, None, None, None, ctypes.byref(ne)), "hsweep_strong_export")
        rec = np.zeros(ne.value, np.complex128)
        recoff = (ctypes.c_longlong * (nleaves + 1))()
        rstride = (ctypes.c_int * nleaves)()
        _check(_lib.hsweep_strong_export(self.raw, m, rec.ctypes.data_as(ctypes.c_void_p), recoff, rstride,
                                         ctypes.byref(ne)), "hsweep_strong_export")
        return rec, np.array(list(recoff), dtype=np.int64), np.array(list(rstride), dtype=np.int64)

    def import_layer(self, m, leaves, fac, ranks):
        import numpy as np
        nl, nf, nn = self._layer_sizes()
        leaves = np.ascontiguousarray(leaves, np.complex128)
        fac = np.ascontiguousarray(fac, np.complex128)
        assert leaves.size == nl and fac.size == nf and len(ranks) == nn
        rk = (ctypes.c_int * nn)(*[int(x) for x in ranks])
        _check(_lib.hsweep_import_layer(self.raw, m, leaves.ctypes.data_as(ctypes.c_void_p),
                                        fac.ctypes.data_as(ctypes.c_void_p), rk), "hsweep_import_layer")


def _make(fn, c, omega, pml_width, eps_H, opts, name):
    if not (c.is_cuda and c.dtype == torch.float64 and c.dim() == 2 and c.shape[0] == c.shape[1]):
        raise ValueError("c must be an (n, n) float64 CUDA tensor")
    c = c.contiguous()
    n = c.shape[0]
    raw = ctypes.c_void_p()
    o = opts if opts is not None else default_opts()
    _check(fn(ctypes.c_void_p(c.data_ptr()), float(omega), n, int(pml_width), float(eps_H), ctypes.byref(o),
              _stream(), ctypes.byref(raw)), name)
    return Handle(raw, n)


def hsweep_setup(c, omega, pml_width, eps_H, opts=None):
    """Assemble A and run the setup sweep of Algorithm 2.5 on the GPU."""
    return _make(_lib.hsweep_setup, c, omega, pml_width, eps_H, opts, "hsweep_setup")


def hsweep_create(c, omega, pml_width, eps_H, opts=None):
    """Assemble A only (empty factors, for import_layer)."""
    return _make(_lib.hsweep_create, c, omega, pml_width, eps_H, opts, "hsweep_create")


def hsweep_apply(h, r, z=None):
    return h.apply(r, z)


def hsweep_apply_noalloc(h, r, z):
    """z = M r with the library's fixed scratch array (no device allocation); r and z
    are preallocated (nrhs, n*n) complex128 CUDA tensors."""
    r2 = r.reshape(-1, h.N)
    _check(_lib.hsweep_apply_noalloc(h.raw, _ptr(r2, torch.complex128), _ptr(z, torch.complex128), r2.shape[0]),
           "hsweep_apply_noalloc")
    return z


def hsweep_matvec(h, x, y=None):
    return h.matvec(x, y)


def hsweep_solve(h, f, tol, u=None, check=True):
    return h.solve(f, tol, u, check)


def hsweep_grad(h, f, rec_idx, d, tol):
    return h.grad(f, rec_idx, d, tol)


def hsweep_status(h):
    return h.status()


def hsweep_free(h):
    h.free()
