"""Thin ctypes binding of the nlfem C-ABI (argument marshalling only).

Every step of the method runs in the CUDA kernels of ``libnlfem.so``; this
module only converts arrays, passes PyTorch's caching allocator and current
stream to the library, and wraps the returned handles.  If the shared
library is missing the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnlfem.so")

NL_OK, NL_EINVAL, NL_ENOMEM, NL_ECUDA, NL_ENOTCONV, NL_ETIMEOUT, NL_EBUSY, NL_EGEOM = range(8)
NOCAPS, APPROXCAPS, FULLCAPS = 0, 1, 2
BARYCENTER, OVERLAP, INSIDE = 3, 4, 5
FULLCAPS_QMC = 6      # fullcaps with digitally shifted Sobol' cap points (nl_strategy)
FP64, FP32_COMP = 0, 1
HOST, DEVICE = 0, 1
MAT_K, MAT_A, MAT_LIFT = 0, 1, 2

_STATUS = {0: "NL_OK", 1: "NL_EINVAL", 2: "NL_ENOMEM", 3: "NL_ECUDA", 4: "NL_ENOTCONV", 5: "NL_ETIMEOUT",
           6: "NL_EBUSY", 7: "NL_EGEOM"}


class NlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class nl_device(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p), ("stream", C.c_void_p)]


class nl_pairs_info(C.Structure):
    _fields_ = [("n_vert", C.c_int64), ("n_tet", C.c_int64), ("n_outer", C.c_int64), ("n_pairs", C.c_int64),
                ("nnz", C.c_int64), ("n_free", C.c_int64), ("nnz_a", C.c_int64), ("max_row", C.c_int32),
                ("delta", C.c_double), ("nnz_lift", C.c_int64)]


class nl_assemble_opts(C.Structure):
    _fields_ = [("strategy", C.c_int), ("mc_points", C.c_int), ("seed", C.c_uint64), ("precision", C.c_int),
                ("gamma", C.c_double), ("f_const", C.c_double), ("g_nodal", C.c_void_p), ("g_where", C.c_int),
                ("f_nodal", C.c_void_p), ("f_where", C.c_int), ("kernel_poly", C.c_void_p)]


class nl_csr_view(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class nl_assemble_stats(C.Structure):
    _fields_ = [("pairs", C.c_uint64), ("cut_points", C.c_uint64), ("inside_points", C.c_uint64),
                ("mc_samples", C.c_uint64), ("mc_accepted", C.c_uint64), ("hull_fallbacks", C.c_uint64),
                ("quadrature_ms", C.c_double), ("reduce_ms", C.c_double), ("classify_ms", C.c_double),
                ("events_ms", C.c_double), ("combine_ms", C.c_double)]


class nl_batch_opts(C.Structure):
    _fields_ = [("autotune", C.c_int), ("use_graph", C.c_int), ("units_per_chunk", C.c_int64),
                ("classify_threads", C.c_int)]


class nl_batch_info(C.Structure):
    _fields_ = [("n_problems", C.c_int), ("n_groups", C.c_int), ("graph", C.c_int),
                ("launches_per_run", C.c_uint64), ("last_run_ms", C.c_double), ("units_per_chunk", C.c_int64),
                ("classify_threads", C.c_int), ("n_tried", C.c_int), ("tried_units_per_chunk", C.c_int64 * 16),
                ("tried_classify_threads", C.c_int * 16), ("tried_ms", C.c_double * 16), ("pairs", C.c_uint64),
                ("cut_points", C.c_uint64), ("inside_points", C.c_uint64), ("mc_samples", C.c_uint64),
                ("mc_accepted", C.c_uint64), ("hull_fallbacks", C.c_uint64)]


class nl_solve_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int), ("mixed", C.c_int), ("inner_rtol", C.c_double),
                ("check_every", C.c_int)]


class nl_server_opts(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("workers", C.c_int), ("queue_capacity", C.c_int), ("cache", C.c_int)]


class nl_request(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("cells", C.c_int32), ("omega_lo", C.c_double),
                ("omega_hi", C.c_double), ("delta", C.c_double), ("assemble", nl_assemble_opts),
                ("g_quadratic", C.c_int), ("solve", nl_solve_opts), ("jitter_frac", C.c_double),
                ("jitter_seed", C.c_uint64)]


class nl_result(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("assemble_ms", C.c_double), ("solve_ms", C.c_double),
                ("n_pairs", C.c_int64), ("n_free", C.c_int64), ("n_vert", C.c_int64), ("est_bytes", C.c_int64),
                ("iterations", C.c_int), ("refinements", C.c_int), ("cache_hit", C.c_int),
                ("queue_depth_at_start", C.c_int), ("rel_residual", C.c_double), ("message", C.c_char * 160)]


class nl_server_load(C.Structure):
    _fields_ = [("queued", C.c_int), ("running", C.c_int), ("cache_entries", C.c_int), ("cache_bytes", C.c_int64),
                ("running_bytes", C.c_int64)]


class nl_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("rel_residual", C.c_double),
                ("barrier_fallbacks", C.c_int)]


# every symbol the header declares (checked by the CPU test suite)
EXPORTED = ["nl_mesh_create", "nl_mesh_destroy", "nl_pairs_build", "nl_pairs_destroy", "nl_pairs_get_info",
            "nl_pairs_export", "nl_assemble", "nl_system_destroy", "nl_system_csr", "nl_system_rhs",
            "nl_system_stats", "nl_solve", "nl_probe_moments", "nl_probe_philox", "nl_last_error", "nl_version", "nl_kernel_launches",
            "nl_solve_static", "nl_batch_create", "nl_batch_run", "nl_batch_system", "nl_batch_get_info",
            "nl_batch_destroy", "nl_mesh_create_box", "nl_server_create", "nl_server_submit", "nl_server_poll",
            "nl_server_wait", "nl_server_release", "nl_server_get_load", "nl_server_destroy", "nl_spmv_time",
            "nl_probe_mc_samples", "nl_probe_qmc_samples", "nl_probe_alu_rates"]

_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libnlfem.so is not built; run __graft_entry__.build() or "
                          "python paper_2302_07499_gb300/build.py (nvcc, sm_103a)")
    L = C.CDLL(LIB_PATH)
    vp, i64, dp = C.c_void_p, C.c_int64, C.c_double
    L.nl_mesh_create.argtypes = [C.POINTER(nl_device), vp, i64, vp, i64, vp, vp, C.c_int, C.POINTER(vp)]
    L.nl_mesh_destroy.argtypes = [vp]
    L.nl_mesh_destroy.restype = None
    L.nl_pairs_build.argtypes = [vp, dp, C.POINTER(vp)]
    L.nl_pairs_destroy.argtypes = [vp]
    L.nl_pairs_destroy.restype = None
    L.nl_pairs_get_info.argtypes = [vp, C.POINTER(nl_pairs_info)]
    L.nl_pairs_export.argtypes = [vp, vp, vp, vp, C.c_int]
    L.nl_assemble.argtypes = [vp, C.POINTER(nl_assemble_opts), C.POINTER(vp)]
    L.nl_system_destroy.argtypes = [vp]
    L.nl_system_destroy.restype = None
    L.nl_system_csr.argtypes = [vp, C.c_int, C.POINTER(nl_csr_view)]
    L.nl_system_rhs.argtypes = [vp, C.POINTER(vp), C.POINTER(vp)]
    L.nl_system_stats.argtypes = [vp, C.POINTER(nl_assemble_stats)]
    L.nl_solve.argtypes = [vp, C.POINTER(nl_solve_opts), vp, C.c_int, C.POINTER(nl_solve_info)]
    L.nl_probe_moments.argtypes = [vp, vp, vp, i64, dp, C.c_int, C.c_int, C.c_uint64, C.c_int, vp]
    L.nl_probe_philox.argtypes = [vp, C.c_uint64, i64, vp]
    L.nl_probe_alu_rates.argtypes = [vp, C.c_int]
    L.nl_probe_mc_samples.argtypes = [vp, vp, vp, i64, dp, C.c_int, C.c_uint64, C.c_int, vp, vp, vp, vp]
    L.nl_probe_qmc_samples.argtypes = L.nl_probe_mc_samples.argtypes
    L.nl_last_error.restype = C.c_char_p
    L.nl_version.restype = C.c_char_p
    L.nl_kernel_launches.restype = C.c_uint64
    L.nl_batch_create.argtypes = [vp, vp, C.c_int, C.POINTER(nl_batch_opts), C.POINTER(vp)]
    L.nl_batch_run.argtypes = [vp]
    L.nl_batch_system.argtypes = [vp, C.c_int, C.POINTER(vp)]
    L.nl_batch_get_info.argtypes = [vp, C.POINTER(nl_batch_info)]
    L.nl_batch_destroy.argtypes = [vp]
    L.nl_batch_destroy.restype = None
    L.nl_mesh_create_box.argtypes = [C.POINTER(nl_device), dp, dp, C.c_int32, dp, dp, dp, C.c_uint64, C.POINTER(vp)]
    L.nl_server_create.argtypes = [C.POINTER(nl_server_opts), C.POINTER(vp)]
    L.nl_server_submit.argtypes = [vp, C.POINTER(nl_request), C.POINTER(C.c_uint64)]
    L.nl_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(nl_result)]
    L.nl_server_wait.argtypes = [vp, C.c_uint64, dp, C.POINTER(nl_result), vp, i64]
    L.nl_server_release.argtypes = [vp, C.c_uint64]
    L.nl_server_get_load.argtypes = [vp, C.POINTER(nl_server_load)]
    L.nl_server_destroy.argtypes = [vp]
    L.nl_server_destroy.restype = None
    L.nl_spmv_time.argtypes = [vp, C.c_int, C.c_int, i64, C.POINTER(dp), C.POINTER(dp)]
    _lib = L
    return L


def _check(st):
    if st != NL_OK:
        raise NlError(st, lib().nl_last_error().decode())


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (data must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


class Device:
    """Allocator hooks bound to PyTorch's caching allocator and a CUDA stream."""

    def __init__(self, stream=None, use_torch=True):
        import torch
        self.torch = torch
        self.dev_index = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._live = {}
        if use_torch:
            def _alloc(n, ctx):
                try:
                    p = torch.cuda.caching_allocator_alloc(int(n), self.dev_index, self.stream)
                except Exception:
                    return None
                return p

            def _free(p, ctx):
                torch.cuda.caching_allocator_delete(p)

            self._a = ALLOC_FN(_alloc)
            self._f = FREE_FN(_free)
        else:
            self._a = ALLOC_FN()
            self._f = FREE_FN()
        self.c = nl_device(self._a, self._f, None, C.c_void_p(self.stream.cuda_stream))


class _CAI:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}


def _as_tensor(ptr, n, dtype):
    import torch
    ts = {torch.float64: "<f8", torch.int64: "<i8", torch.int32: "<i4", torch.float32: "<f4"}[dtype]
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_CAI(ptr, n, ts), device="cuda")


class Mesh:
    def __init__(self, verts, tets, tet_in_omega, node_free, device: Device | None = None, unfolded: bool = False):
        """unfolded=True marks every element as an outer element (tet_in_omega
        all 1): the assembly is then the unfolded form of Eq. weak0, outer
        integral over all of Omega-hat and no collar weight (nl_mesh_create)."""
        import torch
        self.device = device or Device()
        self._keep = []
        if unfolded:
            tet_in_omega = (torch.ones_like(tet_in_omega) if isinstance(tet_in_omega, torch.Tensor)
                            else np.ones(len(tet_in_omega), dtype=np.uint8))
        if isinstance(verts, torch.Tensor) and verts.is_cuda:
            arrs = [verts.contiguous().double(), tets.contiguous().int(), tet_in_omega.contiguous().to(torch.uint8),
                    node_free.contiguous().to(torch.uint8)]
            where = DEVICE
        else:
            arrs = [np.ascontiguousarray(verts, dtype=np.float64), np.ascontiguousarray(tets, dtype=np.int32),
                    np.ascontiguousarray(tet_in_omega, dtype=np.uint8),
                    np.ascontiguousarray(node_free, dtype=np.uint8)]
            where = HOST
        self._keep = arrs
        self.nv = int(arrs[0].shape[0])
        self.nt = int(arrs[1].shape[0])
        h = C.c_void_p()
        _check(lib().nl_mesh_create(C.byref(self.device.c), _ptr(arrs[0]), self.nv, _ptr(arrs[1]), self.nt,
                                    _ptr(arrs[2]), _ptr(arrs[3]), where, C.byref(h)))
        self.h = h
        self._keep = None

    @classmethod
    def from_handle(cls, h, device, nv, nt):
        m = cls.__new__(cls)
        m.device, m._keep, m.h, m.nv, m.nt = device, None, h, int(nv), int(nt)
        return m

    def close(self):
        if getattr(self, "h", None):
            lib().nl_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pairs:
    def __init__(self, mesh: Mesh, delta: float):
        self.mesh = mesh
        h = C.c_void_p()
        _check(lib().nl_pairs_build(mesh.h, float(delta), C.byref(h)))
        self.h = h
        inf = nl_pairs_info()
        _check(lib().nl_pairs_get_info(self.h, C.byref(inf)))
        self.info = {k: getattr(inf, k) for k, _ in nl_pairs_info._fields_}

    def export(self):
        n_outer, npairs = self.info["n_outer"], self.info["n_pairs"]
        outer = np.zeros(n_outer, dtype=np.int32)
        ptr = np.zeros(n_outer + 1, dtype=np.int64)
        tp = np.zeros(max(npairs, 1), dtype=np.int32)
        _check(lib().nl_pairs_export(self.h, _ptr(outer), _ptr(ptr), _ptr(tp), HOST))
        return outer, ptr, tp[:npairs]

    def close(self):
        if getattr(self, "h", None):
            lib().nl_pairs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    def __init__(self, pairs: Pairs, strategy=NOCAPS, mc_points=64, seed=1, precision=FP64, gamma=1.0,
                 f_const=0.0, g=None, f=None, kernel=None):
        """g: nodal volume constraint; f: nodal source values added to f_const
        (numpy arrays or CUDA tensors of n_vert doubles, or None); kernel: the
        kernel shape's 4 coefficients (None: constant kernel)."""
        self.pairs = pairs
        o, keep = _assemble_opts(strategy, mc_points, seed, precision, gamma, f_const, g, f, kernel)
        h = C.c_void_p()
        _check(lib().nl_assemble(pairs.h, C.byref(o), C.byref(h)))
        self.h = h
        del keep

    def csr(self, which=MAT_K):
        """(rowptr, col, val) as torch CUDA tensors viewing library memory (valid until close)."""
        import torch
        v = nl_csr_view()
        _check(lib().nl_system_csr(self.h, int(which), C.byref(v)))
        return (_as_tensor(v.rowptr, v.n_rows + 1, torch.int64), _as_tensor(v.col, v.nnz, torch.int32),
                _as_tensor(v.val, v.nnz, torch.float64))

    def csr_numpy(self, which=MAT_K):
        rp, c, v = self.csr(which)
        return rp.cpu().numpy(), c.cpu().numpy(), v.cpu().numpy()

    def scipy(self, which=MAT_K):
        import scipy.sparse as sp
        rp, c, v = self.csr_numpy(which)
        n = rp.size - 1
        ncol = self.pairs.info["n_vert"] if which == MAT_LIFT else n
        return sp.csr_matrix((v, c, rp), shape=(n, ncol))

    def rhs(self):
        import torch
        b = C.c_void_p()
        fn = C.c_void_p()
        _check(lib().nl_system_rhs(self.h, C.byref(b), C.byref(fn)))
        nf = self.pairs.info["n_free"]
        return _as_tensor(b.value, nf, torch.float64), _as_tensor(fn.value, nf, torch.int32)

    def stats(self):
        s = nl_assemble_stats()
        _check(lib().nl_system_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in nl_assemble_stats._fields_}

    def solve(self, rtol=1e-12, max_iter=0, mixed=False, inner_rtol=0.0, check_every=0, out=None):
        """Returns (u, info).  u: full nodal vector; numpy unless `out` is a CUDA tensor."""
        o = nl_solve_opts(float(rtol), int(max_iter), int(bool(mixed)), float(inner_rtol), int(check_every))
        inf = nl_solve_info()
        if out is None:
            u = np.zeros(self.pairs.info["n_vert"])
            where = HOST
        else:
            u = out
            where = DEVICE
        st = lib().nl_solve(self.h, C.byref(o), _ptr(u), where, C.byref(inf))
        info = {"iterations": inf.iterations, "refinements": inf.refinements, "rel_residual": inf.rel_residual,
                "barrier_fallbacks": inf.barrier_fallbacks, "status": st}
        if st not in (NL_OK, NL_ENOTCONV):
            _check(st)
        return u, info

    def spmv_time(self, precision=FP64, reps=50, flush_bytes=0):
        """(ms per SpMV of the CG on A, algorithmic bytes per SpMV); with
        flush_bytes > 0 each launch is timed alone after an L2 flush."""
        ms, by = C.c_double(), C.c_double()
        _check(lib().nl_spmv_time(self.h, int(precision), int(reps), int(flush_bytes), C.byref(ms), C.byref(by)))
        return ms.value, by.value

    def close(self):
        if getattr(self, "h", None):
            lib().nl_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _nodal(a):
    """(kept array, pointer, where) of optional nodal values."""
    if a is None:
        return None, None, HOST
    if isinstance(a, np.ndarray):
        k = np.ascontiguousarray(a, dtype=np.float64)
        return k, _ptr(k), HOST
    k = a.contiguous().double()
    return k, _ptr(k), DEVICE


def _assemble_opts(strategy=NOCAPS, mc_points=64, seed=1, precision=FP64, gamma=1.0, f_const=0.0, g=None, f=None,
                   kernel=None):
    """nl_assemble_opts and the arrays that must stay alive while the call runs.
    kernel: None (constant kernel) or the 4 coefficients of the kernel shape
    phi(s) = c0 + c1 s + c2 s^2 + c3 s^3, s = min(|x - y|^2 / delta^2, 1)."""
    kg, gp, gw = _nodal(g)
    kf, fp, fw = _nodal(f)
    kk, kp = None, None
    if kernel is not None:
        coef = [float(c) for c in kernel]
        if len(coef) != 4:
            raise ValueError("kernel needs 4 coefficients")
        kk = (C.c_double * 4)(*coef)
        kp = C.cast(kk, C.c_void_p)
    o = nl_assemble_opts(int(strategy), int(mc_points), int(seed), int(precision), float(gamma), float(f_const),
                         gp, gw, fp, fw, kp)
    return o, (kg, kf, kk)


class _BorrowedSystem(System):
    """A system owned by a batch (closing it does nothing)."""

    def __init__(self, pairs, h):
        self.pairs = pairs
        self.h = h

    def close(self):
        self.h = None


class Batch:
    """Batched assembly of independent problems (nl_batch_*).

    problems: list of (Pairs, dict of System options).  Each problem's system
    is bitwise equal to System(pairs, **options)."""

    def __init__(self, problems, autotune=True, use_graph=True, shape=None):
        self.pairs = [p for p, _ in problems]
        n = len(problems)
        arr = (nl_assemble_opts * n)()
        keep = []
        for i, (_, kw) in enumerate(problems):
            o, k = _assemble_opts(**kw)
            arr[i] = o
            keep.append(k)
        hp = (C.c_void_p * n)(*[p.h for p in self.pairs])
        up, ct = shape if shape else (0, 0)
        bo = nl_batch_opts(int(bool(autotune)), int(bool(use_graph)), int(up), int(ct))
        h = C.c_void_p()
        _check(lib().nl_batch_create(C.cast(hp, C.c_void_p), C.cast(arr, C.c_void_p), n, C.byref(bo), C.byref(h)))
        self.h = h
        del keep

    def run(self):
        _check(lib().nl_batch_run(self.h))

    def system(self, i):
        h = C.c_void_p()
        _check(lib().nl_batch_system(self.h, int(i), C.byref(h)))
        return _BorrowedSystem(self.pairs[i], h)

    def info(self):
        inf = nl_batch_info()
        _check(lib().nl_batch_get_info(self.h, C.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in nl_batch_info._fields_ if not k.startswith("tried")}
        d["tried"] = [(int(inf.tried_units_per_chunk[k]), int(inf.tried_classify_threads[k]), float(inf.tried_ms[k]))
                      for k in range(inf.n_tried)]
        return d

    def close(self):
        if getattr(self, "h", None):
            lib().nl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(r):
    d = {k: getattr(r, k) for k, _ in nl_result._fields_ if k != "message"}
    d["message"] = r.message.decode(errors="replace")
    return d


class Server:
    """Request server (nl_server_*): assemble-and-solve requests on Kuhn box
    meshes, served by `workers` concurrent device streams under an admission
    budget, with mesh / pairs / pattern residency between requests."""

    def __init__(self, budget_bytes=150 * 10 ** 9, workers=4, queue_capacity=100000, cache=True):
        o = nl_server_opts(int(budget_bytes), int(workers), int(queue_capacity), int(bool(cache)))
        h = C.c_void_p()
        _check(lib().nl_server_create(C.byref(o), C.byref(h)))
        self.h = h

    @staticmethod
    def box_request(inv_h, ratio, strategy=NOCAPS, mc_points=64, seed=1, precision=FP64, f_const=-6.0,
                    g_quadratic=True, rtol=1e-10, mixed=False, max_iter=0, gamma=None, jitter_frac=0.0,
                    jitter_seed=0):
        """The unit-cube problem with h = 1/inv_h, delta = ratio*h and a collar
        of ceil(ratio) cells (the box of the inputs module's cube_problem)."""
        import math
        h = 1.0 / inv_h
        collar = int(math.ceil(ratio - 1e-12))
        lo, hi = -collar * h, 1.0 + collar * h
        delta = ratio * h
        if gamma is None:
            gamma = 15.0 / (2.0 * math.pi * delta ** 5)
        a = nl_assemble_opts(int(strategy), int(mc_points), int(seed), int(precision), float(gamma), float(f_const),
                             None, HOST, None, HOST)
        sv = nl_solve_opts(float(rtol), int(max_iter), int(bool(mixed)), 0.0, 0)
        return nl_request(lo, hi, inv_h + 2 * collar, 0.0, 1.0, delta, a, int(bool(g_quadratic)), sv,
                          float(jitter_frac), int(jitter_seed))

    def submit(self, req):
        t = C.c_uint64()
        _check(lib().nl_server_submit(self.h, C.byref(req), C.byref(t)))
        return int(t.value)

    def poll(self, ticket):
        r = nl_result()
        _check(lib().nl_server_poll(self.h, int(ticket), C.byref(r)))
        return _result_dict(r)

    def wait(self, ticket, timeout_s=0.0, want_u=False):
        """(result dict, u or None); does not release the ticket."""
        r = nl_result()
        _check(lib().nl_server_poll(self.h, int(ticket), C.byref(r)))
        u = None
        if want_u:
            st = lib().nl_server_wait(self.h, int(ticket), float(timeout_s), C.byref(r), None, 0)
            if st != NL_OK:
                _check(st)
            u = np.zeros(r.n_vert)
            _check(lib().nl_server_wait(self.h, int(ticket), float(timeout_s), C.byref(r), u.ctypes.data, u.size))
        else:
            _check(lib().nl_server_wait(self.h, int(ticket), float(timeout_s), C.byref(r), None, 0))
        return _result_dict(r), u

    def release(self, ticket):
        _check(lib().nl_server_release(self.h, int(ticket)))

    def load(self):
        o = nl_server_load()
        _check(lib().nl_server_get_load(self.h, C.byref(o)))
        return {k: getattr(o, k) for k, _ in nl_server_load._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().nl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_box(lo, hi, cells, omega_lo=0.0, omega_hi=1.0, device=None, jitter_frac=0.0, seed=0):
    """nl_mesh_create_box: a Kuhn box mesh (optionally jittered) generated on the device."""
    device = device or Device()
    h = C.c_void_p()
    _check(lib().nl_mesh_create_box(C.byref(device.c), float(lo), float(hi), int(cells), float(omega_lo),
                                    float(omega_hi), float(jitter_frac), int(seed), C.byref(h)))
    return Mesh.from_handle(h, device, (cells + 1) ** 3, 6 * cells ** 3)


def kernel_launches():
    return int(lib().nl_kernel_launches())


def probe_moments(tets_xyz, x, ids, delta, strategy, mc_points=0, seed=1, precision=FP64):
    tv = np.ascontiguousarray(tets_xyz, dtype=np.float64).reshape(-1, 12)
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    ii = np.ascontiguousarray(ids, dtype=np.uint32).reshape(-1, 3)
    n = tv.shape[0]
    out = np.zeros((n, 15))
    _check(lib().nl_probe_moments(_ptr(tv), _ptr(xs), _ptr(ii), n, float(delta), int(strategy), int(mc_points),
                                  int(seed), int(precision), _ptr(out)))
    return out


def probe_mc_samples(tets_xyz, x, ids, delta, mc_points, seed=1, precision=FP64, qmc=False):
    """(n_samples [n], cell [n, mc], accepted [n, mc], y [n, mc, 3]) of the
    fullcaps Monte Carlo samples of single cases (nl_probe_mc_samples; with
    qmc, the shifted Sobol' samples of nl_probe_qmc_samples)."""
    tv = np.ascontiguousarray(tets_xyz, dtype=np.float64).reshape(-1, 12)
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    ii = np.ascontiguousarray(ids, dtype=np.uint32).reshape(-1, 3)
    n = tv.shape[0]
    ns = np.zeros(n, dtype=np.int32)
    cell = np.zeros((n, mc_points), dtype=np.int32)
    acc = np.zeros((n, mc_points), dtype=np.uint8)
    y = np.zeros((n, mc_points, 3))
    fn = lib().nl_probe_qmc_samples if qmc else lib().nl_probe_mc_samples
    _check(fn(_ptr(tv), _ptr(xs), _ptr(ii), n, float(delta), int(mc_points), int(seed),
              int(precision), _ptr(ns), _ptr(cell), _ptr(acc), _ptr(y)))
    return ns, cell, acc.astype(bool), y


ALU_RATE_NAMES = ("ffma_fp32", "dfma_fp64", "mad_lo_u32", "mul_hi_u32", "xor3_as_2", "philox_ops",
                  "fullcaps_sample_ops")


def probe_alu_rates():
    """Measured operations per second of the ALU microbenchmarks of
    nl_probe_alu_rates, by name."""
    out = np.zeros(len(ALU_RATE_NAMES))
    _check(lib().nl_probe_alu_rates(_ptr(out), out.size))
    return dict(zip(ALU_RATE_NAMES, out.tolist()))


def probe_philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    _check(lib().nl_probe_philox(_ptr(c), int(key), c.shape[0], _ptr(out)))
    return out
