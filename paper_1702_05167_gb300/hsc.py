"""Thin ctypes binding of libhsc (include/hsc.h): same entry-point names, argument marshalling only.

Every step of the solve runs inside libhsc's CUDA kernels; this module only converts numpy arrays or
torch tensors to pointers. If the shared library is missing it raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HSC_OK, HSC_ERR_ARG, HSC_ERR_NOT_SYMMETRIC, HSC_ERR_STATE, HSC_ERR_SINGULAR, \
    HSC_ERR_NOT_SELECTED, HSC_ERR_OOM, HSC_ERR_CUDA, HSC_ERR_TIMEOUT = range(9)
HSC_FP64, HSC_MIXED = 0, 1
STATUS = {0: "HSC_OK", 1: "HSC_ERR_ARG", 2: "HSC_ERR_NOT_SYMMETRIC", 3: "HSC_ERR_STATE",
          4: "HSC_ERR_SINGULAR", 5: "HSC_ERR_NOT_SELECTED", 6: "HSC_ERR_OOM", 7: "HSC_ERR_CUDA",
          8: "HSC_ERR_TIMEOUT"}

EXPORTS = ["hsc_create", "hsc_analyze", "hsc_cluster", "hsc_solve", "hsc_solve_batch",
           "hsc_tune", "hsc_set_option", "hsc_get_option", "hsc_set_contact_dense", "hsc_solve_dense",
           "hsc_set_merge",
           "hsc_profile",
           "hsc_profile_read", "hsc_growth", "hsc_cluster_growth",
           "hsc_residual",
           "hsc_device_fp64_peaks", "hsc_observables", "hsc_scba", "hsc_last_error", "hsc_destroy",
           "hsc_mlp_create", "hsc_mlp_num_params", "hsc_mlp_set_params", "hsc_mlp_get_params",
           "hsc_mlp_forward", "hsc_mlp_loss_grad", "hsc_mlp_adam", "hsc_mlp_destroy"]
HSC_OPT_GJ_PANEL, HSC_OPT_FP64_LEVELS, HSC_OPT_MIXED_GJ_FP64, HSC_OPT_LEAF, HSC_OPT_COMPLEX_4M = 1, 2, 3, 4, 5
HSC_OPT_FP64_ENGINE, HSC_OPT_RESOLVE_DIGITS, HSC_OPT_TREE_VARIANT, HSC_OPT_ORDERING = 6, 7, 8, 9
HSC_OPT_MAX_CLUSTER, HSC_OPT_TREE_FORM, HSC_OPT_GJ_WIDE, HSC_OPT_LEAF_BAND, HSC_OPT_LEAF_SPARSE = 10, 11, 12, 13, 14


class hsc_tree_stats(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int32), ("n_heights", ctypes.c_int32),
                ("n_depths", ctypes.c_int32), ("max_n", ctypes.c_int32), ("max_m", ctypes.c_int32),
                ("n_lesser", ctypes.c_int32), ("n_unknowns", ctypes.c_int64),
                ("flops_gr", ctypes.c_double), ("flops_gl", ctypes.c_double),
                ("bytes_per_energy", ctypes.c_int64)]


class hsc_cluster_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("parent", ctypes.c_int32),
                ("child", ctypes.c_int32 * 2), ("height", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("lesser", ctypes.c_int32)]


class hsc_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("timed", ctypes.c_int64),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class hsc_batch_item(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("n_E", ctypes.c_int64), ("E", ctypes.c_void_p),
                ("sigma_r", ctypes.c_void_p), ("sigma_less", ctypes.c_void_p),
                ("n_req", ctypes.c_int32), ("req_pairs", ctypes.c_void_p),
                ("diag_gr", ctypes.c_void_p), ("diag_gl", ctypes.c_void_p),
                ("req_gr", ctypes.c_void_p), ("req_gl", ctypes.c_void_p)]


class hsc_tune_result(ctypes.Structure):
    _fields_ = [("leaf_max", ctypes.c_int32), ("gj_panel", ctypes.c_int32),
                ("ms_per_energy", ctypes.c_double), ("from_cache", ctypes.c_int32),
                ("n_tried", ctypes.c_int32)]


class HSCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def lib_path():
    return os.environ.get("HSC_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                     "libhsc.so")


def load():
    """Load libhsc.so (built in-tree by __graft_entry__.build()); raise if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libhsc.so not found at {p}: build it with __graft_entry__.build()")
    L = ctypes.CDLL(p)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.hsc_create.argtypes = [ctypes.POINTER(vp), i64, i32, vp, vp, vp, i32, vp, vp, vp]
    L.hsc_analyze.argtypes = [vp, i32, ctypes.POINTER(hsc_tree_stats)]
    L.hsc_cluster.argtypes = [vp, i32, ctypes.POINTER(hsc_cluster_info), vp, vp]
    L.hsc_solve.argtypes = [vp, i64, vp, dp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, i32]
    L.hsc_solve_batch.argtypes = [i32, ctypes.POINTER(hsc_batch_item), dp, i32, vp, i32]
    L.hsc_tune.argtypes = [vp, i64, vp, dp, vp, vp, i32, ctypes.c_char_p,
                           ctypes.POINTER(hsc_tune_result)]
    L.hsc_set_option.argtypes = [vp, i32, i32]
    L.hsc_set_contact_dense.argtypes = [vp, i32, i32]
    L.hsc_set_merge.argtypes = [vp, i32, vp]
    L.hsc_solve_dense.argtypes = [vp, i64, vp, dp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, i32]
    L.hsc_get_option.argtypes = [vp, i32, ctypes.POINTER(i32)]
    L.hsc_observables.argtypes = [vp, i64, vp, vp, vp, i32, vp, vp]
    L.hsc_scba.argtypes = [vp, i64, vp, dp, vp, vp, dp, dp, dp, i32, i32, vp, vp,
                           ctypes.POINTER(i32), ctypes.POINTER(dp), vp, i32]
    L.hsc_mlp_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, i32]
    L.hsc_mlp_num_params.argtypes = [vp, ctypes.POINTER(i64)]
    L.hsc_mlp_set_params.argtypes = [vp, vp]
    L.hsc_mlp_get_params.argtypes = [vp, vp]
    L.hsc_mlp_forward.argtypes = [vp, i32, vp, vp, i32, vp]
    L.hsc_mlp_loss_grad.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.hsc_mlp_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
    L.hsc_mlp_destroy.argtypes = [vp]
    L.hsc_profile.argtypes = [vp, i32]
    L.hsc_growth.argtypes = [vp, i64, vp]
    L.hsc_cluster_growth.argtypes = [vp, i64, vp]
    L.hsc_residual.argtypes = [vp, i64, vp]
    L.hsc_profile_read.argtypes = [vp, ctypes.POINTER(hsc_kernel_stat), i32, ctypes.POINTER(i32)]
    L.hsc_device_fp64_peaks.argtypes = [ctypes.POINTER(dp), ctypes.POINTER(dp)]
    L.hsc_last_error.argtypes = [vp]
    L.hsc_last_error.restype = ctypes.c_char_p
    L.hsc_destroy.argtypes = [vp]
    for name in ("hsc_create", "hsc_analyze", "hsc_cluster", "hsc_solve", "hsc_solve_batch",
                 "hsc_tune", "hsc_set_option", "hsc_get_option", "hsc_profile",
                 "hsc_profile_read", "hsc_device_fp64_peaks", "hsc_observables", "hsc_scba",
                 "hsc_set_contact_dense", "hsc_solve_dense", "hsc_set_merge", "hsc_destroy",
                 "hsc_mlp_create", "hsc_mlp_num_params", "hsc_mlp_set_params", "hsc_mlp_get_params",
                 "hsc_mlp_forward", "hsc_mlp_loss_grad", "hsc_mlp_adam", "hsc_mlp_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check_io(on_device, **bufs):
    """Each buffer must hold float64 or complex128 values and live where io_on_device says: CUDA
    tensors for device I/O, numpy arrays or CPU tensors for host I/O. The library cannot tell a
    host pointer from a device one, and a wrong one would be dereferenced by a kernel."""
    for name, a in bufs.items():
        if a is None:
            continue
        if isinstance(a, np.ndarray):
            if on_device:
                raise ValueError(f"{name}: io_on_device needs CUDA tensors, got a numpy array")
            if a.dtype not in (np.float64, np.complex128):
                raise TypeError(f"{name}: float64 or complex128 expected, got {a.dtype}")
        elif hasattr(a, "data_ptr"):
            if bool(a.is_cuda) != bool(on_device):
                raise ValueError(f"{name}: a {'CUDA' if on_device else 'host'} buffer is expected")
            if str(a.dtype) not in ("torch.float64", "torch.complex128"):
                raise TypeError(f"{name}: float64 or complex128 expected, got {a.dtype}")


def _check(h, code):
    if code != HSC_OK:
        msg = load().hsc_last_error(h).decode(errors="replace")
        raise HSCError(code, msg)


def hsc_create(n, orb, rowptr, col, val, contact_ptr, contact_sites, grid_dims=None):
    L = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.complex128)
    contact_ptr = np.ascontiguousarray(contact_ptr, dtype=np.int64)
    contact_sites = np.ascontiguousarray(contact_sites, dtype=np.int32)
    dims = None if grid_dims is None else np.ascontiguousarray(grid_dims, dtype=np.int32)
    h = ctypes.c_void_p()
    code = L.hsc_create(ctypes.byref(h), int(n), int(orb), _ptr(rowptr), _ptr(col), _ptr(val),
                        len(contact_ptr) - 1, _ptr(contact_ptr), _ptr(contact_sites), _ptr(dims))
    _check(None, code)
    return h


def hsc_analyze(h, leaf_max):
    st = hsc_tree_stats()
    _check(h, load().hsc_analyze(h, int(leaf_max), ctypes.byref(st)))
    return st


def hsc_cluster(h, i, want_sets=True):
    info = hsc_cluster_info()
    _check(h, load().hsc_cluster(h, int(i), ctypes.byref(info), None, None))
    own = upd = None
    if want_sets:
        own = np.empty(info.n, dtype=np.int32)
        upd = np.empty(info.m, dtype=np.int32)
        _check(h, load().hsc_cluster(h, int(i), None, _ptr(own), _ptr(upd)))
    return info, own, upd


def hsc_solve(h, E, eta, sigma_r, sigma_less, precision, req_pairs, diag_gr, diag_gl, req_gr,
              req_gl, stream=None, io_on_device=False):
    """Marshal buffers to hsc_solve. Buffers are numpy (host) or torch (device) arrays; complex128
    arrays are passed as interleaved doubles."""
    n_E = int(E.shape[0])
    _check_io(io_on_device, E=E, sigma_r=sigma_r, sigma_less=sigma_less, diag_gr=diag_gr,
              diag_gl=diag_gl, req_gr=req_gr, req_gl=req_gl)
    pairs = None
    n_req = 0
    if req_pairs is not None and len(req_pairs):
        pairs = np.ascontiguousarray(req_pairs, dtype=np.int32)
        n_req = pairs.shape[0]
    s = None if stream is None else ctypes.c_void_p(int(stream))
    code = load().hsc_solve(h, n_E, _ptr(E), float(eta), _ptr(sigma_r), _ptr(sigma_less),
                            int(precision), n_req, _ptr(pairs), _ptr(diag_gr), _ptr(diag_gl),
                            _ptr(req_gr), _ptr(req_gl), s, 1 if io_on_device else 0)
    _check(h, code)


def hsc_scba(h, E, eta, sigma_r, sigma_less, d0, mix, tol, max_iter, precision, diag_gr, diag_gl,
             stream=None, io_on_device=False):
    """Marshal buffers to hsc_scba (as hsc_solve). Returns (solves made, last delta)."""
    _check_io(io_on_device, E=E, sigma_r=sigma_r, sigma_less=sigma_less, diag_gr=diag_gr,
              diag_gl=diag_gl)
    it = ctypes.c_int32()
    dl = ctypes.c_double()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    code = load().hsc_scba(h, int(E.shape[0]), _ptr(E), float(eta), _ptr(sigma_r), _ptr(sigma_less),
                           float(d0), float(mix), float(tol), int(max_iter), int(precision),
                           _ptr(diag_gr), _ptr(diag_gl), ctypes.byref(it), ctypes.byref(dl), s,
                           1 if io_on_device else 0)
    _check(h, code)
    return it.value, dl.value


def hsc_solve_dense(h, E, eta, sigma_r, sigma_less, dense_r, dense_less, precision, req_pairs, diag_gr,
                    diag_gl, req_gr, req_gl, stream=None, io_on_device=False):
    """Marshal buffers to hsc_solve_dense (as hsc_solve, plus the dense contact blocks)."""
    _check_io(io_on_device, E=E, sigma_r=sigma_r, sigma_less=sigma_less, dense_r=dense_r,
              dense_less=dense_less, diag_gr=diag_gr, diag_gl=diag_gl, req_gr=req_gr, req_gl=req_gl)
    pairs = None
    n_req = 0
    if req_pairs is not None and len(req_pairs):
        pairs = np.ascontiguousarray(req_pairs, dtype=np.int32)
        n_req = pairs.shape[0]
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(h, load().hsc_solve_dense(h, int(E.shape[0]), _ptr(E), float(eta), _ptr(sigma_r),
                                     _ptr(sigma_less), _ptr(dense_r), _ptr(dense_less), int(precision),
                                     n_req, _ptr(pairs), _ptr(diag_gr), _ptr(diag_gl), _ptr(req_gr),
                                     _ptr(req_gl), s, 1 if io_on_device else 0))


def hsc_set_option(h, option, value):
    _check(h, load().hsc_set_option(h, int(option), int(value)))


def hsc_set_merge(h, clusters):
    arr = np.ascontiguousarray(clusters, dtype=np.int32)
    _check(h, load().hsc_set_merge(h, len(arr), _ptr(arr) if len(arr) else None))


def hsc_set_contact_dense(h, contact, dense=True):
    _check(h, load().hsc_set_contact_dense(h, int(contact), 1 if dense else 0))


def hsc_get_option(h, option):
    v = ctypes.c_int32()
    _check(h, load().hsc_get_option(h, int(option), ctypes.byref(v)))
    return v.value


def hsc_solve_batch(items, eta, precision, stream=None, use_graph=True):
    """items: list of dicts with keys h, E, sigma_r, sigma_less, pairs, diag_gr, diag_gl, req_gr,
    req_gl (device tensors except `pairs`, a host int32 array or None)."""
    arr = (hsc_batch_item * len(items))()
    keep = []
    for k, it in enumerate(items):
        _check_io(True, **{f"items[{k}].{x}": it.get(x) for x in ("E", "sigma_r", "sigma_less", "diag_gr",
                                                                  "diag_gl", "req_gr", "req_gl")})
        pairs = it.get("pairs")
        if pairs is not None and len(pairs):
            pairs = np.ascontiguousarray(pairs, dtype=np.int32)
            keep.append(pairs)
        else:
            pairs = None
        arr[k] = hsc_batch_item(it["h"], int(it["E"].shape[0]), _ptr(it["E"]), _ptr(it["sigma_r"]),
                                _ptr(it.get("sigma_less")), 0 if pairs is None else len(pairs),
                                _ptr(pairs), _ptr(it["diag_gr"]), _ptr(it.get("diag_gl")),
                                _ptr(it.get("req_gr")), _ptr(it.get("req_gl")))
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(None, load().hsc_solve_batch(len(items), arr, float(eta), int(precision), s,
                                        1 if use_graph else 0))


def hsc_tune(h, E, eta, sigma_r, sigma_less, precision=HSC_FP64, cache_path=None):
    E = np.ascontiguousarray(E, dtype=np.float64)
    sigma_r = np.ascontiguousarray(sigma_r, dtype=np.complex128)
    if sigma_less is not None:
        sigma_less = np.ascontiguousarray(sigma_less, dtype=np.complex128)
    r = hsc_tune_result()
    cp = None if cache_path is None else str(cache_path).encode()
    _check(h, load().hsc_tune(h, len(E), _ptr(E), float(eta), _ptr(sigma_r), _ptr(sigma_less),
                              int(precision), cp, ctypes.byref(r)))
    return dict(leaf_max=r.leaf_max, gj_panel=r.gj_panel, ms_per_energy=r.ms_per_energy,
                from_cache=bool(r.from_cache), n_tried=r.n_tried)


def hsc_growth(h, n_E):
    """Per-energy element growth of the last solve: max over the cluster blocks of max |D_i^{-1}|."""
    out = np.zeros(n_E)
    _check(h, load().hsc_growth(h, int(n_E), _ptr(out)))
    return out


def hsc_cluster_growth(h, n_E, n_clusters):
    """Per-energy, per-cluster ||D_i^{-1}||_F of the last solve (n_E x n_clusters, postorder ids)."""
    out = np.zeros((n_E, n_clusters))
    _check(h, load().hsc_cluster_growth(h, int(n_E), _ptr(out)))
    return out


def hsc_residual(h, n_E):
    """Per-energy residual of the last solve: max_u |(A G^r - I)_uu| from the computed blocks."""
    out = np.zeros(n_E)
    _check(h, load().hsc_residual(h, int(n_E), _ptr(out)))
    return out


def hsc_profile(h, enable):
    _check(h, load().hsc_profile(h, 1 if enable else 0))


def hsc_profile_read(h):
    """Per-kernel-class statistics as a list of dicts (name, launches, timed, ms, flops, bytes)."""
    n = ctypes.c_int32()
    _check(h, load().hsc_profile_read(h, None, 0, ctypes.byref(n)))
    arr = (hsc_kernel_stat * n.value)()
    _check(h, load().hsc_profile_read(h, arr, n.value, ctypes.byref(n)))
    return [dict(name=a.name.decode(), launches=a.launches, timed=a.timed, ms=a.ms, flops=a.flops,
                 bytes=a.bytes) for a in arr]


def hsc_device_fp64_peaks():
    """(FP64 tensor-pipe GFLOP/s, scalar FP64 FMA GFLOP/s) measured on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(None, load().hsc_device_fp64_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hsc_block_inverse_noalloc(n, batch, A, Ainv, stream=None):
    """Invert `batch` n x n complex128 device blocks (torch float64 or complex128 CUDA tensors,
    interleaved re/im) with the library's allocation-free entry point. batch = 0 only sets up the
    current device's scratch (A and Ainv may be None)."""
    if int(batch) > 0:
        if A is None or Ainv is None:
            raise ValueError("A and Ainv are required when batch > 0")
        _check_io(True, A=A, Ainv=Ainv)
        need = int(batch) * int(n) * int(n) * 16
        for name, t in (("A", A), ("Ainv", Ainv)):
            have = t.numel() * t.element_size()
            if have < need:
                raise ValueError(f"{name} holds {have} bytes, {need} needed for {batch} blocks of {n} x {n}")
    L = load()
    L.hsc_block_inverse_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]
    L.hsc_block_inverse_noalloc.restype = ctypes.c_int
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(None, L.hsc_block_inverse_noalloc(int(n), int(batch), _ptr(A), _ptr(Ainv), s))


def hsc_observables(h, diag_gr, diag_gl, sigma_r, contact, out, stream=None):
    """out: device float64 [n_E, 3] <- (DOS, T into `contact`, sum Im G^<) per energy."""
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(h, load().hsc_observables(h, int(diag_gr.shape[0]), _ptr(diag_gr), _ptr(diag_gl),
                                     _ptr(sigma_r), int(contact), _ptr(out), s))


class MLP:
    """Owner of an hsc_mlp handle (include/hsc_mlp.h); buffers are torch CUDA float32 tensors."""

    def __init__(self, n_in, width, hidden, n_out, max_batch):
        L = load()
        self.h = ctypes.c_void_p()
        _check(None, L.hsc_mlp_create(ctypes.byref(self.h), n_in, width, hidden, n_out, max_batch))
        n = ctypes.c_int64()
        _check(None, L.hsc_mlp_num_params(self.h, ctypes.byref(n)))
        self.n_params = n.value
        self.shape = (n_in, width, hidden, n_out)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(None, load().hsc_mlp_set_params(self.h, _ptr(p)))

    def get_params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        _check(None, load().hsc_mlp_get_params(self.h, _ptr(p)))
        return p

    def forward(self, x, y, bf16=False, stream=None):
        s = None if stream is None else ctypes.c_void_p(int(stream))
        _check(None, load().hsc_mlp_forward(self.h, int(x.shape[0]), _ptr(x), _ptr(y),
                                            1 if bf16 else 0, s))

    def loss_grad(self, x, t, want_grad=False, stream=None):
        s = None if stream is None else ctypes.c_void_p(int(stream))
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32) if want_grad else None
        _check(None, load().hsc_mlp_loss_grad(self.h, int(x.shape[0]), _ptr(x), _ptr(t), _ptr(loss),
                                              _ptr(g), s))
        return (float(loss[0]), g) if want_grad else float(loss[0])

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        s = None if stream is None else ctypes.c_void_p(int(stream))
        _check(None, load().hsc_mlp_adam(self.h, lr, beta1, beta2, eps, s))

    def close(self):
        if self.h:
            load().hsc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hsc_last_error(h=None):
    return load().hsc_last_error(h).decode(errors="replace")


def hsc_destroy(h):
    if h is not None:
        load().hsc_destroy(h)


class Solver:
    """Convenience owner of one handle for a workloads.Device (create + analyze)."""

    def __init__(self, dev, leaf_max, geometric=True, ordering=None):
        self.dev = dev
        self.h = hsc_create(dev.n, dev.orb, dev.rowptr, dev.col, dev.val, dev.contact_ptr,
                            dev.contact_sites, dev.dims if geometric else None)
        if ordering is not None:
            hsc_set_option(self.h, HSC_OPT_ORDERING, ordering)
        self.stats = hsc_analyze(self.h, leaf_max)

    def solve(self, E, eta, sigma_r, sigma_less=None, precision=HSC_FP64, pairs=None):
        """Host-memory solve; returns (diag_gr, diag_gl, req_gr, req_gl) as numpy arrays."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        n_E, n = len(E), self.dev.n
        sigma_r = np.ascontiguousarray(sigma_r, dtype=np.complex128)
        if sigma_less is not None:
            sigma_less = np.ascontiguousarray(sigma_less, dtype=np.complex128)
        n_req = 0 if pairs is None else len(pairs)
        dgr = np.zeros((n_E, n), dtype=np.complex128)
        dgl = np.zeros((n_E, n), dtype=np.complex128) if sigma_less is not None else None
        rgr = np.zeros((n_E, n_req), dtype=np.complex128) if n_req else None
        rgl = np.zeros((n_E, n_req), dtype=np.complex128) if (n_req and sigma_less is not None) else None
        hsc_solve(self.h, E, eta, sigma_r, sigma_less, precision, pairs, dgr, dgl, rgr, rgl)
        return dgr, dgl, rgr, rgl

    def close(self):
        hsc_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass
