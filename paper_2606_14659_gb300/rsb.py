"""Python binding of librsb (include/rsb.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts tensors and
arrays to the C structs and back.  PyTorch is used for device memory and the
current stream.  If librsb.so has not been built the calls raise; there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librsb.so")

RSB_OK, RSB_EINVAL, RSB_ENOMEM, RSB_ECUDA, RSB_ENOCONV, RSB_ETIMEOUT, RSB_EDISCONNECTED = range(7)
RSB_LANCZOS, RSB_INVERSE, RSB_RCB = 0, 1, 2
RSB_FP64, RSB_MIXED = 0, 1
RSB_DEGEN_NONE, RSB_DEGEN_RESOLVE = 0, 1

EXPORTED = ["rsb_options_default", "rsb_partition", "rsb_partition_batch", "rsb_fiedler",
            "rsb_laplacian_apply", "rsb_laplacian_apply_f32", "rsb_laplacian_bench",
            "rsb_strerror", "rsb_last_error_detail", "rsb_release", "rsb_profile_begin",
            "rsb_profile_end", "rsb_laplacian_apply_noalloc", "rsb_autotune",
            "rsb_test_poison_barrier", "rsb_profile_read", "rsb_dual_graph",
            "rsb_laplacian_apply_gs", "rsb_laplacian_apply_gs_f32", "rsb_laplacian_bench_gs"]

RSB_TUNE_CANDIDATES = 6
TUNE_CANDIDATES = [(2, 3), (4, 3), (8, 3), (2, 1), (4, 1), (8, 1)]  # (tile_rows, use_graph)


class rsb_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("weight", C.c_void_p), ("gid", C.c_void_p), ("coords", C.c_void_p)]


class rsb_options(C.Structure):
    _fields_ = [("method", C.c_int), ("precision", C.c_int), ("krylov_dim", C.c_int),
                ("max_restarts", C.c_int), ("tol", C.c_double), ("cg_tol", C.c_double),
                ("cg_maxit", C.c_int), ("max_outer", C.c_int), ("seed", C.c_uint64),
                ("degenerate_policy", C.c_int), ("cluster_tol", C.c_double),
                ("tie_rel", C.c_double), ("mixed_tol", C.c_double), ("batched", C.c_int),
                ("use_graph", C.c_int), ("validate", C.c_int), ("polish_cycles", C.c_int),
                ("keep", C.c_int), ("tile_rows", C.c_int), ("polish_dim", C.c_int),
                ("block", C.c_int), ("reorder", C.c_int), ("amg", C.c_int)]


class rsb_stats(C.Structure):
    _fields_ = [("levels", C.c_int), ("nonconverged", C.c_int), ("solves", C.c_int64),
                ("cycles", C.c_int64), ("inner", C.c_int64), ("elements_bisected", C.c_int64),
                ("lambda_first", C.c_double), ("resid_max", C.c_double),
                ("seconds", C.c_double), ("kernel_launches", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load():
    """Loads librsb.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librsb.so not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.rsb_options_default.argtypes = [C.POINTER(rsb_options)]
    lib.rsb_options_default.restype = None
    lib.rsb_partition.argtypes = [C.POINTER(rsb_csr), C.c_int32, C.POINTER(rsb_options), vp,
                                  C.POINTER(rsb_stats), vp]
    lib.rsb_partition_batch.argtypes = [C.POINTER(rsb_csr), C.c_int32, C.POINTER(C.c_int32),
                                        C.POINTER(rsb_options), C.POINTER(vp),
                                        C.POINTER(rsb_stats), vp]
    lib.rsb_fiedler.argtypes = [C.POINTER(rsb_csr), C.POINTER(rsb_options),
                                C.POINTER(C.c_double), vp, C.POINTER(C.c_double), vp]
    lib.rsb_laplacian_apply.argtypes = [C.POINTER(rsb_csr), vp, vp, vp]
    lib.rsb_laplacian_apply_f32.argtypes = [C.POINTER(rsb_csr), vp, vp, vp]
    lib.rsb_laplacian_apply_noalloc.argtypes = [C.POINTER(rsb_csr), vp, vp, vp]
    lib.rsb_laplacian_bench.argtypes = [C.POINTER(rsb_csr), C.c_int, C.c_int,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.rsb_autotune.argtypes = [C.POINTER(rsb_csr), C.c_int32, C.POINTER(C.c_int32),
                                 C.POINTER(rsb_options), C.POINTER(vp), C.POINTER(C.c_double), vp]
    lib.rsb_dual_graph.argtypes = [C.c_int64, C.c_int, vp, vp, vp, vp, C.c_int64,
                                   C.POINTER(C.c_int64), vp]
    lib.rsb_laplacian_apply_gs.argtypes = [C.c_int64, C.c_int, vp, vp, vp, vp]
    lib.rsb_laplacian_apply_gs_f32.argtypes = [C.c_int64, C.c_int, vp, vp, vp, vp]
    lib.rsb_laplacian_bench_gs.argtypes = [C.c_int64, C.c_int, vp, C.c_int, C.c_int,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.rsb_test_poison_barrier.argtypes = [C.c_int]
    lib.rsb_test_poison_barrier.restype = None
    lib.rsb_strerror.argtypes = [C.c_int]
    lib.rsb_strerror.restype = C.c_char_p
    lib.rsb_last_error_detail.argtypes = []
    lib.rsb_last_error_detail.restype = C.c_char_p
    lib.rsb_release.argtypes = []
    lib.rsb_release.restype = None
    lib.rsb_profile_begin.argtypes = [C.c_int]
    lib.rsb_profile_begin.restype = None
    lib.rsb_profile_end.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double)]
    lib.rsb_profile_end.restype = None
    lib.rsb_profile_read.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double)]
    lib.rsb_profile_read.restype = None
    for name in ("rsb_partition", "rsb_partition_batch", "rsb_fiedler", "rsb_autotune",
                 "rsb_laplacian_apply",
                 "rsb_laplacian_apply_f32", "rsb_laplacian_bench", "rsb_laplacian_apply_noalloc",
                 "rsb_dual_graph", "rsb_laplacian_apply_gs", "rsb_laplacian_apply_gs_f32",
                 "rsb_laplacian_bench_gs"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class RSBError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        self.code = code
        msg = lib.rsb_strerror(code).decode()
        detail = lib.rsb_last_error_detail().decode()
        super().__init__(f"{where}: {msg} ({detail})" if detail else f"{where}: {msg}")


def _check(code: int, where: str, allow=(RSB_OK,)):
    if code not in allow:
        raise RSBError(code, where)
    return code


# ----------------------------------------------------------------------------
# graphs
# ----------------------------------------------------------------------------


@dataclass
class Graph:
    """A CSR graph whose arrays live on the device (torch) or the host (numpy)."""

    n: int
    row_ptr: object
    col: object
    weight: object
    gid: object
    device: str
    coords: object = None

    def c_struct(self) -> rsb_csr:
        return rsb_csr(self.n, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.weight),
                       _ptr(self.gid), _ptr(self.coords))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def graph(g, device: str = "cuda", gid: bool = True, coords=None) -> Graph:
    """Wraps a meshgen.DualGraph (or anything with n/row_ptr/col/w/gid) for the ABI.

    device="cuda": arrays are copied to the current GPU as torch tensors;
    device="host": numpy arrays are passed and the library copies them itself.
    coords: n x 3 element coordinates; by default the centroids of a box mesh
    when the graph has them.
    """
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = None if getattr(g, "w", None) is None else np.ascontiguousarray(g.w, dtype=np.int32)
    gd = np.ascontiguousarray(g.gid, dtype=np.int64) if gid and g.gid is not None else None
    if coords is None and hasattr(g, "centroids") and getattr(g, "dims", None) is not None:
        try:
            coords = g.centroids()
        except ValueError:
            coords = None
    xyz = None if coords is None else np.ascontiguousarray(coords, dtype=np.float64).reshape(-1)
    if device == "host":
        return Graph(int(g.n), rp, col, w, gd, "host", xyz)
    import torch

    def t(a):
        return None if a is None else torch.from_numpy(a).to(device)

    return Graph(int(g.n), t(rp), t(col), t(w), t(gd), device, t(xyz))


def options(**kw) -> rsb_options:
    """rsb_options with the library defaults, overridden by keyword."""
    o = rsb_options()
    load().rsb_options_default(C.byref(o))
    names = {"method": {"lanczos": RSB_LANCZOS, "inverse": RSB_INVERSE, "rcb": RSB_RCB},
             "precision": {"fp64": RSB_FP64, "mixed": RSB_MIXED},
             "degenerate_policy": {"none": RSB_DEGEN_NONE, "resolve": RSB_DEGEN_RESOLVE}}
    for k, v in kw.items():
        if k in names and isinstance(v, str):
            v = names[k][v]
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


# ----------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------


def rsb_partition(g: Graph, nparts: int, opts: rsb_options | None = None, out=None,
                  stream=None, allow_noconv: bool = True):
    """Part id per row.  Returns (parts, stats dict, status code)."""
    lib = load()
    if out is None:
        if g.device == "host":
            out = np.empty(g.n, dtype=np.int32)
        else:
            import torch

            out = torch.empty(g.n, dtype=torch.int32, device=g.device)
    cs = g.c_struct()
    st = rsb_stats()
    o = opts if opts is not None else options()
    code = lib.rsb_partition(C.byref(cs), int(nparts), C.byref(o), _ptr(out), C.byref(st),
                             _stream(stream))
    _check(code, "rsb_partition", (RSB_OK, RSB_ENOCONV) if allow_noconv else (RSB_OK,))
    return out, st.as_dict(), code


def rsb_partition_batch(gs: list, nparts: list, opts: rsb_options | None = None, outs=None,
                        stream=None, allow_noconv: bool = True):
    """rsb_partition over several meshes in one call.  Returns (parts list, stats, code)."""
    lib = load()
    m = len(gs)
    if outs is None:
        outs = []
        for g in gs:
            if g.device == "host":
                outs.append(np.empty(g.n, dtype=np.int32))
            else:
                import torch

                outs.append(torch.empty(g.n, dtype=torch.int32, device=g.device))
    arr = (rsb_csr * m)(*[g.c_struct() for g in gs])
    np_ = (C.c_int32 * m)(*[int(p) for p in nparts])
    ptrs = (C.c_void_p * m)(*[_ptr(o) for o in outs])
    st = rsb_stats()
    o = opts if opts is not None else options()
    code = lib.rsb_partition_batch(arr, m, np_, C.byref(o), ptrs, C.byref(st), _stream(stream))
    _check(code, "rsb_partition_batch", (RSB_OK, RSB_ENOCONV) if allow_noconv else (RSB_OK,))
    return outs, st.as_dict(), code


def rsb_autotune(gs: list, nparts: list, opts: rsb_options | None = None, outs=None,
                 stream=None):
    """Times the tile-rows x launch-mode candidates on one bisection level of the
    given meshes.  Returns (options with the chosen tile_rows and use_graph,
    {(tile_rows, use_graph): ms})."""
    lib = load()
    import torch

    m = len(gs)
    if outs is None:
        outs = [torch.empty(g.n, dtype=torch.int32, device=g.device) for g in gs]
    arr = (rsb_csr * m)(*[g.c_struct() for g in gs])
    np_ = (C.c_int32 * m)(*[int(p) for p in nparts])
    ptrs = (C.c_void_p * m)(*[_ptr(o) for o in outs])
    o = rsb_options()
    C.memmove(C.byref(o), C.byref(opts if opts is not None else options()), C.sizeof(o))
    ms = (C.c_double * RSB_TUNE_CANDIDATES)()
    code = lib.rsb_autotune(arr, m, np_, C.byref(o), ptrs, ms, _stream(stream))
    _check(code, "rsb_autotune")
    return o, {c: ms[i] for i, c in enumerate(TUNE_CANDIDATES)}


def rsb_fiedler(g: Graph, opts: rsb_options | None = None, out=None, stream=None):
    """(lambda2, v, residual, status code); v is oriented per the library's rule."""
    lib = load()
    if out is None:
        if g.device == "host":
            out = np.empty(g.n, dtype=np.float64)
        else:
            import torch

            out = torch.empty(g.n, dtype=torch.float64, device=g.device)
    cs = g.c_struct()
    lam = C.c_double(0.0)
    res = C.c_double(0.0)
    o = opts if opts is not None else options()
    code = lib.rsb_fiedler(C.byref(cs), C.byref(o), C.byref(lam), _ptr(out), C.byref(res),
                           _stream(stream))
    _check(code, "rsb_fiedler", (RSB_OK, RSB_ENOCONV, RSB_EDISCONNECTED))
    return lam.value, out, res.value, code


def rsb_laplacian_apply(g: Graph, x, y=None, stream=None):
    """y = L x in the precision of x (float64 or float32)."""
    lib = load()
    is_np = isinstance(x, np.ndarray)
    f32 = (x.dtype == np.float32) if is_np else (str(x.dtype) == "torch.float32")
    if y is None:
        if is_np:
            y = np.empty_like(x)
        else:
            import torch

            y = torch.empty_like(x)
    cs = g.c_struct()
    fn = lib.rsb_laplacian_apply_f32 if f32 else lib.rsb_laplacian_apply
    _check(fn(C.byref(cs), _ptr(x), _ptr(y), _stream(stream)), "rsb_laplacian_apply")
    return y


def rsb_laplacian_apply_noalloc(g: Graph, x, y, stream=None):
    """y = L x (FP64, device tensors) without any device allocation in the library."""
    lib = load()
    cs = g.c_struct()
    return lib.rsb_laplacian_apply_noalloc(C.byref(cs), _ptr(x), _ptr(y), _stream(stream))


def rsb_laplacian_bench(g: Graph, f32: bool, reps: int = 20, stream=None):
    """(mean ms per Laplacian launch, algorithmic bytes per launch)."""
    lib = load()
    cs = g.c_struct()
    ms = C.c_double(0.0)
    by = C.c_double(0.0)
    _check(lib.rsb_laplacian_bench(C.byref(cs), int(bool(f32)), int(reps), C.byref(ms),
                                   C.byref(by), _stream(stream)), "rsb_laplacian_bench")
    return ms.value, by.value


def rsb_dual_graph(ev, device: str = "cuda", stream=None):
    """Dual graph (n, row_ptr, col, weight) of elements given by their vertex
    ids ev (ne x nv integer array or tensor); arrays on `device` ("cuda" or
    "host")."""
    lib = load()
    import torch

    evt = ev if not isinstance(ev, np.ndarray) else torch.from_numpy(
        np.ascontiguousarray(ev, dtype=np.int64))
    if device != "host":
        evt = evt.to(device)
    ne, nv = int(evt.shape[0]), int(evt.shape[1])
    dev = "cpu" if device == "host" else device
    rp = torch.empty(ne + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(0)
    st = _stream(stream)
    _check(lib.rsb_dual_graph(ne, nv, _ptr(evt), _ptr(rp), None, None, 0, C.byref(nnz), st),
           "rsb_dual_graph")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    w = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    _check(lib.rsb_dual_graph(ne, nv, _ptr(evt), _ptr(rp), _ptr(col), _ptr(w), nnz.value,
                              C.byref(nnz), st), "rsb_dual_graph")
    return ne, rp, col[:nnz.value], w[:nnz.value]


def rsb_laplacian_apply_gs(ev, x, y=None, stream=None):
    """y = L x by gather-scatter from the element -> vertex ids (precision of x)."""
    lib = load()
    import torch

    f32 = str(x.dtype) == "torch.float32"
    if y is None:
        y = torch.empty_like(x)
    fn = lib.rsb_laplacian_apply_gs_f32 if f32 else lib.rsb_laplacian_apply_gs
    _check(fn(int(ev.shape[0]), int(ev.shape[1]), _ptr(ev), _ptr(x), _ptr(y), _stream(stream)),
           "rsb_laplacian_apply_gs")
    return y


def rsb_laplacian_bench_gs(ev, f32: bool, reps: int = 20, stream=None):
    """(mean ms per gather-scatter Laplacian, algorithmic bytes per application)."""
    lib = load()
    ms = C.c_double(0.0)
    by = C.c_double(0.0)
    _check(lib.rsb_laplacian_bench_gs(int(ev.shape[0]), int(ev.shape[1]), _ptr(ev),
                                      int(bool(f32)), int(reps), C.byref(ms), C.byref(by),
                                      _stream(stream)), "rsb_laplacian_bench_gs")
    return ms.value, by.value


def rsb_test_poison_barrier(on: bool):
    """Failure-path test hook: the persistent launch modes' grid barrier times out."""
    load().rsb_test_poison_barrier(1 if on else 0)


def rsb_release():
    load().rsb_release()


PROFILE_FAMILIES = {"lz_a": 1, "lz_b": 2, "lz_c": 3, "cg_ap": 4, "spmv": 5, "cycle": 6,
                    "lz_a2": 7, "amg": 8, "all": -1}


def rsb_profile_begin(family: str | int):
    """Times every launch of one kernel family in the following calls."""
    fam = PROFILE_FAMILIES[family] if isinstance(family, str) else int(family)
    load().rsb_profile_begin(fam)


def rsb_profile_end():
    """(total ms, launches, algorithmic bytes) of the profiled families."""
    ms = C.c_double(0.0)
    n = C.c_int64(0)
    by = C.c_double(0.0)
    load().rsb_profile_end(C.byref(ms), C.byref(n), C.byref(by))
    return ms.value, n.value, by.value


def rsb_profile_read(family: str | int):
    """(ms, launches, algorithmic bytes) of one family of the last profiled interval."""
    fam = PROFILE_FAMILIES[family] if isinstance(family, str) else int(family)
    ms = C.c_double(0.0)
    n = C.c_int64(0)
    by = C.c_double(0.0)
    load().rsb_profile_read(fam, C.byref(ms), C.byref(n), C.byref(by))
    return ms.value, n.value, by.value
