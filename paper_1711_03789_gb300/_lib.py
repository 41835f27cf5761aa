"""ctypes declarations of include/mxas.h and argument marshalling."""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_PKG, "libmxas.so")
if not os.path.exists(lib_path):
    raise ImportError(f"{lib_path} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")
lib = C.CDLL(lib_path)

MX_OK, MX_EINVAL, MX_ENOMEM, MX_ENOTFACTORED = 0, -1, -2, -3
MX_ESINGULAR, MX_ENOCONV, MX_ETIMEOUT, MX_ECUDA = -4, -5, -6, -7
MX_PLAIN_FP64, MX_MIXED = 0, 1
_NAMES = {0: "MX_OK", -1: "MX_EINVAL", -2: "MX_ENOMEM", -3: "MX_ENOTFACTORED", -4: "MX_ESINGULAR",
          -5: "MX_ENOCONV", -6: "MX_ETIMEOUT", -7: "MX_ECUDA"}


class MxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("n_cells", C.c_int), ("boundary", C.c_int)]


class DdDesc(C.Structure):
    _fields_ = [("core_cells", C.c_int), ("overlap_cells", C.c_int)]


class CoarseDesc(C.Structure):
    _fields_ = [("n_cells", C.c_int)]


class ProblemInfo(C.Structure):
    _fields_ = [("n_dof", C.c_int64), ("nnz", C.c_int64), ("n_sub", C.c_int32), ("max_local", C.c_int32),
                ("sum_local", C.c_int64), ("n_coarse", C.c_int64), ("nnz_r0", C.c_int64),
                ("factor_bytes", C.c_int64), ("coarse_band", C.c_int32), ("precision", C.c_int32),
                ("growth_subdomain", C.c_int32), ("max_growth", C.c_double)]


class RhsStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("rel_estimate", C.c_double)]


class Timing(C.Structure):
    _fields_ = [("build_ms", C.c_double), ("factor_ms", C.c_double), ("solve_ms", C.c_double),
                ("solve_launches", C.c_int64), ("restarts", C.c_int32), ("max_iterations", C.c_int32),
                ("coarse_inner_iterations", C.c_int64), ("coarse_inner_solves", C.c_int64)]


H = C.c_void_p
P = C.c_void_p
_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_sig = {
    "mx_version": (C.c_char_p, []),
    "mx_last_error": (C.c_char_p, []),
    "mx_set_allocator": (C.c_int, [_ALLOC, _FREE, C.c_void_p]),
    "mx_set_dense_local": (C.c_int, [H, C.c_int]),
    "mx_set_growth_limit": (C.c_int, [H, C.c_double]),
    "mx_test_bounded_wait": (C.c_int, [H, C.c_int, C.c_int]),
    "mx_set_tuning": (C.c_int, [H, C.c_int, C.c_int]),
    "mx_set_preconditioner": (C.c_int, [H, C.c_int]),
    "mx_set_weighted_gmres": (C.c_int, [H, C.c_int]),
    "mx_set_coarse_solver": (C.c_int, [H, C.c_int, C.POINTER(DdDesc), C.c_double, C.c_int, C.c_int]),
    "mx_build_problem": (C.c_int, [C.POINTER(MeshDesc), C.c_double, C.c_double, C.c_double, C.POINTER(DdDesc),
                                   C.POINTER(CoarseDesc), C.c_int, C.POINTER(H)]),
    "mx_set_xi_prob": (C.c_int, [H, C.c_double]),
    "mx_set_stream": (C.c_int, [H, C.c_void_p]),
    "mx_factor": (C.c_int, [H]),
    "mx_load_vector": (C.c_int, [H, C.c_int, C.c_int, P, P, C.c_double, P]),
    "mx_solve": (C.c_int, [H, P, C.c_int, C.c_double, C.c_int, C.c_int, P, C.POINTER(RhsStats)]),
    "mx_num_dofs": (C.c_int64, [H]),
    "mx_info": (C.c_int, [H, C.POINTER(ProblemInfo)]),
    "mx_timings": (C.c_int, [H, C.POINTER(Timing)]),
    "mx_destroy": (None, [H]),
    "mx_get_mesh": (C.c_int, [H, P, P]),
    "mx_get_subdomains": (C.c_int, [H, P, P, P, P]),
    "mx_get_csr": (C.c_int, [H, C.c_int, P, P, P, P]),
    "mx_get_boundary_mass": (C.c_int, [H, C.c_int, P]),
    "mx_get_coarse_restriction": (C.c_int, [H, P, P, P]),
    "mx_spmv": (C.c_int, [H, P, P, C.c_int]),
    "mx_spmv_mixed": (C.c_int, [H, P, P, C.c_int]),
    "mx_precond": (C.c_int, [H, P, P, C.c_int, C.c_int]),
    "mx_get_local": (C.c_int, [H, C.c_int, P]),
    "mx_dots": (C.c_int, [P, P, C.c_int64, C.c_int, C.c_int, P, C.c_void_p]),
    "mx_dots_noalloc": (C.c_int, [P, P, C.c_int64, C.c_int, C.c_int, P, C.c_void_p]),
    "mx_launch_count": (C.c_int64, []),
    "mx_profile": (C.c_int, [C.c_int]),
    "mx_profile_read": (C.c_int, [P, P, P, P]),
    "mx_profile_name": (C.c_char_p, [C.c_int]),
}
for _n, (_r, _a) in _sig.items():
    _f = getattr(lib, _n)
    _f.restype = _r
    _f.argtypes = _a


def _check(rc, allow=()):
    if rc != MX_OK and rc not in allow:
        raise MxError(rc, lib.mx_last_error().decode())
    return rc


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "array must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _nrhs(a, n):
    shape = tuple(a.shape)
    if len(shape) == 1:
        assert shape[0] == n
        return 1
    assert len(shape) == 2 and shape[1] == n, f"expected [nrhs, {n}], got {shape}"
    return shape[0]


def mx_version():
    return lib.mx_version().decode()


def mx_last_error():
    return lib.mx_last_error().decode()


MX_BC_PEC, MX_BC_IMPEDANCE = 0, 1


def mx_build_problem(n_cells, k, xi_prob, xi_prec, core_cells=5, overlap_cells=1, coarse_cells=0,
                     precision=MX_MIXED, bc=MX_BC_PEC):
    h = H()
    _check(lib.mx_build_problem(C.byref(MeshDesc(n_cells, bc)), k, xi_prob, xi_prec,
                                C.byref(DdDesc(core_cells, overlap_cells)), C.byref(CoarseDesc(coarse_cells)),
                                precision, C.byref(h)))
    return h


def mx_set_xi_prob(h, xi_prob):
    _check(lib.mx_set_xi_prob(h, xi_prob))


def mx_set_stream(h, stream):
    """stream: a cudaStream_t value (int), e.g. torch.cuda.current_stream().cuda_stream."""
    _check(lib.mx_set_stream(h, C.c_void_p(int(stream))))


def mx_set_dense_local(h, dense):
    _check(lib.mx_set_dense_local(h, int(bool(dense))))


MX_TUNE_LOCAL_RHS_GROUP = 1
MX_TUNE_LU_TENSOR = 2
MX_TUNE_COARSE_BLOCKS = 3
MX_TUNE_LOCAL_TENSOR = 4
MX_TUNE_COARSE_INVERSE = 5
MX_TUNE_LU_GRID = 6
MX_TUNE_DOTS = 7


def mx_set_tuning(h, key, value):
    _check(lib.mx_set_tuning(h, int(key), int(value)))


def mx_set_growth_limit(h, limit):
    """Pivot-growth limit checked by mx_factor (<= 0: the default for the precision)."""
    _check(lib.mx_set_growth_limit(h, float(limit)))


def mx_test_bounded_wait(h, limit=1024, blocks=4):
    """Failure-path probe: bounded waits on an mbarrier nothing arrives on; returns the
    library's code (MX_ETIMEOUT expected) without raising."""
    return lib.mx_test_bounded_wait(h, int(limit), int(blocks))


MX_PREC_AS, MX_PREC_RAS, MX_PREC_HRAS, MX_PREC_ADEF1 = 0, 1, 2, 3


def mx_set_preconditioner(h, kind):
    _check(lib.mx_set_preconditioner(h, int(kind)))


def mx_set_weighted_gmres(h, weighted):
    _check(lib.mx_set_weighted_gmres(h, int(bool(weighted))))


MX_COARSE_DIRECT, MX_COARSE_GMRES = 0, 1


def mx_set_coarse_solver(h, kind, core_cells=1, overlap_cells=1, tol=0.1, max_it=100, prec_kind=MX_PREC_RAS):
    dd = DdDesc(int(core_cells), int(overlap_cells))
    _check(lib.mx_set_coarse_solver(h, int(kind), C.byref(dd), float(tol), int(max_it), int(prec_kind)))


def mx_factor(h):
    _check(lib.mx_factor(h))


def mx_load_vector(h, centres, pol, width, out=None):
    """centres [nrhs, nbumps, 3] float64, pol [nrhs, nbumps, 3] complex128 (host numpy);
    out: [nrhs, n] complex128 (numpy or torch, host or CUDA); returns out."""
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    pol = np.ascontiguousarray(pol, dtype=np.complex128)
    nrhs, nb = centres.shape[0], centres.shape[1]
    n = mx_num_dofs(h)
    if out is None:
        out = np.empty((nrhs, n), dtype=np.complex128)
    _check(lib.mx_load_vector(h, nrhs, nb, _ptr(centres), _ptr(pol), float(width), _ptr(out)))
    return out


def mx_solve(h, rhs, tol=1e-6, restart=0, max_it=200, x=None):
    """Returns (x, stats list of dicts, rc); rc is MX_OK or MX_ENOCONV."""
    n = mx_num_dofs(h)
    nrhs = _nrhs(rhs, n)
    if x is None:
        x = np.empty_like(rhs) if isinstance(rhs, np.ndarray) else rhs.new_empty(rhs.shape)
    st = (RhsStats * nrhs)()
    rc = _check(lib.mx_solve(h, _ptr(rhs), nrhs, float(tol), int(restart), int(max_it), _ptr(x), st),
                allow=(MX_ENOCONV,))
    stats = [dict(iterations=s.iterations, converged=bool(s.converged), rel_residual=s.rel_residual,
                  rel_estimate=s.rel_estimate) for s in st]
    return x, stats, rc


def mx_num_dofs(h):
    return int(lib.mx_num_dofs(h))


def mx_info(h):
    i = ProblemInfo()
    _check(lib.mx_info(h, C.byref(i)))
    return {f: getattr(i, f) for f, _ in ProblemInfo._fields_}


def mx_timings(h):
    t = Timing()
    _check(lib.mx_timings(h, C.byref(t)))
    return {f: getattr(t, f) for f, _ in Timing._fields_}


def mx_destroy(h):
    lib.mx_destroy(h)


def mx_get_mesh(h, n_cells):
    n = mx_num_dofs(h)
    key = np.empty(n, dtype=np.int32)
    t2d = np.empty((6 * n_cells ** 3, 6), dtype=np.int32)
    _check(lib.mx_get_mesh(h, _ptr(key), _ptr(t2d)))
    return key, t2d


def mx_get_subdomains(h):
    info = mx_info(h)
    n, ns, sl = info["n_dof"], info["n_sub"], info["sum_local"]
    off = np.empty(ns + 1, dtype=np.int64)
    lists = np.empty(sl, dtype=np.int32)
    iptr = np.empty(n + 1, dtype=np.int32)
    ipos = np.empty(sl, dtype=np.int32)
    _check(lib.mx_get_subdomains(h, _ptr(off), _ptr(lists), _ptr(iptr), _ptr(ipos)))
    return off, lists, iptr, ipos


def mx_get_csr(h, which=0):
    info = mx_info(h)
    rows = info["n_dof"] if which == 0 else info["n_coarse"]
    rowptr = np.empty(rows + 1, dtype=np.int32)
    _check(lib.mx_get_csr(h, which, _ptr(rowptr), None, None, None))
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    K = np.empty(nnz)
    M = np.empty(nnz)
    _check(lib.mx_get_csr(h, which, None, _ptr(col), _ptr(K), _ptr(M)))
    return rowptr, col, K, M


def mx_get_boundary_mass(h, which=0):
    """B values on the pattern of mx_get_csr(h, which) (zeros with PEC)."""
    rowptr = mx_get_csr(h, which)[0]
    B = np.empty(int(rowptr[-1]))
    _check(lib.mx_get_boundary_mass(h, which, _ptr(B)))
    return B


def mx_get_coarse_restriction(h):
    info = mx_info(h)
    rowptr = np.empty(info["n_coarse"] + 1, dtype=np.int32)
    _check(lib.mx_get_coarse_restriction(h, _ptr(rowptr), None, None))
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz)
    _check(lib.mx_get_coarse_restriction(h, None, _ptr(col), _ptr(val)))
    return rowptr, col, val


def mx_spmv(h, x, y=None):
    n = mx_num_dofs(h)
    nrhs = _nrhs(x, n)
    if y is None:
        y = np.empty_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
    _check(lib.mx_spmv(h, _ptr(x), _ptr(y), nrhs))
    return y


def mx_spmv_mixed(h, x, y=None):
    """y = A x as the mixed form's Krylov process computes it (c64 x, double-float sums)."""
    n = mx_num_dofs(h)
    nrhs = _nrhs(x, n)
    if y is None:
        y = np.empty_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
    _check(lib.mx_spmv_mixed(h, _ptr(x), _ptr(y), nrhs))
    return y


def mx_precond(h, v, z=None, levels=3):
    n = mx_num_dofs(h)
    nrhs = _nrhs(v, n)
    if z is None:
        z = np.empty_like(v) if isinstance(v, np.ndarray) else v.new_empty(v.shape)
    _check(lib.mx_precond(h, _ptr(v), _ptr(z), nrhs, int(levels)))
    return z


def mx_get_local(h, l, n_l):
    out = np.empty((n_l, n_l), dtype=np.complex128)  # column-major content
    _check(lib.mx_get_local(h, int(l), _ptr(out)))
    return out.T.copy()  # row-major [i, j]


def mx_dots(V, w, h=None, stream=0):
    """h[i, r] = sum_x conj(V[i, x, r]) w[x, r]; V [nvec, n, nrhs], w [n, nrhs] complex128 CUDA
    tensors; h [nvec, nrhs] (numpy or torch, host or CUDA; numpy by default)."""
    nvec, n, nrhs = V.shape
    assert tuple(w.shape) == (n, nrhs)
    if h is None:
        h = np.empty((nvec, nrhs), dtype=np.complex128)
    _check(lib.mx_dots(_ptr(V), _ptr(w), n, nrhs, nvec, _ptr(h), C.c_void_p(int(stream))))
    return h


def mx_dots_noalloc(V, w, h=None, stream=0):
    """mx_dots without any device allocation (block partials in the library's fixed 4 MiB
    device array); for callers that cannot allocate. Requires nvec * nrhs <= 16384."""
    nvec, n, nrhs = V.shape
    assert tuple(w.shape) == (n, nrhs)
    if h is None:
        h = np.empty((nvec, nrhs), dtype=np.complex128)
    _check(lib.mx_dots_noalloc(_ptr(V), _ptr(w), n, nrhs, nvec, _ptr(h), C.c_void_p(int(stream))))
    return h


def mx_launch_count():
    return int(lib.mx_launch_count())


def mx_profile(enable):
    _check(lib.mx_profile(int(bool(enable))))


def mx_profile_name(i):
    return lib.mx_profile_name(int(i)).decode()


def mx_profile_read():
    """{kernel name: dict(ms, launches, bytes, flops)} accumulated since mx_profile(1)."""
    n = 64
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    by = np.zeros(n)
    fl = np.zeros(n)
    k = lib.mx_profile_read(_ptr(ms), _ptr(cnt), _ptr(by), _ptr(fl))
    if k < 0:
        _check(k)
    return {mx_profile_name(i): dict(ms=float(ms[i]), launches=int(cnt[i]), bytes=float(by[i]), flops=float(fl[i]))
            for i in range(k)}


_keep = []


def mx_set_allocator(alloc, release, ctx=None):
    """alloc(bytes) -> int pointer, release(int pointer) -> None; None restores cudaMalloc."""
    if alloc is None:
        _check(lib.mx_set_allocator(_ALLOC(), _FREE(), None))
        return
    a = _ALLOC(lambda nbytes, _ctx: alloc(nbytes))
    f = _FREE(lambda p, _ctx: release(p))
    _keep.append((a, f))
    _check(lib.mx_set_allocator(a, f, ctx))


def use_torch_allocator(device=0):
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    def alloc(nbytes):
        return torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), device)

    def release(p):
        torch.cuda.caching_allocator_delete(p)

    mx_set_allocator(alloc, release)


# ---- serving ---------------------------------------------------------------------------
class MxRequest(C.Structure):
    _fields_ = [("n_cells", C.c_int), ("k", C.c_double), ("xi_prob", C.c_double), ("xi_prec", C.c_double),
                ("core_cells", C.c_int), ("overlap_cells", C.c_int), ("coarse_cells", C.c_int),
                ("precision", C.c_int), ("nrhs", C.c_int), ("nbumps", C.c_int), ("centres", C.c_void_p),
                ("pol", C.c_void_p), ("width", C.c_double), ("tol", C.c_double), ("restart", C.c_int),
                ("max_it", C.c_int), ("boundary", C.c_int), ("prec_kind", C.c_int)]


class RequestTiming(C.Structure):
    _fields_ = [("latency_ms", C.c_double), ("queue_ms", C.c_double), ("n_dof", C.c_int64)]


class ServerInfo(C.Structure):
    _fields_ = [("batches", C.c_int64), ("factorisations", C.c_int64), ("evictions", C.c_int64),
                ("completed", C.c_int64), ("cached_bytes", C.c_int64), ("cached_operators", C.c_int32),
                ("pending", C.c_int32), ("joined", C.c_int64), ("waiting_for_memory", C.c_int32)]


MX_PENDING = 1
for _n, (_r, _a) in {
    "mx_server_create": (C.c_int, [C.c_int64, C.c_int, C.POINTER(C.c_void_p)]),
    "mx_server_submit": (C.c_int, [C.c_void_p, C.POINTER(MxRequest), C.POINTER(C.c_int64)]),
    "mx_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, P, C.POINTER(RhsStats), C.POINTER(RequestTiming)]),
    "mx_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerInfo)]),
    "mx_server_destroy": (None, [C.c_void_p]),
}.items():
    _f = getattr(lib, _n)
    _f.restype = _r
    _f.argtypes = _a


def mx_server_create(budget_bytes, workers=2):
    s = C.c_void_p()
    _check(lib.mx_server_create(int(budget_bytes), int(workers), C.byref(s)))
    return s


def mx_server_submit(s, n_cells, k, xi_prob, xi_prec, centres, pol, width=0.1, core_cells=5, overlap_cells=1,
                     coarse_cells=0, precision=MX_MIXED, tol=1e-6, restart=0, max_it=200, bc=MX_BC_PEC,
                     prec_kind=MX_PREC_AS):
    """Queue one request (centres [nrhs, nbumps, 3], pol [nrhs, nbumps, 3] complex); returns its ticket."""
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    pol = np.ascontiguousarray(pol, dtype=np.complex128)
    q = MxRequest(n_cells, k, xi_prob, xi_prec, core_cells, overlap_cells, coarse_cells, precision,
                  centres.shape[0], centres.shape[1], centres.ctypes.data, pol.ctypes.data, width, tol, restart,
                  max_it, int(bc), int(prec_kind))
    t = C.c_int64()
    _check(lib.mx_server_submit(s, C.byref(q), C.byref(t)))
    return t.value


def mx_server_poll(s, ticket, n_dof, nrhs, wait=True):
    """Returns None while pending (wait=False), else (x [nrhs, n_dof], stats, timing dict, rc)."""
    x = np.empty((nrhs, n_dof), dtype=np.complex128)
    st = (RhsStats * nrhs)()
    tm = RequestTiming()
    rc = lib.mx_server_poll(s, int(ticket), int(bool(wait)), _ptr(x), st, C.byref(tm))
    if rc == MX_PENDING and not wait:
        return None
    _check(rc, allow=(MX_ENOCONV,))
    stats = [dict(iterations=v.iterations, converged=bool(v.converged), rel_residual=v.rel_residual) for v in st]
    return x, stats, dict(latency_ms=tm.latency_ms, queue_ms=tm.queue_ms), rc


def mx_server_stats(s):
    i = ServerInfo()
    _check(lib.mx_server_stats(s, C.byref(i)))
    return {f: getattr(i, f) for f, _ in ServerInfo._fields_}


def mx_server_destroy(s):
    lib.mx_server_destroy(s)
