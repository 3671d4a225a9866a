"""Thin ctypes binding of libgmg.so (C ABI declared in include/gmg.h).

Argument marshalling only: every step of the smoother, the transfer, the
V-cycle and the CG runs in the library's CUDA kernels.  PyTorch provides
device memory (tensors) and the stream.  The binding never falls back to a
CPU path: if the library is missing or cannot be loaded, every call raises.

The functions carry the C names (gmg_create, gmg_smooth, ...); ``Problem``
is a small convenience wrapper around them.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmg.so")

GMG_OK = 0
GMG_FP64 = 0
GMG_FP32 = 1
GMG_FP32_TC = 2
GMG_FP32_TF32 = 3
STATUS = {0: "ok", -1: "invalid argument", -2: "device out of memory", -3: "CUDA error",
          -4: "non-finite value in solver", -5: "CG breakdown", -6: "not converged",
          -7: "unsupported", -8: "device wait timed out"}

EXPORTS = ["gmg_create", "gmg_destroy", "gmg_vector_layout", "gmg_level_info",
           "gmg_apply_operator", "gmg_apply_operator_f64", "gmg_smooth", "gmg_smooth_colour",
           "gmg_restrict", "gmg_prolongate_add", "gmg_coarse_solve", "gmg_vcycle",
           "cg_gmg_solve", "gmg_patch_fd_1d", "gmg_kernel_launch_count", "gmg_status_string",
           "gmg_smooth_noalloc", "gmg_smooth_variant", "gmg_batch_create", "gmg_batch_destroy",
           "gmg_batch_layout", "gmg_batch_problem", "gmg_batch_smooth", "gmg_batch_vcycle",
           "gmg_batch_cg_solve", "gmg_batch_autotune", "gmg_batch_set_ppc",
           "gmg_set_coefficient", "gmg_set_local_solver", "gmg_learned_train",
           "gmg_learned_corrections", "gmg_mlp_loss_grad", "gmg_tc_status", "gmg_tc_probe",
           "gmg_set_slab_width", "gmg_slab_width", "gmg_set_shared_faces", "gmg_shared_faces",
           "gmg_set_small_sweep", "gmg_small_sweep",
           "gmg_set_three_pass_operator", "gmg_three_pass_operator", "gmg_exact_patch_solve",
           "gmg_set_phase_timing", "gmg_fma_peak", "gmg_learned_levels", "gmg_learned_set_levels",
           "gmg_set_operator_tile", "gmg_autotune"]
PHASES = ("smooth", "operator", "transfer", "coarse", "vector")
GMG_LOCAL_FD_MEAN, GMG_LOCAL_LEARNED = 0, 1
GMG_SWEEP_COMBINED, GMG_SWEEP_SEPARATED, GMG_SWEEP_BATCHED = 0, 1, 2


class GmgDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("n_cells", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("precision", ctypes.c_int), ("damping", ctypes.c_double),
                ("pre_sweeps", ctypes.c_int), ("post_sweeps", ctypes.c_int), ("stream", ctypes.c_void_p)]


class GmgSolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("initial_residual", ctypes.c_double), ("final_residual", ctypes.c_double),
                ("relative_residual", ctypes.c_double), ("residual_history", ctypes.c_double * 64),
                ("phase_ms", ctypes.c_double * 5)]


class GmgTuning(ctypes.Structure):
    _fields_ = [("slab_width", ctypes.c_int), ("operator_tile", ctypes.c_int),
                ("sweep_ms", ctypes.c_double), ("sweep_ms_default", ctypes.c_double),
                ("operator_ms", ctypes.c_double), ("operator_ms_default", ctypes.c_double)]


class GmgError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


_LIB = None


def lib():
    """Load libgmg.so (built in-tree by paper_2407_02100_gb300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2407_02100_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "gmg_create": [ctypes.POINTER(GmgDesc), ctypes.POINTER(vp)],
            "gmg_destroy": [vp],
            "gmg_vector_layout": [vp, i, ctypes.POINTER(ll), ctypes.POINTER(i), ctypes.POINTER(i),
                                  ctypes.POINTER(ll)],
            "gmg_level_info": [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)],
            "gmg_apply_operator": [vp, i, vp, vp],
            "gmg_apply_operator_f64": [vp, i, vp, vp],
            "gmg_smooth": [vp, i, vp, vp, i, i],
            "gmg_smooth_colour": [vp, i, vp, vp, i],
            "gmg_smooth_variant": [vp, i, vp, vp, i, ll, i],
            "gmg_restrict": [vp, i, vp, vp],
            "gmg_prolongate_add": [vp, i, vp, vp],
            "gmg_coarse_solve": [vp, vp, vp],
            "gmg_vcycle": [vp, vp, vp],
            "cg_gmg_solve": [vp, vp, vp, d, i, ctypes.POINTER(GmgSolveStats)],
            "gmg_patch_fd_1d": [i, vp, vp, vp, vp],
            "gmg_kernel_launch_count": [],
            "gmg_batch_create": [ctypes.POINTER(GmgDesc), i, ctypes.POINTER(i), ctypes.POINTER(vp)],
            "gmg_batch_destroy": [vp],
            "gmg_batch_layout": [vp, i, ctypes.POINTER(ll), ctypes.POINTER(ll), ctypes.POINTER(ll)],
            "gmg_batch_problem": [vp, i, ctypes.POINTER(vp)],
            "gmg_batch_smooth": [vp, vp, vp, i],
            "gmg_batch_vcycle": [vp, vp, vp],
            "gmg_batch_cg_solve": [vp, vp, vp, d, i, ctypes.POINTER(i), ctypes.POINTER(d)],
            "gmg_batch_autotune": [vp, ctypes.POINTER(i)],
            "gmg_batch_set_ppc": [vp, i],
            "gmg_set_coefficient": [vp, vp],
            "gmg_set_local_solver": [vp, i],
            "gmg_learned_train": [vp, i, ctypes.POINTER(i), vp, i, i, d, ctypes.c_uint,
                                  ctypes.POINTER(d), ctypes.POINTER(i)],
            "gmg_learned_corrections": [vp, i, vp, ll],
            "gmg_mlp_loss_grad": [i, i, i, i, i, vp, vp, vp, vp, vp, ctypes.POINTER(d), vp],
            "gmg_exact_patch_solve": [i, i, i, vp, vp, vp, vp],
            "gmg_set_phase_timing": [vp, i],
            "gmg_fma_peak": [i, ctypes.POINTER(d)],
            "gmg_learned_levels": [vp],
            "gmg_learned_set_levels": [vp, i],
            "gmg_set_operator_tile": [vp, i],
            "gmg_autotune": [vp, ctypes.POINTER(GmgTuning)],
            "gmg_smooth_noalloc": [i, i, i, d, vp, vp, i, i, vp],
            "gmg_status_string": [i],
            "gmg_tc_status": [],
            "gmg_tc_probe": [vp, vp, vp, i],
            "gmg_set_slab_width": [vp, i],
            "gmg_slab_width": [vp, i],
            "gmg_set_shared_faces": [vp, i],
            "gmg_shared_faces": [vp],
            "gmg_set_small_sweep": [vp, i],
            "gmg_small_sweep": [vp],
            "gmg_set_three_pass_operator": [vp, i],
            "gmg_three_pass_operator": [vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = {"gmg_status_string": ctypes.c_char_p,
                         "gmg_kernel_launch_count": ctypes.c_longlong}.get(name, ctypes.c_int)
        _LIB = L
    return _LIB


def _check(fn, st):
    if st != GMG_OK:
        raise GmgError(fn, st)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# C names

def gmg_create(dim, degree, n_cells, n_levels=0, precision=GMG_FP64, damping=1.0,
               pre_sweeps=1, post_sweeps=1, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    desc = GmgDesc(dim, degree, n_cells, n_levels, precision, damping, pre_sweeps, post_sweeps,
                   ctypes.c_void_p(stream))
    h = ctypes.c_void_p()
    _check("gmg_create", lib().gmg_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def gmg_destroy(h):
    _check("gmg_destroy", lib().gmg_destroy(h))


def gmg_vector_layout(h, level):
    n, N, py, pz = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check("gmg_vector_layout", lib().gmg_vector_layout(h, level, ctypes.byref(n), ctypes.byref(N),
                                                          ctypes.byref(py), ctypes.byref(pz)))
    return n.value, N.value, py.value, pz.value


def gmg_level_info(h, level):
    n, L = ctypes.c_int(), ctypes.c_int()
    _check("gmg_level_info", lib().gmg_level_info(h, level, ctypes.byref(n), ctypes.byref(L)))
    return n.value, L.value


def gmg_apply_operator(h, level, x, y):
    _check("gmg_apply_operator", lib().gmg_apply_operator(h, level, _ptr(x), _ptr(y)))


def gmg_apply_operator_f64(h, level, x, y):
    _check("gmg_apply_operator_f64", lib().gmg_apply_operator_f64(h, level, _ptr(x), _ptr(y)))


def gmg_smooth(h, level, u, b, n_sweeps=1, reverse=False):
    _check("gmg_smooth", lib().gmg_smooth(h, level, _ptr(u), _ptr(b), n_sweeps, int(bool(reverse))))


def gmg_smooth_colour(h, level, u, b, colour):
    _check("gmg_smooth_colour", lib().gmg_smooth_colour(h, level, _ptr(u), _ptr(b), colour))


def gmg_smooth_variant(h, level, u, b, variant, batch_size=1, reverse=False):
    _check("gmg_smooth_variant", lib().gmg_smooth_variant(h, level, _ptr(u), _ptr(b), variant,
                                                          batch_size, int(bool(reverse))))


def gmg_restrict(h, fine_level, fine, coarse):
    _check("gmg_restrict", lib().gmg_restrict(h, fine_level, _ptr(fine), _ptr(coarse)))


def gmg_prolongate_add(h, coarse_level, coarse, fine):
    _check("gmg_prolongate_add", lib().gmg_prolongate_add(h, coarse_level, _ptr(coarse), _ptr(fine)))


def gmg_coarse_solve(h, b, x):
    _check("gmg_coarse_solve", lib().gmg_coarse_solve(h, _ptr(b), _ptr(x)))


def gmg_vcycle(h, x, b):
    _check("gmg_vcycle", lib().gmg_vcycle(h, _ptr(x), _ptr(b)))


def cg_gmg_solve(h, u, b, rtol=1e-10, max_it=100, raise_on_error=True):
    st = GmgSolveStats()
    status = lib().cg_gmg_solve(h, _ptr(u), _ptr(b), rtol, max_it, ctypes.byref(st))
    if raise_on_error:
        _check("cg_gmg_solve", status)
    return status, st


def gmg_fma_peak(precision):
    """Measured FMA peak of the current device in TFLOP/s (GMG_FP64 or GMG_FP32)."""
    out = ctypes.c_double()
    _check("gmg_fma_peak", lib().gmg_fma_peak(precision, ctypes.byref(out)))
    return out.value


def gmg_set_operator_tile(h, tile):
    _check("gmg_set_operator_tile", lib().gmg_set_operator_tile(h, tile))


def gmg_autotune(h):
    """Times and keeps the fastest slab width and operator tile shape;
    returns the GmgTuning record."""
    t = GmgTuning()
    _check("gmg_autotune", lib().gmg_autotune(h, ctypes.byref(t)))
    return t


def gmg_set_phase_timing(h, enable):
    _check("gmg_set_phase_timing", lib().gmg_set_phase_timing(h, 1 if enable else 0))


def phase_times(stats):
    """{phase name: GPU milliseconds} from a gmg_solve_stats."""
    return {name: stats.phase_ms[i] for i, name in enumerate(PHASES)}


def gmg_patch_fd_1d(degree):
    """Host-only: (M, K, T, lambda) of the two-unit-cell patch (numpy)."""
    m = 2 * degree - 1
    M, K, T = (np.zeros((m, m)) for _ in range(3))
    lam = np.zeros(m)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check("gmg_patch_fd_1d", lib().gmg_patch_fd_1d(degree, p(M), p(K), p(T), p(lam)))
    return M, K, T, lam


def gmg_smooth_noalloc(dim, degree, n_cells, u, b, n_sweeps=1, reverse=False, damping=1.0,
                       stream=None):
    """FP64 smoothing of one level without a problem object and without
    device allocation (for callers whose device memory belongs to another
    allocator); u, b: float64 CUDA tensors in the level layout."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check("gmg_smooth_noalloc", lib().gmg_smooth_noalloc(dim, degree, n_cells, damping, _ptr(u), _ptr(b),
                                                          n_sweeps, int(bool(reverse)),
                                                          ctypes.c_void_p(stream)))


def gmg_set_coefficient(h, coef):
    """coef: per-cell coefficients, numpy array of n^dim values (c_0 fastest
    in C order, i.e. shape (n,)*dim indexed [c_{dim-1}, ..., c_0])."""
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).ravel())
    _check("gmg_set_coefficient", lib().gmg_set_coefficient(h, c.ctypes.data_as(ctypes.c_void_p)))


def gmg_set_local_solver(h, solver):
    _check("gmg_set_local_solver", lib().gmg_set_local_solver(h, solver))


def gmg_learned_train(h, sample_vertices, residuals, steps=300, batch=1024, lr=3e-3, seed=0):
    """sample_vertices: host int array of patch ids over all levels, finest
    level first (see learned_patch_count); residuals: CUDA float64 tensor
    [n_samples, m^d].  Returns (loss history, kept patch count)."""
    verts = np.ascontiguousarray(np.asarray(sample_vertices, dtype=np.int32))
    hist = (ctypes.c_double * max(steps, 1))()
    kept = ctypes.c_int()
    _check("gmg_learned_train", lib().gmg_learned_train(
        h, len(verts), verts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(residuals), steps, batch,
        lr, seed, hist, ctypes.byref(kept)))
    return list(hist)[:steps], kept.value


def gmg_learned_levels(h):
    """Bit mask of the levels whose learned correction is in use."""
    mask = lib().gmg_learned_levels(h)
    if mask < 0:
        _check("gmg_learned_levels", mask)
    return mask


def gmg_learned_set_levels(h, mask):
    _check("gmg_learned_set_levels", lib().gmg_learned_set_levels(h, int(mask)))


def learned_patch_count(dim, n_cells, n_levels):
    """Number of patch ids gmg_learned_train accepts: the interior vertices
    of every level, finest level first."""
    return sum((n_cells // 2 ** l - 1) ** dim for l in range(n_levels))


def gmg_learned_corrections(h, level, n_patches, per_patch):
    out = np.zeros(n_patches * per_patch, dtype=np.float32)
    _check("gmg_learned_corrections", lib().gmg_learned_corrections(
        h, level, out.ctypes.data_as(ctypes.c_void_p), out.size))
    return out.reshape(n_patches, per_patch)


def gmg_mlp_loss_grad(dim, degree, rank, hidden, params, X, R, DFD, DEX):
    """All arrays CUDA tensors (params, X float32; R, DFD, DEX float64).
    Returns (loss, grads tensor)."""
    import torch
    grads = torch.zeros_like(params)
    loss = ctypes.c_double()
    _check("gmg_mlp_loss_grad", lib().gmg_mlp_loss_grad(
        dim, degree, rank, hidden, X.shape[0], _ptr(params), _ptr(X), _ptr(R), _ptr(DFD), _ptr(DEX),
        ctypes.byref(loss), _ptr(grads)))
    return loss.value, grads


def gmg_exact_patch_solve(dim, degree, w, r):
    """w: CUDA float64 [n, 2^dim] cell weights (geometric mean 1 per row), r:
    CUDA float64 [n, m^dim] residuals.  Returns (d_exact, d_fd) tensors."""
    import torch
    d_ex = torch.zeros_like(r)
    d_fd = torch.zeros_like(r)
    _check("gmg_exact_patch_solve", lib().gmg_exact_patch_solve(
        dim, degree, r.shape[0], _ptr(w), _ptr(r), _ptr(d_ex), _ptr(d_fd)))
    return d_ex, d_fd


def gmg_kernel_launch_count():
    return lib().gmg_kernel_launch_count()


def gmg_set_slab_width(h, width):
    _check("gmg_set_slab_width", lib().gmg_set_slab_width(h, width))


def gmg_slab_width(h, level):
    w = lib().gmg_slab_width(h, level)
    if w < 0:
        raise GmgError("gmg_slab_width", w)
    return w


def gmg_set_shared_faces(h, enable):
    _check("gmg_set_shared_faces", lib().gmg_set_shared_faces(h, 1 if enable else 0))


def gmg_set_small_sweep(h, max_patches):
    """FP64 colour steps of at most max_patches patches use the coarse-level
    kernel, one output per thread (0: never)."""
    _check("gmg_set_small_sweep", lib().gmg_set_small_sweep(h, int(max_patches)))


def gmg_small_sweep(h):
    v = lib().gmg_small_sweep(h)
    if v < 0:
        _check("gmg_small_sweep", v)
    return v


def gmg_shared_faces(h):
    """1 if whole-colour FP64 3D sweeps of the problem use the shared-face form."""
    r = lib().gmg_shared_faces(h)
    if r < 0:
        raise GmgError("gmg_shared_faces", r)
    return r


def gmg_set_three_pass_operator(h, enable):
    _check("gmg_set_three_pass_operator", lib().gmg_set_three_pass_operator(h, 1 if enable else 0))


def gmg_three_pass_operator(h):
    """1 if the FP64 operator of the problem runs as three passes (3D, k >= 3)."""
    r = lib().gmg_three_pass_operator(h)
    if r < 0:
        raise GmgError("gmg_three_pass_operator", r)
    return r


def gmg_tc_status():
    """Synchronise; the status recorded by the tensor-core sweep (cleared)."""
    return lib().gmg_tc_status()


def gmg_tc_probe(A, B, force_timeout=False, raise_on_error=True):
    """D = A B^T on the tensor cores (A 128x16, B 32x16 float32, host).
    With raise_on_error=False returns (status, D)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    assert A.shape == (128, 16) and B.shape == (32, 16)
    D = np.zeros((128, 32), dtype=np.float32)
    st = lib().gmg_tc_probe(A.ctypes.data_as(ctypes.c_void_p), B.ctypes.data_as(ctypes.c_void_p),
                            D.ctypes.data_as(ctypes.c_void_p), 1 if force_timeout else 0)
    if not raise_on_error:
        return st, D
    _check("gmg_tc_probe", st)
    return D


def gmg_status_string(status):
    return lib().gmg_status_string(status).decode()


# ---------------------------------------------------------------------------
# convenience wrapper

class Problem:
    """Owns one gmg_problem.  Vectors are torch CUDA tensors in the padded
    layout of include/gmg.h; to_device/from_device convert from/to the dense
    (n k + 1)^dim node arrays (x index fastest) used by the tests."""

    def __init__(self, dim, degree, n_cells, n_levels=0, precision=GMG_FP64, damping=1.0,
                 pre_sweeps=1, post_sweeps=1, stream=None, small_sweep=None):
        import torch
        self.torch = torch
        self.dim, self.degree, self.n_cells = dim, degree, n_cells
        self.precision = precision
        self.dtype = torch.float64 if precision == GMG_FP64 else torch.float32
        self.h = gmg_create(dim, degree, n_cells, n_levels, precision, damping, pre_sweeps,
                            post_sweeps, stream)
        self.n_levels = gmg_level_info(self.h, 0)[1]
        if small_sweep is not None:  # 0: no colour step takes the coarse-level kernel
            gmg_set_small_sweep(self.h, small_sweep)

    def close(self):
        if self.h is not None:
            gmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def finest(self):
        return self.n_levels - 1

    def layout(self, level=None):
        return gmg_vector_layout(self.h, self.finest if level is None else level)

    def zeros(self, level=None, dtype=None):
        n = self.layout(level)[0]
        return self.torch.zeros(n, dtype=dtype or self.dtype, device="cuda")

    def to_device(self, dense, level=None, dtype=None):
        """Dense node array (N^dim, x fastest) -> padded device vector."""
        n, N, py, pz = self.layout(level)
        t = self.torch
        dense = t.as_tensor(np.asarray(dense)).to(dtype or self.dtype)
        out = t.zeros(n, dtype=dtype or self.dtype)
        if self.dim == 2:
            out.view(N, py)[:, :N] = dense.view(N, N)
        else:
            out.view(N, N, py)[:, :, :N] = dense.view(N, N, N)
        return out.cuda()

    def from_device(self, vec, level=None):
        """Padded device vector -> dense float64 numpy node array."""
        n, N, py, pz = self.layout(level)
        v = vec.detach().to("cpu", self.torch.float64)
        if self.dim == 2:
            return v.view(N, py)[:, :N].reshape(-1).numpy().copy()
        return v.view(N, N, py)[:, :, :N].reshape(-1).numpy().copy()


# ---------------------------------------------------------------------------
# batches of independent problems

def gmg_batch_create(dim, degree, n_cells, precision=GMG_FP64, damping=1.0, pre_sweeps=1,
                     post_sweeps=1, stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    desc = GmgDesc(dim, degree, 0, 0, precision, damping, pre_sweeps, post_sweeps, ctypes.c_void_p(stream))
    arr = (ctypes.c_int * len(n_cells))(*[int(n) for n in n_cells])
    h = ctypes.c_void_p()
    _check("gmg_batch_create", lib().gmg_batch_create(ctypes.byref(desc), len(n_cells), arr, ctypes.byref(h)))
    return h


def gmg_batch_destroy(h):
    _check("gmg_batch_destroy", lib().gmg_batch_destroy(h))


def gmg_batch_layout(h, problem):
    o, n, t = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check("gmg_batch_layout", lib().gmg_batch_layout(h, problem, ctypes.byref(o), ctypes.byref(n), ctypes.byref(t)))
    return o.value, n.value, t.value


def gmg_batch_problem(h, problem):
    out = ctypes.c_void_p()
    _check("gmg_batch_problem", lib().gmg_batch_problem(h, problem, ctypes.byref(out)))
    return out


def gmg_batch_smooth(h, u, b, reverse=False):
    _check("gmg_batch_smooth", lib().gmg_batch_smooth(h, _ptr(u), _ptr(b), int(bool(reverse))))


def gmg_batch_vcycle(h, x, b):
    _check("gmg_batch_vcycle", lib().gmg_batch_vcycle(h, _ptr(x), _ptr(b)))


def gmg_batch_cg_solve(h, n_problems, u, b, rtol=1e-10, max_it=100, raise_on_error=True):
    its = (ctypes.c_int * n_problems)()
    res = (ctypes.c_double * n_problems)()
    st = lib().gmg_batch_cg_solve(h, _ptr(u), _ptr(b), rtol, max_it, its, res)
    if raise_on_error:
        _check("gmg_batch_cg_solve", st)
    return st, list(its), list(res)


def gmg_batch_autotune(h):
    out = ctypes.c_int()
    _check("gmg_batch_autotune", lib().gmg_batch_autotune(h, ctypes.byref(out)))
    return out.value


def gmg_batch_set_ppc(h, ppc):
    _check("gmg_batch_set_ppc", lib().gmg_batch_set_ppc(h, ppc))


class Batch:
    """Owns one gmg_batch; batch vectors are single CUDA tensors holding the
    padded finest-level vectors of all problems at their offsets."""

    def __init__(self, dim, degree, n_cells, precision=GMG_FP64, damping=1.0, stream=None):
        import torch
        self.torch = torch
        self.dim, self.degree, self.n_cells = dim, degree, list(n_cells)
        self.dtype = torch.float64 if precision == GMG_FP64 else torch.float32
        self.h = gmg_batch_create(dim, degree, self.n_cells, precision, damping, stream=stream)
        self.layouts = []
        for i in range(len(self.n_cells)):
            off, n, total = gmg_batch_layout(self.h, i)
            p = gmg_batch_problem(self.h, i)
            nl = gmg_level_info(p, 0)[1]
            self.layouts.append((off, n, gmg_vector_layout(p, nl - 1)))
        self.total = total

    def close(self):
        if self.h is not None:
            gmg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self, dtype=None):
        return self.torch.zeros(self.total, dtype=dtype or self.dtype, device="cuda")

    def pack(self, dense_list, dtype=None):
        """Dense per-problem node arrays -> one padded batch vector (device)."""
        t = self.torch
        out = t.zeros(self.total, dtype=dtype or self.dtype)
        for (off, n, (ne, N, py, pz)), dense in zip(self.layouts, dense_list):
            v = out[off:off + n]
            d = t.as_tensor(np.asarray(dense)).to(out.dtype)
            if self.dim == 2:
                v.view(N, py)[:, :N] = d.view(N, N)
            else:
                v.view(N, N, py)[:, :, :N] = d.view(N, N, N)
        return out.cuda()

    def unpack(self, vec):
        """Batch vector -> list of dense float64 numpy node arrays."""
        v = vec.detach().to("cpu", self.torch.float64)
        out = []
        for off, n, (ne, N, py, pz) in self.layouts:
            w = v[off:off + n]
            if self.dim == 2:
                out.append(w.view(N, py)[:, :N].reshape(-1).numpy().copy())
            else:
                out.append(w.view(N, N, py)[:, :, :N].reshape(-1).numpy().copy())
        return out
