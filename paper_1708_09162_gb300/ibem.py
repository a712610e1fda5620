"""ctypes binding of libibem (declared in include/ibem.h).

Argument marshalling only: every function below has the name of the C entry
point it calls, checks nothing beyond what ctypes needs, and raises
``IbemError`` (with the library's last-error text) when the call does not
return IBEM_OK.  Device buffers are passed as ``torch.Tensor`` objects (their
``data_ptr()`` is handed to the library); host buffers as numpy arrays.

Loading fails loudly: if libibem.so has not been built (see ``build.py``) the
import raises, and there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

IBEM_OK = 0
IBEM_ERR_NOCONV = 5
IBEM_PATCH_NURBS, IBEM_PATCH_SPHERE_FACE = 0, 1
IBEM_LAPLACE, IBEM_HELMHOLTZ = 0, 1
IBEM_FP64, IBEM_FP32, IBEM_BF16 = 0, 1, 2
IBEM_PRECOND_NONE, IBEM_PRECOND_JACOBI, IBEM_PRECOND_BLOCK_JACOBI, IBEM_PRECOND_LEARNED = 0, 1, 2, 3
IBEM_AUGMENT_PHASE, IBEM_AUGMENT_DIHEDRAL = 1, 2

EXPORTED = ("ibem_create", "ibem_destroy", "ibem_get_info", "ibem_assemble", "ibem_quad_points",
            "ibem_rhs", "ibem_matvec", "ibem_matvec_host", "ibem_solve", "ibem_potential",
            "ibem_block_tree", "ibem_last_error", "ibem_status_string", "ibem_profile_enable",
            "ibem_profile_read", "ibem_set_wait_limit", "ibem_device_status", "ibem_potential_noalloc",
            "ibem_potential_fmm",
            "ibem_batch_create", "ibem_batch_offsets", "ibem_batch_matvec", "ibem_batch_info", "ibem_batch_destroy",
            "ibem_batch_solve",
            "ibem_cnn_create", "ibem_cnn_destroy", "ibem_cnn_params", "ibem_cnn_forward", "ibem_cnn_gradients",
            "ibem_cnn_train_step", "ibem_cnn_train", "ibem_cnn_launches", "ibem_set_learned_preconditioner",
            "ibem_learned_apply", "ibem_solver_pairs", "ibem_solver_residuals", "ibem_cnn_operator_gradients",
            "ibem_cnn_train_operator", "ibem_cnn_device_status", "ibem_cnn_set_coarsening", "ibem_near_orders",
            "ibem_set_fp32_coupling", "ibem_rhs_sources")


class IbemError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status, message))
        self.status = status


class ibem_patch(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("deg_u", ctypes.c_int), ("deg_v", ctypes.c_int),
                ("ncp_u", ctypes.c_int), ("ncp_v", ctypes.c_int),
                ("knots_u", ctypes.POINTER(ctypes.c_double)), ("knots_v", ctypes.POINTER(ctypes.c_double)),
                ("ctrl_xyz", ctypes.POINTER(ctypes.c_double)), ("weights", ctypes.POINTER(ctypes.c_double)),
                ("face", ctypes.c_int), ("radius", ctypes.c_double), ("center", ctypes.c_double * 3),
                ("perturbed", ctypes.c_int)]


class ibem_params(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("kappa", ctypes.c_double), ("p", ctypes.c_int), ("m", ctypes.c_int),
                ("q_cheb", ctypes.c_int), ("eta", ctypes.c_double), ("gauss_regular", ctypes.c_int),
                ("gauss_singular", ctypes.c_int), ("fp64_coupling", ctypes.c_int), ("admissibility", ctypes.c_int),
                ("fp32_coupling", ctypes.c_int), ("gauss_grading", ctypes.c_int)]


class ibem_info(ctypes.Structure):
    _fields_ = [("ndof", ctypes.c_int64), ("ndof_super", ctypes.c_int64), ("n_elements", ctypes.c_int64),
                ("n_clusters", ctypes.c_int64), ("n_quad_points", ctypes.c_int64), ("n_near", ctypes.c_int64),
                ("n_far", ctypes.c_int64), ("n_near_singular", ctypes.c_int64 * 4),
                ("bytes_near", ctypes.c_int64), ("bytes_far", ctypes.c_int64), ("assembled", ctypes.c_int),
                ("max_gauss_order", ctypes.c_int), ("n_near_graded", ctypes.c_int64),
                ("stored_ring_depth", ctypes.c_int)]


class ibem_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("steps", ctypes.c_int)]


class ibem_profile_data(ctypes.Structure):
    _fields_ = [("applications", ctypes.c_int64), ("launches", ctypes.c_int64), ("ms", ctypes.c_double * 6)]


PHASES = ("lift", "upward", "coupling", "downward", "near", "restrict")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libibem.so is not built; run paper_1708_09162_gb300/build.py (no fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "ibem_create": (I32, [ctypes.POINTER(ibem_patch), I32, ctypes.POINTER(ibem_params), P, ctypes.POINTER(P)]),
        "ibem_destroy": (I32, [P]),
        "ibem_get_info": (I32, [P, ctypes.POINTER(ibem_info)]),
        "ibem_assemble": (I32, [P]),
        "ibem_quad_points": (I32, [P, P]),
        "ibem_rhs": (I32, [P, P, I32, P]),
        "ibem_matvec": (I32, [P, P, P, I32, I32]),
        "ibem_matvec_host": (I32, [P, P, P, I32, I32]),
        "ibem_solve": (I32, [P, P, P, I32, ctypes.c_double, I32, I32, I32, ctypes.POINTER(ibem_solve_info)]),
        "ibem_potential": (I32, [P, P, I32, P, I64, P]),
        "ibem_potential_noalloc": (I32, [P, P, I32, P, I64, P]),
        "ibem_potential_fmm": (I32, [P, P, I32, P, I64, P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "ibem_block_tree": (I32, [ctypes.POINTER(ibem_patch), I32, ctypes.POINTER(ibem_params),
                                  ctypes.POINTER(I64), P, ctypes.POINTER(I64), P]),
        "ibem_set_fp32_coupling": (I32, [P, I32]),
        "ibem_rhs_sources": (I32, [P, P, P, I32, I64, P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "ibem_near_orders": (I32, [ctypes.POINTER(ibem_patch), I32, ctypes.POINTER(ibem_params),
                                   ctypes.POINTER(I64), P]),
        "ibem_profile_enable": (I32, [P, I32]),
        "ibem_profile_read": (I32, [P, ctypes.POINTER(ibem_profile_data)]),
        "ibem_set_wait_limit": (I32, [P, ctypes.c_longlong]),
        "ibem_batch_create": (I32, [ctypes.POINTER(P), I32, ctypes.POINTER(I32), P, ctypes.POINTER(P)]),
        "ibem_batch_offsets": (I32, [P, ctypes.POINTER(I64)]),
        "ibem_batch_matvec": (I32, [P, P, P]),
        "ibem_batch_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "ibem_batch_destroy": (I32, [P]),
        "ibem_batch_solve": (I32, [P, P, P, ctypes.c_double, I32, I32, ctypes.POINTER(ibem_solve_info)]),
        "ibem_device_status": (I32, [P, ctypes.POINTER(I32)]),
        "ibem_cnn_create": (I32, [I32, ctypes.c_ulonglong, P, ctypes.POINTER(P)]),
        "ibem_cnn_destroy": (I32, [P]),
        "ibem_cnn_params": (I32, [P, P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "ibem_cnn_forward": (I32, [P, P, I32, I32, I32, P, I32]),
        "ibem_cnn_gradients": (I32, [P, P, P, I32, I32, I32, I32, P, ctypes.POINTER(ctypes.c_double)]),
        "ibem_cnn_train_step": (I32, [P, P, P, I32, I32, I32, ctypes.c_float, I32, ctypes.POINTER(ctypes.c_double)]),
        "ibem_cnn_train": (I32, [P, P, P, I32, I32, I32, I32, I32, ctypes.c_float, ctypes.c_ulonglong, I32,
                                 ctypes.POINTER(ctypes.c_double)]),
        "ibem_cnn_launches": (I32, [P, ctypes.POINTER(I64)]),
        "ibem_cnn_device_status": (I32, [P, ctypes.POINTER(I32)]),
        "ibem_cnn_set_coarsening": (I32, [P, I32]),
        "ibem_set_learned_preconditioner": (I32, [P, P]),
        "ibem_learned_apply": (I32, [P, P, P]),
        "ibem_solver_pairs": (I32, [P, P, I32, ctypes.c_double, I32, I32, I32, P, P, ctypes.POINTER(I32),
                                    ctypes.POINTER(ibem_solve_info)]),
        "ibem_solver_residuals": (I32, [P, P, I32, ctypes.c_double, I32, I32, I32, P, ctypes.POINTER(I32),
                                        ctypes.POINTER(ibem_solve_info)]),
        "ibem_cnn_operator_gradients": (I32, [P, P, P, I32, I32, I32, P, ctypes.POINTER(ctypes.c_double)]),
        "ibem_cnn_train_operator": (I32, [P, P, P, I32, I32, I32, ctypes.c_float, ctypes.c_ulonglong, I32, I32,
                                          ctypes.POINTER(ctypes.c_double)]),
        "ibem_last_error": (ctypes.c_char_p, [P]),
        "ibem_status_string": (ctypes.c_char_p, [I32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_lib = _load()


def _check(status, handle=None):
    if status != IBEM_OK:
        msg = _lib.ibem_last_error(handle).decode()
        raise IbemError(_lib.ibem_status_string(status).decode(), msg)


def _dptr(t):
    """Device pointer of a CUDA tensor (must be contiguous float64)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float64":
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _fptr(t):
    """Device pointer of a contiguous float32 CUDA tensor (network images)."""
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float32":
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    """Host pointer of a float64 numpy array or a CPU (e.g. pinned) torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 numpy array")
        return a.ctypes.data_as(ctypes.c_void_p)
    if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float64":
        raise ValueError("expected a contiguous float64 host tensor")
    return ctypes.c_void_p(a.data_ptr())


# ---- patch and parameter builders -------------------------------------------------
def sphere_patches(radius=1.0, center=(0.0, 0.0, 0.0), perturbed=False):
    """The six analytic cube-sphere faces of a sphere (perturbed: each face map
    composed with the piecewise-linear reparametrisation of Sec. 5)."""
    arr = (ibem_patch * 6)()
    for f in range(6):
        arr[f].kind = IBEM_PATCH_SPHERE_FACE
        arr[f].face = f
        arr[f].radius = radius
        arr[f].perturbed = int(bool(perturbed))
        for k in range(3):
            arr[f].center[k] = center[k]
    return arr


def nurbs_patches(specs):
    """specs: list of (deg_u, deg_v, knots_u, knots_v, ctrl [ncp_v][ncp_u][3], weights [ncp_v][ncp_u])."""
    arr = (ibem_patch * len(specs))()
    keep = []
    for i, (du, dv, ku, kv, ctrl, w) in enumerate(specs):
        ku, kv = np.ascontiguousarray(ku, np.float64), np.ascontiguousarray(kv, np.float64)
        ctrl, w = np.ascontiguousarray(ctrl, np.float64), np.ascontiguousarray(w, np.float64)
        keep += [ku, kv, ctrl, w]
        arr[i].kind = IBEM_PATCH_NURBS
        arr[i].deg_u, arr[i].deg_v = du, dv
        arr[i].ncp_u, arr[i].ncp_v = ctrl.shape[1], ctrl.shape[0]
        arr[i].knots_u = ku.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].knots_v = kv.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].ctrl_xyz = ctrl.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    arr._keep = keep
    return arr


IBEM_COUPLING_DF, IBEM_COUPLING_NATIVE, IBEM_COUPLING_NONE, IBEM_COUPLING_GENERATE, IBEM_COUPLING_FP32_ONLY = 0, 1, 2, 3, 4
IBEM_COUPLING_SLICED = 5


IBEM_ADMISSIBLE_ETA_DIAM, IBEM_ADMISSIBLE_ETA_DIST = 0, 1
IBEM_FP32_COUPLING_GENERATE, IBEM_FP32_COUPLING_STORE = 0, 1


def make_params(p, m, q_cheb=6, eta=1.6, kernel=IBEM_LAPLACE, kappa=0.0, gauss_regular=8, gauss_singular=8,
                fp64_coupling=IBEM_COUPLING_DF, admissibility=IBEM_ADMISSIBLE_ETA_DIAM,
                fp32_coupling=IBEM_FP32_COUPLING_GENERATE, gauss_grading=0):
    return ibem_params(kernel, kappa, p, m, q_cheb, eta, gauss_regular, gauss_singular, fp64_coupling,
                       admissibility, fp32_coupling, gauss_grading)


# ---- entry points --------------------------------------------------------------------
def ibem_create(patches, params, stream=None):
    """Returns an opaque handle (ctypes.c_void_p).  ``stream``: a torch.cuda.Stream or None."""
    h = ctypes.c_void_p()
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib.ibem_create(patches, len(patches), ctypes.byref(params), sp, ctypes.byref(h)))
    return h


def ibem_destroy(h):
    _check(_lib.ibem_destroy(h), h)


def ibem_get_info(h):
    info = ibem_info()
    _check(_lib.ibem_get_info(h, ctypes.byref(info)), h)
    return info


def ibem_assemble(h):
    _check(_lib.ibem_assemble(h), h)


def ibem_quad_points(h, xyz):
    _check(_lib.ibem_quad_points(h, _dptr(xyz)), h)


def ibem_rhs(h, g, nrhs, b):
    _check(_lib.ibem_rhs(h, _dptr(g), nrhs, _dptr(b)), h)


def ibem_matvec(h, x, y, nrhs, precision=IBEM_FP64):
    _check(_lib.ibem_matvec(h, _dptr(x), _dptr(y), nrhs, precision), h)


def ibem_matvec_host(h, x, y, nrhs, precision=IBEM_FP64):
    _check(_lib.ibem_matvec_host(h, _hptr(x), _hptr(y), nrhs, precision), h)


def ibem_solve(h, b, w, nrhs, rtol=1e-8, maxit=1000, precond=IBEM_PRECOND_JACOBI, precision=IBEM_FP64,
               check=True):
    info = ibem_solve_info()
    s = _lib.ibem_solve(h, _dptr(b), _dptr(w), nrhs, rtol, maxit, precond, precision, ctypes.byref(info))
    if check:
        _check(s, h)
    return info if check else (s, info)


def ibem_potential(h, w, nrhs, pts, u):
    _check(_lib.ibem_potential(h, _dptr(w), nrhs, _dptr(pts), pts.shape[0], _dptr(u)), h)


def ibem_potential_fmm(h, w, nrhs, pts, u):
    """Potential with the interpolated far field; returns (far terms, near terms)."""
    nf, nn = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.ibem_potential_fmm(h, _dptr(w), nrhs, _dptr(pts), pts.shape[0], _dptr(u), ctypes.byref(nf),
                                   ctypes.byref(nn)), h)
    return nf.value, nn.value


def ibem_rhs_sources(h, src, charges, nrhs, b):
    """Right-hand side of point sources with the interpolated far field; src [nsrc][3],
    charges [nrhs][nsrc] (complex: [..][2]); returns (far terms, near terms)."""
    nf, nn = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.ibem_rhs_sources(h, _dptr(src), _dptr(charges), nrhs, src.shape[0], _dptr(b), ctypes.byref(nf),
                                 ctypes.byref(nn)), h)
    return nf.value, nn.value


def ibem_potential_noalloc(h, w, nrhs, pts, u):
    """ibem_potential without device allocation (fixed scratch inside libibem)."""
    _check(_lib.ibem_potential_noalloc(h, _dptr(w), nrhs, _dptr(pts), pts.shape[0], _dptr(u)), h)


def ibem_block_tree(patches, params):
    """Host only.  Returns (near [n_near, 8] int32, far [n_far, 8] int32)."""
    nn, nf = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.ibem_block_tree(patches, len(patches), ctypes.byref(params), ctypes.byref(nn), None,
                                ctypes.byref(nf), None))
    near = np.zeros((nn.value, 8), dtype=np.int32)
    far = np.zeros((nf.value, 8), dtype=np.int32)
    _check(_lib.ibem_block_tree(patches, len(patches), ctypes.byref(params), ctypes.byref(nn),
                                near.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nf),
                                far.ctypes.data_as(ctypes.c_void_p)))
    return near, far


def ibem_set_fp32_coupling(h, mode):
    _check(_lib.ibem_set_fp32_coupling(h, mode), h)


def ibem_set_fp32_coupling_status(h, mode):
    """As ibem_set_fp32_coupling, returning the status instead of raising (IBEM_ERR_OOM
    keeps the generating path)."""
    return _lib.ibem_set_fp32_coupling(h, mode)


def ibem_near_orders(patches, params):
    """Host only.  Gauss order of every near pair, in the order of ibem_block_tree's near list."""
    nn = ctypes.c_int64()
    _check(_lib.ibem_near_orders(patches, len(patches), ctypes.byref(params), ctypes.byref(nn), None))
    out = np.zeros(nn.value, dtype=np.int32)
    _check(_lib.ibem_near_orders(patches, len(patches), ctypes.byref(params), ctypes.byref(nn),
                                 out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ibem_profile_enable(h, enable=True):
    _check(_lib.ibem_profile_enable(h, 1 if enable else 0), h)


def ibem_profile_read(h):
    """Returns dict(applications, launches, ms={phase: summed ms})."""
    d = ibem_profile_data()
    _check(_lib.ibem_profile_read(h, ctypes.byref(d)), h)
    return {"applications": d.applications, "launches": d.launches,
            "ms": {name: d.ms[i] for i, name in enumerate(PHASES)}}


IBEM_DEVICE_OK, IBEM_DEVICE_TIMEOUT, IBEM_DEVICE_OVERFLOW = 0, 1, 2


def ibem_set_wait_limit(h, limit):
    _check(_lib.ibem_set_wait_limit(h, limit), h)


def ibem_device_status(h):
    st = ctypes.c_int()
    _check(_lib.ibem_device_status(h, ctypes.byref(st)), h)
    return st.value


def ibem_batch_create(handles, nrhs, stream=None):
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.value for h in handles])
    rr = (ctypes.c_int * n)(*nrhs)
    b = ctypes.c_void_p()
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib.ibem_batch_create(arr, n, rr, sp, ctypes.byref(b)))
    return b


def ibem_batch_offsets(b, n):
    off = (ctypes.c_int64 * (n + 1))()
    _check(_lib.ibem_batch_offsets(b, off))
    return list(off)


def ibem_batch_matvec(b, x, y):
    _check(_lib.ibem_batch_matvec(b, _dptr(x), _dptr(y)))


def ibem_batch_info(b):
    l, t, rb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.ibem_batch_info(b, ctypes.byref(l), ctypes.byref(t), ctypes.byref(rb)))
    return {"launches_per_apply": l.value, "coupling_threads": t.value, "coupling_rhs_tile": rb.value}


def ibem_batch_destroy(b):
    _check(_lib.ibem_batch_destroy(b))


def ibem_batch_solve(b, rhs, x, rtol=1e-8, maxit=2000, precond=IBEM_PRECOND_JACOBI, check=True):
    """Concatenated right-hand sides and solutions (float64 CUDA, ibem_batch_offsets
    layout); returns info, or (status, info) with check=False."""
    info = ibem_solve_info()
    s = _lib.ibem_batch_solve(b, _dptr(rhs), _dptr(x), rtol, maxit, precond, ctypes.byref(info))
    if check:
        _check(s)
        return info
    return s, info


def ibem_last_error(h=None):
    return _lib.ibem_last_error(h).decode()


def ibem_status_string(s):
    return _lib.ibem_status_string(s).decode()


# ---- learned preconditioner --------------------------------------------------------
def ibem_cnn_create(channels=32, seed=0, stream=None):
    c = ctypes.c_void_p()
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib.ibem_cnn_create(channels, seed, sp, ctypes.byref(c)))
    return c


def ibem_cnn_destroy(c):
    _check(_lib.ibem_cnn_destroy(c))


def ibem_cnn_params(c, set_params=None):
    """Current parameters (float32 numpy array) after loading set_params if given."""
    n = ctypes.c_size_t()
    _check(_lib.ibem_cnn_params(c, None, None, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.float32)
    src = None
    if set_params is not None:
        src = np.ascontiguousarray(set_params, dtype=np.float32)
        if src.shape != (n.value,):
            raise ValueError("expected %d parameters" % n.value)
    _check(_lib.ibem_cnn_params(c, out.ctypes.data_as(ctypes.c_void_p),
                                src.ctypes.data_as(ctypes.c_void_p) if src is not None else None, None))
    return out


def ibem_cnn_forward(c, x, out, precision=IBEM_BF16):
    B, _, H, W = x.shape
    _check(_lib.ibem_cnn_forward(c, _fptr(x), B, H, W, _fptr(out), precision))


def ibem_cnn_gradients(c, x, target, precision=IBEM_FP32):
    """(loss, gradient as float32 numpy array)."""
    B, _, H, W = x.shape
    n = ctypes.c_size_t()
    _check(_lib.ibem_cnn_params(c, None, None, ctypes.byref(n)))
    g = np.zeros(n.value, dtype=np.float32)
    loss = ctypes.c_double()
    _check(_lib.ibem_cnn_gradients(c, _fptr(x), _fptr(target), B, H, W, precision,
                                   g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)))
    return loss.value, g


def ibem_cnn_train_step(c, x, target, lr, precision=IBEM_BF16):
    B, _, H, W = x.shape
    loss = ctypes.c_double()
    _check(_lib.ibem_cnn_train_step(c, _fptr(x), _fptr(target), B, H, W, lr, precision, ctypes.byref(loss)))
    return loss.value


def ibem_cnn_train(c, x, target, batch, epochs, lr, seed=0, augment=IBEM_AUGMENT_PHASE | IBEM_AUGMENT_DIHEDRAL):
    n, _, H, W = x.shape
    loss = ctypes.c_double()
    _check(_lib.ibem_cnn_train(c, _fptr(x), _fptr(target), n, H, W, batch, epochs, lr, seed, augment,
                               ctypes.byref(loss)))
    return loss.value


def ibem_cnn_launches(c):
    n = ctypes.c_int64()
    _check(_lib.ibem_cnn_launches(c, ctypes.byref(n)))
    return n.value


def ibem_cnn_set_coarsening(c, factor):
    _check(_lib.ibem_cnn_set_coarsening(c, factor))


def ibem_set_learned_preconditioner(h, c):
    _check(_lib.ibem_set_learned_preconditioner(h, c), h)


def ibem_learned_apply(h, v, z):
    _check(_lib.ibem_learned_apply(h, _dptr(v), _dptr(z)), h)


def ibem_solver_pairs(h, b, nrhs, in_img, tgt_img, rtol=1e-10, maxit=400, stride=1, max_pairs=32, check=True):
    """Writes pairs into the float32 image tensors; returns (n_pairs, info) or
    (status, n_pairs, info) with check=False."""
    n = ctypes.c_int()
    info = ibem_solve_info()
    s = _lib.ibem_solver_pairs(h, _dptr(b), nrhs, rtol, maxit, stride, max_pairs, _fptr(in_img), _fptr(tgt_img),
                               ctypes.byref(n), ctypes.byref(info))
    if check:
        _check(s, h)
        return n.value, info
    return s, n.value, info


def ibem_solver_residuals(h, b, nrhs, r_out, rtol=1e-10, maxit=400, stride=1, max_vecs=32, check=True):
    """Unit-norm solver residuals into r_out (float64 CUDA [nrhs * max_vecs, ndof, 2]);
    returns (n, info) or (status, n, info) with check=False."""
    n = ctypes.c_int()
    info = ibem_solve_info()
    s = _lib.ibem_solver_residuals(h, _dptr(b), nrhs, rtol, maxit, stride, max_vecs, _dptr(r_out), ctypes.byref(n),
                                   ctypes.byref(info))
    if check:
        _check(s, h)
        return n.value, info
    return s, n.value, info


def ibem_cnn_operator_gradients(h, c, r, n, precision=IBEM_FP32, op_precision=IBEM_FP64):
    """(loss, gradient) of the residual-norm objective on n residuals r (float64 CUDA)."""
    m = ctypes.c_size_t()
    _check(_lib.ibem_cnn_params(c, None, None, ctypes.byref(m)))
    g = np.zeros(m.value, dtype=np.float32)
    loss = ctypes.c_double()
    _check(_lib.ibem_cnn_operator_gradients(h, c, _dptr(r), n, precision, op_precision,
                                            g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)), h)
    return loss.value, g


def ibem_cnn_train_operator(h, c, r, n, batch, epochs, lr, seed=0, augment=IBEM_AUGMENT_PHASE, op_precision=IBEM_FP32):
    loss = ctypes.c_double()
    _check(_lib.ibem_cnn_train_operator(h, c, _dptr(r), n, batch, epochs, lr, seed, augment, op_precision,
                                        ctypes.byref(loss)), h)
    return loss.value


def ibem_cnn_device_status(c):
    st = ctypes.c_int()
    _check(_lib.ibem_cnn_device_status(c, ctypes.byref(st)))
    return st.value
