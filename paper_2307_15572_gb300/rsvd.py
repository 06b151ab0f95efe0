"""Python binding of the C ABI in include/rsvd.h (argument marshalling only).

Every function here forwards to the compiled library ``_lib/librsvd.so``;
no step of the decomposition runs in Python.  Loading fails loudly when the
library is missing or no CUDA device is present -- there is no CPU fallback.

Low-level names mirror the C entry points (``rsvd_plan``, ``rsvd_decompose``,
``rsvd_decompose_batched``, ``rsvd_reconstruct_error``, ``rsvd_plan_destroy``).
``Plan`` is a thin convenience wrapper that takes torch CUDA tensors (or host
numpy arrays) and allocates the caller-owned output buffers with torch.
"""

import ctypes as C
import os

import numpy as np

from . import build as _build

# ------------------------------------------------------------------ enums
RSVD_OK = 0
RSVD_WARN_SHIFTED_CQR = 1
RSVD_WARN_RANK_CAPPED = 2
RSVD_ERR_INVALID_ARG = -1
RSVD_ERR_CUDA = -2
RSVD_ERR_OOM = -3
RSVD_ERR_NONFINITE = -4
RSVD_ERR_NOT_CONVERGED = -5
RSVD_ERR_TOL_NOT_MET = -6
RSVD_ERR_TIMEOUT = -7
RSVD_ERR_UNSUPPORTED = -8

PREC = {"fp64": 0, "bf16x": 1}
POLICY = {"fixed": 0, "tol": 1, "adaptive": 2, "learned": 3}
DENSE_F64, TILE_RULE = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1


class Opts(C.Structure):
    _fields_ = [("n_max", C.c_int64), ("k", C.c_int32), ("p", C.c_int32), ("q", C.c_int32),
                ("tol", C.c_double), ("l_max", C.c_int32), ("block_b", C.c_int32),
                ("precision", C.c_int32), ("slices", C.c_int32), ("rank_policy", C.c_int32),
                ("rayleigh_ritz", C.c_int32), ("seed", C.c_uint64), ("stream", C.c_void_p),
                ("mlp_weights", C.c_void_p)]


class Matrix(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mem", C.c_int32), ("n", C.c_int64), ("data", C.c_void_p),
                ("ld", C.c_int64), ("rule_m", C.c_int32), ("rule_c", C.c_void_p),
                ("rule_s", C.c_void_p), ("rule_w", C.c_void_p), ("rule_eta", C.c_double),
                ("rule_seed", C.c_uint64)]


class Factors(C.Structure):
    _fields_ = [("mem", C.c_int32), ("U", C.c_void_p), ("ldu", C.c_int64), ("S", C.c_void_p),
                ("V", C.c_void_p), ("ldv", C.c_int64), ("k_cap", C.c_int32), ("k_out", C.c_int32),
                ("l_used", C.c_int32), ("err_est", C.c_double), ("status", C.c_int32),
                ("tol", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("tc_launches", C.c_int64), ("tc_ms", C.c_double),
                ("tc_bytes", C.c_double), ("tc_flops", C.c_double), ("f64_launches", C.c_int64),
                ("f64_ms", C.c_double), ("f64_flops", C.c_double), ("gen_launches", C.c_int64),
                ("gen_ms", C.c_double), ("gen_flops", C.c_double), ("gen_mma_flops", C.c_double),
                ("cvt_launches", C.c_int64), ("cvt_ms", C.c_double), ("cvt_bytes", C.c_double),
                ("gram_launches", C.c_int64), ("gram_ms", C.c_double), ("gram_flops", C.c_double),
                ("gram_mma_flops", C.c_double), ("nn_launches", C.c_int64), ("nn_ms", C.c_double),
                ("nn_flops", C.c_double), ("f64in_launches", C.c_int64), ("f64in_ms", C.c_double),
                ("f64in_bytes", C.c_double), ("f64in_flops", C.c_double)]


class TuneRecord(C.Structure):
    _fields_ = [("kind", C.c_int32), ("candidates", C.c_int32), ("choice", C.c_int32), ("bn", C.c_int32),
                ("split_target", C.c_int32), ("min_split", C.c_int32), ("stages", C.c_int32),
                ("order", C.c_int32), ("ms_default", C.c_float), ("ms_best", C.c_float),
                ("tune_ms", C.c_float)]


_lib = None


def load(build=True):
    """Load (building first if needed) the C-ABI library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("librsvd.so not found at %s; run paper_2307_15572_gb300.build.build()" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.rsvd_plan.argtypes = [C.POINTER(P), C.POINTER(Opts)]
    lib.rsvd_plan.restype = C.c_int
    lib.rsvd_plan_destroy.argtypes = [P]
    lib.rsvd_plan_destroy.restype = None
    lib.rsvd_decompose.argtypes = [P, C.POINTER(Matrix), C.POINTER(Factors)]
    lib.rsvd_decompose.restype = C.c_int
    lib.rsvd_decompose_batched.argtypes = [P, C.c_int32, C.POINTER(Matrix), C.POINTER(Factors),
                                           C.POINTER(C.c_int)]
    lib.rsvd_decompose_batched.restype = C.c_int
    lib.rsvd_reconstruct_error.argtypes = [P, C.POINTER(Matrix), C.POINTER(Factors), C.POINTER(C.c_double)]
    lib.rsvd_reconstruct_error.restype = C.c_int
    lib.rsvd_plan_workspace_bytes.argtypes = [P]
    lib.rsvd_plan_workspace_bytes.restype = C.c_int64
    lib.rsvd_last_error_string.argtypes = []
    lib.rsvd_last_error_string.restype = C.c_char_p
    lib.rsvd_version.argtypes = []
    lib.rsvd_version.restype = C.c_int32
    lib.rsvd_plan_set_profiling.argtypes = [P, C.c_int32]
    lib.rsvd_plan_set_profiling.restype = C.c_int
    lib.rsvd_plan_set_graphs.argtypes = [P, C.c_int32]
    lib.rsvd_plan_set_graphs.restype = C.c_int
    lib.rsvd_plan_set_autotune.argtypes = [P, C.c_int32]
    lib.rsvd_plan_set_autotune.restype = C.c_int
    lib.rsvd_plan_tune_records.argtypes = [P, C.POINTER(TuneRecord), C.c_int32, C.POINTER(C.c_int32)]
    lib.rsvd_plan_tune_records.restype = C.c_int
    lib.rsvd_plan_profile.argtypes = [P, C.POINTER(Profile), C.c_int32]
    lib.rsvd_plan_profile.restype = C.c_int
    lib.rsvd_mlp_param_count.argtypes = [C.c_int32]
    lib.rsvd_mlp_param_count.restype = C.c_int64
    lib.rsvd_mlp_work_floats.argtypes = [C.c_int32, C.c_int32]
    lib.rsvd_mlp_work_floats.restype = C.c_int64
    lib.rsvd_mlp_forward.argtypes = [P, C.c_int32, P, C.c_int32, P, P]
    lib.rsvd_mlp_forward.restype = C.c_int
    lib.rsvd_mlp_loss_grad.argtypes = [P, C.c_int32, P, P, C.c_int32, P, P, P, P]
    lib.rsvd_mlp_loss_grad.restype = C.c_int
    lib.rsvd_mlp_adam.argtypes = [P, P, P, P, C.c_int64, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float, P]
    lib.rsvd_mlp_adam.restype = C.c_int
    lib.rsvd_mlp_standardize.argtypes = [P, C.c_int32, C.c_int32, C.c_float, P, P, P, P]
    lib.rsvd_mlp_standardize.restype = C.c_int
    lib.rsvd_mlp_fold.argtypes = [P, C.c_int32, P, P, P, P, P, P]
    lib.rsvd_mlp_fold.restype = C.c_int
    lib.rsvd_mlp_gather_rows.argtypes = [P, P, C.c_int32, C.c_int32, P, P]
    lib.rsvd_mlp_gather_rows.restype = C.c_int
    lib.rsvd_probe_features.argtypes = [P, C.c_int32, C.POINTER(Matrix), C.POINTER(C.c_double), P]
    lib.rsvd_probe_features.restype = C.c_int
    lib.rsvd_reconstruct_error_noalloc.argtypes = [P, C.c_int64, C.c_int64, P, C.c_int64, P, P, C.c_int64,
                                                   C.c_int32, P, P]
    lib.rsvd_reconstruct_error_noalloc.restype = C.c_int
    lib.rsvd_transform_factors.argtypes = [P, C.POINTER(Factors), C.c_int64, P, C.c_int64, C.c_int64, P, C.c_int64,
                                           P, C.c_int64]
    lib.rsvd_transform_factors.restype = C.c_int
    lib.rsvd_symmetric_signs.argtypes = [P, C.POINTER(Factors), C.c_int64, P]
    lib.rsvd_symmetric_signs.restype = C.c_int
    lib.rsvd_compression_ratio.argtypes = [C.c_int64, C.c_int32, C.c_int32]
    lib.rsvd_compression_ratio.restype = C.c_double
    lib.rsvd_rule_rows.argtypes = [P, C.POINTER(Matrix), C.c_int64, C.c_int32, P, C.c_int64]
    lib.rsvd_rule_rows.restype = C.c_int
    lib.rsvd_gram_f32.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int32, P, C.c_int32]
    lib.rsvd_gram_f32.restype = C.c_int
    lib.rsvd_panel_product.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int32, P, C.c_int64, C.c_int32, C.c_int32, P,
                                       C.c_int64, C.c_int32]
    lib.rsvd_panel_product.restype = C.c_int
    _lib = lib
    return lib


def last_error():
    return load().rsvd_last_error_string().decode()


class RsvdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("rsvd status %d: %s" % (status, msg))
        self.status = status


def _check(status):
    if status < 0:
        raise RsvdError(status, last_error())
    return status


# -------------------------------------------------------- C-named forwarders
def rsvd_plan(opts):
    h = C.c_void_p()
    _check(load().rsvd_plan(C.byref(h), C.byref(opts)))
    return h


def rsvd_plan_destroy(h):
    load().rsvd_plan_destroy(h)


def rsvd_decompose(h, mat, fac):
    return load().rsvd_decompose(h, C.byref(mat), C.byref(fac))


def rsvd_decompose_batched(h, mats, facs):
    n = len(mats)
    MA = (Matrix * n)(*mats)
    FA = (Factors * n)(*facs)
    st = (C.c_int * n)()
    r = load().rsvd_decompose_batched(h, n, MA, FA, st)
    for i in range(n):
        facs[i] = FA[i]
    return r, list(st)


def rsvd_plan_set_profiling(h, enable):
    _check(load().rsvd_plan_set_profiling(h, 1 if enable else 0))


def rsvd_plan_set_graphs(h, enable):
    _check(load().rsvd_plan_set_graphs(h, 1 if enable else 0))


def rsvd_plan_set_autotune(h, enable):
    _check(load().rsvd_plan_set_autotune(h, 1 if enable else 0))


def rsvd_plan_tune_records(h):
    """The plan's autotuning choices, as dicts, in the order they were made."""
    n = C.c_int32(0)
    _check(load().rsvd_plan_tune_records(h, None, 0, C.byref(n)))
    arr = (TuneRecord * max(1, n.value))()
    _check(load().rsvd_plan_tune_records(h, arr, n.value, C.byref(n)))
    return [{f: getattr(arr[i], f) for f, _ in TuneRecord._fields_} for i in range(n.value)]


def rsvd_plan_profile(h, reset=False):
    p = Profile()
    _check(load().rsvd_plan_profile(h, C.byref(p), 1 if reset else 0))
    return {f: getattr(p, f) for f, _ in Profile._fields_}


RSVD_NOALLOC_MAX_N = 16384
MLP_FEATURES = 19
MLP_HIDDEN = 128


def rsvd_mlp_param_count(d=MLP_FEATURES):
    return load().rsvd_mlp_param_count(d)


def rsvd_mlp_work_floats(d, B):
    return load().rsvd_mlp_work_floats(d, B)


def rsvd_mlp_forward(theta, d, X, B, Y, stream=None):
    return _check(load().rsvd_mlp_forward(theta, d, X, B, Y, stream))


def rsvd_mlp_loss_grad(theta, d, X, T, B, grad, loss, work, stream=None):
    return _check(load().rsvd_mlp_loss_grad(theta, d, X, T, B, grad, loss, work, stream))


def rsvd_mlp_adam(theta, grad, m, v, nparams, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    return _check(load().rsvd_mlp_adam(theta, grad, m, v, nparams, t, lr, beta1, beta2, eps, stream))


def rsvd_mlp_standardize(X, N, d, sd_floor, mean, sd, Xn, stream=None):
    return _check(load().rsvd_mlp_standardize(X, N, d, sd_floor, mean, sd, Xn, stream))


def rsvd_mlp_fold(theta, d, mean_x, sd_x, mean_t, sd_t, out, stream=None):
    return _check(load().rsvd_mlp_fold(theta, d, mean_x, sd_x, mean_t, sd_t, out, stream))


def rsvd_mlp_gather_rows(src, idx, B, cols, dst, stream=None):
    return _check(load().rsvd_mlp_gather_rows(src, idx, B, cols, dst, stream))


def rsvd_probe_features(h, mats, tols, features):
    n = len(mats)
    MA = (Matrix * n)(*mats)
    TA = (C.c_double * n)(*tols)
    return _check(load().rsvd_probe_features(h, n, MA, TA, features))



def rsvd_reconstruct_error_noalloc(A, lda, n, U, ldu, S, V, ldv, k, rel_err, stream=None):
    """Forward to the no-allocation residual entry point (all device pointers)."""
    return load().rsvd_reconstruct_error_noalloc(A, lda, n, U, ldu, S, V, ldv, k, rel_err, stream)


def rsvd_rule_rows(h, mat, r0, rows, out, ldo):
    """Rows r0..r0+rows-1 of a tile rule into the device FP32 buffer `out` (row-major, ld ldo)."""
    return _check(load().rsvd_rule_rows(h, C.byref(mat), int(r0), int(rows), out, int(ldo)))


RSVD_GRAM_TC, RSVD_GRAM_DOT2, RSVD_GRAM_TC_F32 = 0, 1, 2


def rsvd_gram_f32(h, Y, ldy, n, l, G, method=RSVD_GRAM_TC):
    """G = Y^T Y (FP64-grade) of the device FP32 panel Y (n x l, column-major, ld ldy) into device G (l x l)."""
    return _check(load().rsvd_gram_f32(h, Y, int(ldy), int(n), int(l), G, int(method)))


def rsvd_panel_product(h, A, lda, n, K, B, ldb, b_fp64, N, Cout, ldc, c_fp64):
    """C = A B on the tensor cores (device pointers, column-major; A FP32 n x K, B K x N, K, N <= 128)."""
    return _check(load().rsvd_panel_product(h, A, int(lda), int(n), int(K), B, int(ldb), int(bool(b_fp64)), int(N),
                                            Cout, int(ldc), int(bool(c_fp64))))


def rsvd_transform_factors(h, fac, n, B, ldb, m, Lt, ldl, Rt, ldr):
    """Lt = B^T U_k, Rt = B^T V_k (device pointers, column-major)."""
    return _check(load().rsvd_transform_factors(h, C.byref(fac), int(n), B, int(ldb), int(m), Lt, int(ldl), Rt,
                                                int(ldr)))


def rsvd_symmetric_signs(h, fac, n, signs):
    return _check(load().rsvd_symmetric_signs(h, C.byref(fac), int(n), signs))


def rsvd_compression_ratio(n, k, one_factor=False):
    return load().rsvd_compression_ratio(int(n), int(k), 1 if one_factor else 0)


def rsvd_reconstruct_error(h, mat, fac):
    out = C.c_double()
    _check(load().rsvd_reconstruct_error(h, C.byref(mat), C.byref(fac), C.byref(out)))
    return out.value


# ---------------------------------------------------------------- wrapper
def make_opts(n_max, k=0, p=10, q=0, tol=0.0, precision="fp64", slices=0, policy="fixed", seed=0,
              stream=None, rayleigh_ritz=False, l_max=0, block_b=0, mlp_weights=None):
    o = Opts()
    o.n_max = int(n_max)
    o.k = int(k)
    o.p = int(p)
    o.q = int(q)
    o.tol = float(tol)
    o.l_max = int(l_max)
    o.block_b = int(block_b)
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.slices = int(slices)
    o.rank_policy = POLICY[policy] if isinstance(policy, str) else int(policy)
    o.rayleigh_ritz = 1 if rayleigh_ritz else 0
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.stream = stream
    o.mlp_weights = mlp_weights
    return o


def dense(A):
    """Matrix descriptor of a torch CUDA tensor (FP64, n x n) or a host numpy array."""
    m = Matrix()
    m.kind = DENSE_F64
    if isinstance(A, np.ndarray):
        assert A.dtype == np.float64 and A.ndim == 2 and A.shape[0] == A.shape[1]
        assert A.flags.c_contiguous or A.strides[1] == 8
        m.mem = MEM_HOST
        m.n = A.shape[0]
        m.ld = A.strides[0] // 8
        m.data = A.ctypes.data
    else:
        import torch
        assert A.dtype == torch.float64 and A.dim() == 2 and A.shape[0] == A.shape[1]
        assert A.stride(1) == 1
        m.mem = MEM_DEVICE if A.is_cuda else MEM_HOST
        m.n = A.shape[0]
        m.ld = A.stride(0)
        m.data = A.data_ptr()
    return m


def rule(n, c, s, w, eta=0.0, seed=0):
    """Descriptor of a tile-rule channel; the host parameter arrays are kept
    alive on the returned object."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (c, s, w)]
    assert arrs[0].shape == arrs[1].shape == arrs[2].shape and arrs[0].ndim == 1
    m = Matrix()
    m.kind = TILE_RULE
    m.mem = MEM_DEVICE
    m.n = int(n)
    m.data = None
    m.ld = int(n)
    m.rule_m = arrs[0].shape[0]
    m.rule_c, m.rule_s, m.rule_w = (a.ctypes.data for a in arrs)
    m.rule_eta = float(eta)
    m.rule_seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    m._keep = arrs
    return m


class Plan:
    """Plan plus torch-allocated output buffers; see include/rsvd.h for the semantics."""

    def __init__(self, n_max, autotune=False, **kw):
        load()
        self.opts = make_opts(n_max, **kw)
        self.h = rsvd_plan(self.opts)
        if autotune:
            rsvd_plan_set_autotune(self.h, True)

    def close(self):
        if self.h is not None:
            rsvd_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def factors_for(n, k_cap, device="cuda"):
        import torch
        U = torch.empty((k_cap, n), dtype=torch.float64, device=device)   # column-major n x k_cap
        V = torch.empty((k_cap, n), dtype=torch.float64, device=device)
        S = torch.empty((k_cap,), dtype=torch.float64, device=device)
        f = Factors()
        f.mem = MEM_DEVICE
        f.U, f.ldu = U.data_ptr(), n
        f.V, f.ldv = V.data_ptr(), n
        f.S = S.data_ptr()
        f.k_cap = k_cap
        return f, (U, S, V)

    def decompose_batched(self, mats, k_cap):
        """mats: list of torch CUDA FP64 tensors.  Returns (status, [result dicts])."""
        descs, facs, bufs = [], [], []
        for A in mats:
            descs.append(A if isinstance(A, Matrix) else dense(A))
            n = descs[-1].n
            f, b = self.factors_for(n, min(k_cap, n))
            facs.append(f)
            bufs.append(b)
        r, per = rsvd_decompose_batched(self.h, descs, facs)
        out = []
        for f, (U, S, V), s in zip(facs, bufs, per):
            k = f.k_out
            out.append(dict(U=U[:k].T, S=S[:k], V=V[:k].T, k=k, l=f.l_used, err_est=f.err_est, status=s,
                            _fac=f))
        return r, out

    def decompose(self, A, k_cap):
        r, out = self.decompose_batched([A], k_cap)
        return r, out[0]

    def reconstruct_error(self, A, res):
        return rsvd_reconstruct_error(self.h, A if isinstance(A, Matrix) else dense(A), res["_fac"])
