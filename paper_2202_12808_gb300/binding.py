"""ctypes binding of libcofem (include/cofem.h): argument marshalling only.

Every function below has the name of the C entry point it calls and does no
arithmetic of the method: all work runs in the library's CUDA kernels.  The
library is loaded from this package directory (built in-tree by
``build.py``); if it is missing, ``lib()`` raises -- there is no fallback.

Device buffers are passed as integers (``tensor.data_ptr()``); streams as
integers (``torch.cuda.current_stream().cuda_stream``).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcofem.so")

COFEM_F64, COFEM_F32, COFEM_BF16, COFEM_FP8_E4M3 = 0, 1, 2, 3

STATUS = {0: "COFEM_OK", 1: "COFEM_ERR_INVALID_ARG", 2: "COFEM_ERR_CUDA",
          3: "COFEM_ERR_NONFINITE", 4: "COFEM_ERR_BREAKDOWN", 5: "COFEM_ERR_TIMEOUT",
          6: "COFEM_ERR_UNSUPPORTED", 7: "COFEM_ERR_WORKSPACE"}


class CofemError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        msg = "%s failed: %s" % (where, STATUS.get(code, code))
        if detail:
            msg += " [%s]" % detail
        super().__init__(msg)


class cofem_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("em_iters", ctypes.c_int32),
                ("cg_max_iters", ctypes.c_int32), ("fixed_cg_iters", ctypes.c_int32),
                ("resid_replace_every", ctypes.c_int32), ("vec_dtype", ctypes.c_int32),
                ("stop_rule", ctypes.c_int32), ("tasks", ctypes.c_int32),
                ("cg_tol", ctypes.c_double), ("alpha_init", ctypes.c_double),
                ("den_floor", ctypes.c_double), ("support_threshold", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("t_offset", ctypes.c_int64),
                ("mlp", ctypes.c_void_p), ("solver", ctypes.c_int32)]


class cofem_stats(ctypes.Structure):
    _fields_ = [("cg_iters", ctypes.POINTER(ctypes.c_int32)),
                ("relres", ctypes.POINTER(ctypes.c_double)),
                ("clamps", ctypes.POINTER(ctypes.c_int32)),
                ("support", ctypes.POINTER(ctypes.c_int32)),
                ("end_ns", ctypes.POINTER(ctypes.c_int64))]


class cofem_problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("D", ctypes.c_int64), ("phi_dev", ctypes.c_void_p),
                ("ld", ctypes.c_int64), ("y_dev", ctypes.c_void_p), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


_S = ctypes.c_int
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_SZ = ctypes.c_size_t

_SIGS = {
    "cofem_status_string": (ctypes.c_char_p, [_S]),
    "cofem_last_error": (ctypes.c_char_p, []),
    "cofem_op_dense": (_S, [_I64, _I64, _S, _P, _I64, _P, ctypes.POINTER(_P)]),
    "cofem_op_dense_set_terms": (_S, [_P, _I32]),
    "cofem_op_dense_set_tile_rows": (_S, [_P, _I32]),
    "cofem_op_dense_get_pipeline": (_S, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                         ctypes.POINTER(_I32)]),
    "cofem_op_dense_set_l2_resident": (_S, [_P, _I64]),
    "cofem_dense_packed_bytes": (_SZ, [_I64, _I64]),
    "cofem_op_dense_packed_bytes": (_SZ, [_P]),
    "cofem_quantize_fp8_tiles": (_S, [_P, _I64, _I64, _I64, _P, _I64, _P, _P]),
    "cofem_op_dense_set_pipeline": (_S, [_P, _I32, _I32]),
    "cofem_op_dense_autotune_workspace_bytes": (_SZ, [_P, _I32]),
    "cofem_op_dense_autotune": (_S, [_P, _I32, _P, _SZ, _P, ctypes.POINTER(_I32),
                                     ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)]),
    "cofem_op_dense_attach_packed": (_S, [_P, _P, _SZ, _P]),
    "cofem_op_conv1d": (_S, [_I64, _I32, _I32, _P, ctypes.POINTER(_P)]),
    "cofem_op_conv1d_set_tensor_cores": (_S, [_P, _I32]),
    "cofem_op_dct": (_S, [_I64, _I64, _P, ctypes.POINTER(_P)]),
    "cofem_op_destroy": (None, [_P]),
    "cofem_last_fit_fallbacks": (_I32, []),
    "cofem_op_col_norms": (_S, [_P, _P, _P]),
    "cofem_col_norms_workspace_bytes": (_S, [_P, ctypes.POINTER(_SZ)]),
    "cofem_op_col_norms_ws": (_S, [_P, _P, _P, _SZ, _P]),
    "cofem_mlp_features": (_S, [_P, _P, _D, _P, _P, _I64, _P, _P]),
    "cofem_mlp_targets": (_S, [_P, _P, _D, _P, _P, _I64, _P, _P]),
    "cofem_mlp_forward": (_S, [_P, _S, _P, _I64, _P, _P]),
    "cofem_mlp_train_workspace_bytes": (_SZ, [_I64]),
    "cofem_mlp_grad": (_S, [_P, _S, _P, _P, _I64, _P, _P, _P, _SZ, _P]),
    "cofem_mlp_adam_step": (_S, [_P, _P, _P, _P, _P, _P, _I64, _I32, ctypes.c_float, _P, _SZ,
                                 _P, _P]),
    "cofem_op_shape": (_S, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "cofem_params_default": (None, [ctypes.POINTER(cofem_params)]),
    "cofem_workspace_bytes": (_S, [_P, ctypes.POINTER(cofem_params), ctypes.POINTER(_SZ)]),
    "cofem_fit": (_S, [_P, _P, _D, ctypes.POINTER(cofem_params), _P, _SZ, _P, _P, _P,
                       ctypes.POINTER(cofem_stats), _P]),
    "cofem_batched_workspace_bytes": (_S, [_I32, ctypes.POINTER(cofem_problem),
                                           ctypes.POINTER(cofem_params), ctypes.POINTER(_SZ)]),
    "cofem_fit_batched": (_S, [_I32, ctypes.POINTER(cofem_problem), ctypes.POINTER(cofem_params),
                               _P, _SZ, _P, _P, _P, ctypes.POINTER(cofem_stats), _P]),
    "cofem_probe_fill": (_S, [ctypes.c_uint64, _I64, _I32, _I64, _S, _P, _I64, _P]),
    "cofem_apply_workspace_bytes": (_S, [_P, _S, _I32, ctypes.POINTER(_SZ)]),
    "cofem_op_apply": (_S, [_P, _S, _P, _I64, _I32, _P, _D, _P, _P, _SZ, _P]),
    "cofem_op_apply_timed": (_S, [_P, _S, _P, _I64, _I32, _P, _D, _P, _P, _SZ, _P,
                                  ctypes.POINTER(ctypes.c_float), _I32, ctypes.POINTER(_I32)]),
    "cofem_op_apply_noalloc": (_S, [_P, _S, _P, _I64, _I32, _P, _D, _P, _P]),
    "cofem_noalloc_scratch_capacity": (_SZ, []),
    "cofem_selftest_wait_timeout": (_S, [_I64, _P]),
    "cofem_selftest_cg_update_workspace_bytes": (_SZ, []),
    "cofem_bench_cg_kernels_workspace_bytes": (_SZ, [_I64, _I32]),
    "cofem_bench_cg_kernels": (_S, [_I64, _I32, _I32, _P, _SZ, _P, ctypes.POINTER(ctypes.c_float)]),
    "cofem_bench_bcg_kernels_workspace_bytes": (_SZ, [_I64, _I32]),
    "cofem_bench_bcg_kernels": (_S, [_I64, _I32, _I32, _P, _SZ, _P,
                                     ctypes.POINTER(ctypes.c_float)]),
    "cofem_selftest_cg_update_timeout": (_S, [_I64, _P, _SZ, _P]),
    "cofem_op_forward": (_S, [_P, _S, _P, _I64, _I32, _P, _I64, _P, _SZ, _P]),
    "cofem_op_adjoint": (_S, [_P, _S, _P, _I64, _I32, _P, _I64, _P, _SZ, _P]),
    "cofem_diag_mstep": (_S, [ctypes.c_uint64, _I64, _I32, _I64, _S, _P, _I64, _D, _D, _P,
                              _P, _P, _P, _P]),
}

# Declared in include/cofem.h; the ABI test checks that each is exported.
EXPORTED = sorted(_SIGS)

_lib = None


def lib():
    """Load libcofem.so from the package directory (raises if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcofem.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        detail = ""
        if rc == 2:
            detail = (lib().cofem_last_error() or b"").decode()
        raise CofemError(rc, where, detail)


# ---------------------------------------------------------------- wrappers

def cofem_status_string(code):
    return lib().cofem_status_string(code).decode()


def cofem_op_dense(N, D, dtype, phi_ptr, ld, tile_scales_ptr=None):
    h = _P()
    _check(lib().cofem_op_dense(N, D, dtype, phi_ptr, ld, tile_scales_ptr, ctypes.byref(h)),
           "cofem_op_dense")
    return h


def cofem_op_dense_set_terms(op, nterms):
    _check(lib().cofem_op_dense_set_terms(op, nterms), "cofem_op_dense_set_terms")


def cofem_op_dense_set_l2_resident(op, nbytes):
    _check(lib().cofem_op_dense_set_l2_resident(op, nbytes), "cofem_op_dense_set_l2_resident")


def cofem_op_dense_set_tile_rows(op, rows):
    _check(lib().cofem_op_dense_set_tile_rows(op, rows), "cofem_op_dense_set_tile_rows")


def cofem_op_dense_get_pipeline(op):
    """(stages, ctas_per_sm, tile_rows) of a dense handle's tensor-core pipeline."""
    a, b, c = _I32(), _I32(), _I32()
    _check(lib().cofem_op_dense_get_pipeline(op, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(c)), "cofem_op_dense_get_pipeline")
    return a.value, b.value, c.value


def cofem_op_dense_set_pipeline(op, stages, ctas_per_sm):
    _check(lib().cofem_op_dense_set_pipeline(op, stages, ctas_per_sm),
           "cofem_op_dense_set_pipeline")


def cofem_op_dense_autotune_workspace_bytes(op, ncols):
    return lib().cofem_op_dense_autotune_workspace_bytes(op, ncols)


def cofem_op_dense_autotune(op, ncols, ws_ptr, ws_bytes, stream=0):
    """Returns (stages, ctas_per_sm, microseconds per application)."""
    st, cps, us = _I32(), _I32(), ctypes.c_float()
    _check(lib().cofem_op_dense_autotune(op, ncols, ws_ptr, ws_bytes, stream, ctypes.byref(st),
                                         ctypes.byref(cps), ctypes.byref(us)),
           "cofem_op_dense_autotune")
    return st.value, cps.value, us.value


def cofem_dense_packed_bytes(N, D):
    return lib().cofem_dense_packed_bytes(N, D)


def cofem_quantize_fp8_tiles(phi_ptr, N, D, ld, out_ptr, ld_out, scales_ptr, stream=0):
    _check(lib().cofem_quantize_fp8_tiles(phi_ptr, N, D, ld, out_ptr, ld_out, scales_ptr, stream),
           "cofem_quantize_fp8_tiles")


def cofem_op_dense_packed_bytes(op):
    return lib().cofem_op_dense_packed_bytes(op)


def cofem_op_dense_attach_packed(op, packed_ptr, nbytes, stream=0):
    _check(lib().cofem_op_dense_attach_packed(op, packed_ptr, nbytes, stream),
           "cofem_op_dense_attach_packed")


def cofem_op_conv1d(L, C, T, filters_ptr):
    h = _P()
    _check(lib().cofem_op_conv1d(L, C, T, filters_ptr, ctypes.byref(h)), "cofem_op_conv1d")
    return h


def cofem_op_conv1d_set_tensor_cores(op, on):
    _check(lib().cofem_op_conv1d_set_tensor_cores(op, on), "cofem_op_conv1d_set_tensor_cores")


def cofem_op_dct(D, N, idx_ptr):
    h = _P()
    _check(lib().cofem_op_dct(D, N, idx_ptr, ctypes.byref(h)), "cofem_op_dct")
    return h


def cofem_op_destroy(op):
    lib().cofem_op_destroy(op)


def cofem_op_shape(op):
    n, d = _I64(), _I64()
    _check(lib().cofem_op_shape(op, ctypes.byref(n), ctypes.byref(d)), "cofem_op_shape")
    return n.value, d.value


def cofem_params_default(**overrides):
    p = cofem_params()
    lib().cofem_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def cofem_workspace_bytes(op, params):
    n = _SZ()
    _check(lib().cofem_workspace_bytes(op, ctypes.byref(params), ctypes.byref(n)),
           "cofem_workspace_bytes")
    return n.value


def cofem_fit(op, y_ptr, beta, params, ws_ptr, ws_bytes, mu_ptr, s_ptr, alpha_ptr,
              stream=0, want_stats=True):
    """Runs Algorithm 1; returns a dict of per-EM-iteration statistics."""
    n = max(params.em_iters, 1)
    it = (ctypes.c_int32 * n)()
    rr = (ctypes.c_double * n)()
    cl = (ctypes.c_int32 * n)()
    sp = (ctypes.c_int32 * n)()
    en = (ctypes.c_int64 * n)()
    st = cofem_stats(it, rr, cl, sp, en)
    rc = lib().cofem_fit(op, y_ptr, beta, ctypes.byref(params), ws_ptr, ws_bytes, mu_ptr,
                         s_ptr, alpha_ptr, ctypes.byref(st) if want_stats else None, stream)
    _check(rc, "cofem_fit")
    m = params.em_iters
    return {"cg_iters": list(it)[:m], "relres": list(rr)[:m], "clamps": list(cl)[:m],
            "support": list(sp)[:m], "end_ns": list(en)[:m]}


def cofem_batched_workspace_bytes(problems, params):
    arr = (cofem_problem * len(problems))(*problems)
    n = _SZ()
    _check(lib().cofem_batched_workspace_bytes(len(problems), arr, ctypes.byref(params),
                                               ctypes.byref(n)), "cofem_batched_workspace_bytes")
    return n.value


def cofem_fit_batched(problems, params, ws_ptr, ws_bytes, mu_ptr, s_ptr, alpha_ptr, stream=0):
    """Returns per-problem statistics (lists of em_iters values per problem)."""
    nprob = len(problems)
    arr = (cofem_problem * nprob)(*problems)
    m = max(params.em_iters, 1) * nprob
    it = (ctypes.c_int32 * m)()
    rr = (ctypes.c_double * m)()
    cl = (ctypes.c_int32 * m)()
    sp = (ctypes.c_int32 * m)()
    st = cofem_stats(it, rr, cl, sp)
    _check(lib().cofem_fit_batched(nprob, arr, ctypes.byref(params), ws_ptr, ws_bytes, mu_ptr,
                                   s_ptr, alpha_ptr, ctypes.byref(st), stream),
           "cofem_fit_batched")
    e = params.em_iters

    def split(a):
        return [list(a)[i * e:(i + 1) * e] for i in range(nprob)]
    return {"cg_iters": split(it), "relres": split(rr), "clamps": split(cl), "support": split(sp)}


def cofem_probe_fill(seed, t, K, D, dtype, out_ptr, ld, stream=0):
    _check(lib().cofem_probe_fill(seed, t, K, D, dtype, out_ptr, ld, stream), "cofem_probe_fill")


def cofem_apply_workspace_bytes(op, vec, ncols):
    n = _SZ()
    _check(lib().cofem_apply_workspace_bytes(op, vec, ncols, ctypes.byref(n)),
           "cofem_apply_workspace_bytes")
    return n.value


def cofem_op_apply(op, vec, x_ptr, ld, ncols, alpha_ptr, beta, y_ptr, ws_ptr, ws_bytes,
                   stream=0):
    _check(lib().cofem_op_apply(op, vec, x_ptr, ld, ncols, alpha_ptr, beta, y_ptr, ws_ptr,
                                ws_bytes, stream), "cofem_op_apply")


def cofem_op_apply_timed(op, vec, x_ptr, ld, ncols, alpha_ptr, beta, y_ptr, ws_ptr, ws_bytes,
                         stream=0, max_kernels=8):
    """Runs cofem_op_apply and returns the per-kernel milliseconds."""
    ms = (ctypes.c_float * max_kernels)()
    n = _I32()
    _check(lib().cofem_op_apply_timed(op, vec, x_ptr, ld, ncols, alpha_ptr, beta, y_ptr, ws_ptr,
                                      ws_bytes, stream, ms, max_kernels, ctypes.byref(n)),
           "cofem_op_apply_timed")
    return list(ms)[:n.value]


def cofem_op_apply_noalloc(op, vec, x_ptr, ld, ncols, alpha_ptr, beta, y_ptr, stream=0):
    _check(lib().cofem_op_apply_noalloc(op, vec, x_ptr, ld, ncols, alpha_ptr, beta, y_ptr,
                                        stream), "cofem_op_apply_noalloc")


def cofem_noalloc_scratch_capacity():
    return lib().cofem_noalloc_scratch_capacity()


def cofem_bench_cg_kernels_workspace_bytes(D, ncols):
    return lib().cofem_bench_cg_kernels_workspace_bytes(D, ncols)


def cofem_bench_cg_kernels(D, ncols, reps, ws_ptr, ws_bytes, stream=0):
    """Mean milliseconds per launch (CG update, direction update, diag/M-step)
    and whether the update held the direction update (1.0) or not (0.0)."""
    ms = (ctypes.c_float * 4)()
    _check(lib().cofem_bench_cg_kernels(D, ncols, reps, ws_ptr, ws_bytes, stream, ms),
           "cofem_bench_cg_kernels")
    return tuple(ms)



def cofem_bench_bcg_kernels_workspace_bytes(D, ncols):
    return lib().cofem_bench_bcg_kernels_workspace_bytes(D, ncols)

def cofem_bench_bcg_kernels(D, ncols, reps, ws_ptr, ws_bytes, stream=0):
    """Mean milliseconds per launch of the block-CG passes: xi gram, v gram,
    row, and the three back to back."""
    ms = (ctypes.c_float * 4)()
    _check(lib().cofem_bench_bcg_kernels(D, ncols, reps, ws_ptr, ws_bytes, stream, ms),
           "cofem_bench_bcg_kernels")
    return tuple(ms)


def cofem_selftest_cg_update_workspace_bytes():
    return lib().cofem_selftest_cg_update_workspace_bytes()


def cofem_selftest_cg_update_timeout(limit_ns, ws_ptr, ws_bytes, stream=0):
    """Returns the status code (5 = the waits ran out, as expected)."""
    return lib().cofem_selftest_cg_update_timeout(limit_ns, ws_ptr, ws_bytes, stream)


def cofem_selftest_wait_timeout(limit_ns, stream=0):
    """Status code of the bounded-wait self-test (5 = the wait ran out)."""
    return lib().cofem_selftest_wait_timeout(limit_ns, stream)


def cofem_op_forward(op, vec, z_ptr, ldz, ncols, w_ptr, ldw, ws_ptr, ws_bytes, stream=0):
    _check(lib().cofem_op_forward(op, vec, z_ptr, ldz, ncols, w_ptr, ldw, ws_ptr, ws_bytes,
                                  stream), "cofem_op_forward")


def cofem_op_adjoint(op, vec, w_ptr, ldw, ncols, z_ptr, ldz, ws_ptr, ws_bytes, stream=0):
    _check(lib().cofem_op_adjoint(op, vec, w_ptr, ldw, ncols, z_ptr, ldz, ws_ptr, ws_bytes,
                                  stream), "cofem_op_adjoint")


def cofem_diag_mstep(seed, t, K, D, vec, x_ptr, ld, den_floor, support_threshold, mu_ptr,
                     s_ptr, alpha_ptr, counts_ptr=None, stream=0):
    _check(lib().cofem_diag_mstep(seed, t, K, D, vec, x_ptr, ld, den_floor, support_threshold,
                                  mu_ptr, s_ptr, alpha_ptr, counts_ptr, stream),
           "cofem_diag_mstep")


# ------------------------------------------------------------ learned path

def cofem_last_fit_fallbacks():
    return lib().cofem_last_fit_fallbacks()


def cofem_op_col_norms(op, out_ptr, stream=0):
    _check(lib().cofem_op_col_norms(op, out_ptr, stream), "cofem_op_col_norms")


def cofem_col_norms_workspace_bytes(op):
    n = _SZ()
    _check(lib().cofem_col_norms_workspace_bytes(op, ctypes.byref(n)),
           "cofem_col_norms_workspace_bytes")
    return n.value


def cofem_op_col_norms_ws(op, out_ptr, ws_ptr, ws_bytes, stream=0):
    _check(lib().cofem_op_col_norms_ws(op, out_ptr, ws_ptr, ws_bytes, stream),
           "cofem_op_col_norms_ws")


def cofem_mlp_features(alpha_ptr, pn2_ptr, beta, mu_prev_ptr, s_prev_ptr, D, U_ptr, stream=0):
    _check(lib().cofem_mlp_features(alpha_ptr, pn2_ptr, beta, mu_prev_ptr, s_prev_ptr, D, U_ptr,
                                    stream), "cofem_mlp_features")


def cofem_mlp_targets(alpha_ptr, pn2_ptr, beta, mu_ptr, s_ptr, D, Y_ptr, stream=0):
    _check(lib().cofem_mlp_targets(alpha_ptr, pn2_ptr, beta, mu_ptr, s_ptr, D, Y_ptr, stream),
           "cofem_mlp_targets")


def cofem_mlp_forward(w_ptr, wdtype, U_ptr, n, O_ptr, stream=0):
    _check(lib().cofem_mlp_forward(w_ptr, wdtype, U_ptr, n, O_ptr, stream), "cofem_mlp_forward")


def cofem_mlp_train_workspace_bytes(n):
    return lib().cofem_mlp_train_workspace_bytes(n)


def cofem_mlp_grad(w_ptr, wdtype, U_ptr, Y_ptr, n, grad_ptr, loss_ptr, ws_ptr, ws_bytes,
                   stream=0):
    _check(lib().cofem_mlp_grad(w_ptr, wdtype, U_ptr, Y_ptr, n, grad_ptr, loss_ptr, ws_ptr,
                                ws_bytes, stream), "cofem_mlp_grad")


def cofem_mlp_adam_step(master_ptr, m_ptr, v_ptr, wbf_ptr, U_ptr, Y_ptr, n, step, lr, ws_ptr,
                        ws_bytes, loss_ptr=None, stream=0):
    _check(lib().cofem_mlp_adam_step(master_ptr, m_ptr, v_ptr, wbf_ptr, U_ptr, Y_ptr, n, step,
                                     lr, ws_ptr, ws_bytes, loss_ptr, stream),
           "cofem_mlp_adam_step")
