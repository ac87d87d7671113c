"""Thin Python binding of the C ABI in include/acmhd_fr.h (ctypes).

The functions carry the same names as the C entry points and only marshal
arguments: torch tensors become device pointers, the current torch stream
becomes the cudaStream_t, non-zero status codes become FrError.  Every
step of the computation runs in the CUDA library; if the library is
missing, loading fails loudly (there is no fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libacmhd_fr.so")

FR_OK, FR_EINVAL, FR_ECUDA, FR_ENOCONV, FR_ENONFINITE, FR_ENOMEM = 0, -1, -2, -3, -4, -5
FR_F32, FR_F64, FR_DF64 = 32, 64, 65
FR_CORR_DG, FR_CORR_G2 = 0, 1
FR_GUESS_PREVIOUS, FR_GUESS_EXTRAPOLATE, FR_GUESS_MLP = 0, 1, 2
FR_SCHEDULE_AUTO, FR_SCHEDULE_TWO_KERNELS, FR_SCHEDULE_FUSED_STAGE = 0, 1, 3

EXPORTS = ["fr_create", "fr_destroy", "fr_layout", "fr_rhs", "fr_set_schedule", "fr_trace",
           "fr_rhs_volume",
           "fr_rhs_unfused", "fr_rhs_host",
           "fr_rk_step", "fr_check", "fr_strerror", "fr_last_error", "fr_rhs_static",
           "fr_pseudo_solve", "fr_dual_init", "fr_dual_step", "fr_dual_velocity", "fr_dual_copy",
           "fr_mlp_create", "fr_mlp_destroy", "fr_mlp_info", "fr_mlp_collect", "fr_mlp_loss_grad",
           "fr_mlp_train", "fr_mlp_predict", "fr_mlp_predict_for", "fr_mlp_params", "fr_gemm_bf16",
           "fr_mlp_train_step", "fr_mlp_save", "fr_mlp_load", "fr_fma_probe",
           "fr_pmg_create", "fr_pmg_destroy", "fr_pmg_set_cycle", "fr_pmg_set_dtau",
           "fr_pmg_solve", "fr_pmg_set_anderson", "fr_mlp_set_training",
           "fr_mlp_validation_loss", "fr_gemm_set_kernel", "fr_gemm_check",
           "fr_mlp_set_output_degree"]


class fr_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class fr_dual_opts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dtau", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int), ("guess", ctypes.c_int),
                ("refine", ctypes.c_void_p), ("U_refine", ctypes.c_void_p),
                ("tol_switch", ctypes.c_double), ("mlp", ctypes.c_void_p),
                ("pmg", ctypes.c_void_p), ("refine_pmg", ctypes.c_void_p)]


class fr_dual_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("iters_refine", ctypes.c_int), ("res", ctypes.c_double),
                ("res_switch", ctypes.c_double), ("guess_used", ctypes.c_int),
                ("res_guess", ctypes.c_double * 2), ("mlp_weight", ctypes.c_double),
                ("res_blend", ctypes.c_double)]


class FrError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib().fr_strerror(status).decode()} ({status})"
                         + (f" [{_lib().fr_last_error().decode()}]" if status == FR_ECUDA else ""))


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_2107_14027_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, sz, dbl, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_double, ctypes.c_int
        lib.fr_create.argtypes = [ctypes.POINTER(fr_mesh), i32, i32, dbl, dbl, dbl, i32, i32,
                                  ctypes.POINTER(vp)]
        lib.fr_destroy.argtypes = [vp]
        lib.fr_destroy.restype = None
        lib.fr_layout.argtypes = [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(sz)]
        for name in ("fr_rhs", "fr_rhs_volume", "fr_rhs_unfused", "fr_rhs_host"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp]
        lib.fr_trace.argtypes = [vp, vp, vp]
        lib.fr_set_schedule.argtypes = [vp, i32]
        lib.fr_rk_step.argtypes = [vp, vp, dbl, vp]
        lib.fr_rhs_static.argtypes = [ctypes.POINTER(fr_mesh), i32, i32, dbl, dbl, dbl, i32, i32,
                                      vp, vp, vp]
        lib.fr_check.argtypes = [vp, vp]
        ip, dp = ctypes.POINTER(i32), ctypes.POINTER(dbl)
        lib.fr_pseudo_solve.argtypes = [vp, vp, vp, vp, vp, dbl, i32, dbl, dbl, i32, i32, dbl, ip,
                                        dp, vp]
        lib.fr_dual_init.argtypes = [vp, vp, vp]
        lib.fr_dual_step.argtypes = [vp, vp, ctypes.POINTER(fr_dual_opts),
                                     ctypes.POINTER(fr_dual_stats), vp]
        lib.fr_dual_velocity.argtypes = [vp, vp, vp]
        lib.fr_dual_copy.argtypes = [vp, vp, vp]
        ull = ctypes.c_ulonglong
        lib.fr_mlp_create.argtypes = [vp, i32, i32, ull, ctypes.POINTER(vp)]
        lib.fr_mlp_destroy.argtypes = [vp]
        lib.fr_mlp_destroy.restype = None
        lib.fr_mlp_info.argtypes = [vp, ip, ip, ip, ip, ctypes.POINTER(sz)]
        lib.fr_mlp_collect.argtypes = [vp, i32, ull, ip, vp]
        lib.fr_mlp_loss_grad.argtypes = [vp, dp, vp]
        lib.fr_mlp_train.argtypes = [vp, i32, dbl, dp, vp]
        lib.fr_mlp_predict.argtypes = [vp, vp, vp, vp]
        lib.fr_mlp_predict_for.argtypes = [vp, vp, vp, vp, vp]
        lib.fr_mlp_params.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float), sz, i32]
        lib.fr_mlp_train_step.argtypes = [vp, dbl, dp, vp]
        lib.fr_fma_probe.argtypes = [i32, i32, vp, dp, vp]
        lib.fr_pmg_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
        lib.fr_pmg_destroy.argtypes = [vp]
        lib.fr_pmg_destroy.restype = None
        lib.fr_pmg_set_cycle.argtypes = [vp, i32, ip, ip]
        lib.fr_pmg_set_dtau.argtypes = [vp, dp, i32]
        lib.fr_pmg_set_anderson.argtypes = [vp, i32]
        lib.fr_mlp_set_training.argtypes = [vp, i32, dbl]
        lib.fr_mlp_validation_loss.argtypes = [vp, dp, vp]
        lib.fr_pmg_solve.argtypes = [vp, vp, vp, vp, vp, dbl, i32, dbl, dbl, i32, dbl, ip, dp, vp]
        lib.fr_mlp_save.argtypes = [vp, ctypes.c_char_p]
        lib.fr_mlp_load.argtypes = [vp, ctypes.c_char_p, i32, ctypes.POINTER(vp)]
        lib.fr_gemm_bf16.argtypes = [i32, i32, i32, i32, i32, vp, ctypes.c_longlong, vp,
                                     ctypes.c_longlong, vp, ctypes.c_longlong, vp]
        lib.fr_gemm_set_kernel.argtypes = [i32]
        lib.fr_mlp_set_output_degree.argtypes = [vp, i32]
        lib.fr_gemm_check.argtypes = [vp]
        lib.fr_strerror.argtypes = [i32]
        lib.fr_strerror.restype = ctypes.c_char_p
        lib.fr_last_error.argtypes = []
        lib.fr_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("fr_destroy", "fr_strerror", "fr_last_error", "fr_mlp_destroy",
                            "fr_pmg_destroy"):
                getattr(lib, name).restype = i32
        _LIB = lib
    return _LIB


def _check(status, where):
    if status != FR_OK:
        raise FrError(status, where)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def make_mesh(n, lo, hi):
    d = len(n)
    m = fr_mesh()
    m.dim = d
    for a in range(3):
        m.n[a] = int(n[a]) if a < d else 1
        m.lo[a] = float(lo[a]) if a < d else 0.0
        m.hi[a] = float(hi[a]) if a < d else 1.0
    return m


def fr_create(n, lo, hi, order, nvars, zeta, nu, t_r, precision=FR_F32, correction=FR_CORR_DG):
    """Returns an opaque context handle (int)."""
    mesh = make_mesh(n, lo, hi)
    out = ctypes.c_void_p()
    _check(_lib().fr_create(ctypes.byref(mesh), int(order), int(nvars), float(zeta), float(nu),
                            float(t_r), int(precision), int(correction), ctypes.byref(out)),
           "fr_create")
    return out.value


def fr_create_raw(mesh, order, nvars, zeta, nu, t_r, precision, correction):
    """fr_create on a prepared fr_mesh (or None); returns (status, handle)."""
    out = ctypes.c_void_p()
    st = _lib().fr_create(ctypes.byref(mesh) if mesh is not None else None, int(order), int(nvars),
                          float(zeta), float(nu), float(t_r), int(precision), int(correction),
                          ctypes.byref(out))
    return st, out.value


def fr_destroy(ctx):
    _lib().fr_destroy(ctypes.c_void_p(ctx))


def fr_layout(ctx):
    """(elem_stride, n_elem, bytes_per_state)"""
    s, n, b = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib().fr_layout(ctypes.c_void_p(ctx), ctypes.byref(s), ctypes.byref(n), ctypes.byref(b)),
           "fr_layout")
    return s.value, n.value, b.value


def fr_rhs(ctx, U, R, stream=None):
    _check(_lib().fr_rhs(ctypes.c_void_p(ctx), _ptr(U), _ptr(R), _stream(stream)), "fr_rhs")


def fr_set_schedule(ctx, schedule):
    _check(_lib().fr_set_schedule(ctypes.c_void_p(ctx), int(schedule)), "fr_set_schedule")


def fr_trace(ctx, U, stream=None):
    _check(_lib().fr_trace(ctypes.c_void_p(ctx), _ptr(U), _stream(stream)), "fr_trace")


def fr_rhs_volume(ctx, U, R, stream=None):
    _check(_lib().fr_rhs_volume(ctypes.c_void_p(ctx), _ptr(U), _ptr(R), _stream(stream)),
           "fr_rhs_volume")


def fr_rhs_unfused(ctx, U, R, stream=None):
    _check(_lib().fr_rhs_unfused(ctypes.c_void_p(ctx), _ptr(U), _ptr(R), _stream(stream)),
           "fr_rhs_unfused")


def fr_rhs_host(ctx, U_host, R_host, stream=None):
    """U_host, R_host: CPU torch tensors (pinned for speed) or numpy arrays."""
    def hp(x):
        if isinstance(x, np.ndarray):
            return ctypes.c_void_p(x.ctypes.data)
        return ctypes.c_void_p(x.data_ptr())
    _check(_lib().fr_rhs_host(ctypes.c_void_p(ctx), hp(U_host), hp(R_host), _stream(stream)),
           "fr_rhs_host")


def fr_rhs_static(n, lo, hi, order, nvars, zeta, nu, t_r, precision, correction, U, R,
                  stream=None):
    """fr_rhs without a context and without any device allocation (the face
    traces live in the library's fixed 16 MiB device array)."""
    mesh = make_mesh(n, lo, hi)
    _check(_lib().fr_rhs_static(ctypes.byref(mesh), int(order), int(nvars), float(zeta),
                                float(nu), float(t_r), int(precision), int(correction), _ptr(U),
                                _ptr(R), _stream(stream)), "fr_rhs_static")


def fr_last_error():
    return _lib().fr_last_error().decode()


def fr_rk_step(ctx, U, dtau, stream=None):
    _check(_lib().fr_rk_step(ctypes.c_void_p(ctx), _ptr(U), float(dtau), _stream(stream)),
           "fr_rk_step")


def fr_pseudo_solve(ctx, U, V, Vn, Vnm1, dt, bdf_order, dtau, tol, max_iter, check_every=1,
                    stall=0.0, stream=None, allow_noconv=False):
    """Returns (status, iterations, residual).  FR_ENOCONV raises unless
    allow_noconv is set."""
    it, res = ctypes.c_int(), ctypes.c_double()
    st = _lib().fr_pseudo_solve(ctypes.c_void_p(ctx), _ptr(U), _ptr(V), _ptr(Vn),
                                _ptr(Vnm1) if Vnm1 is not None else None, float(dt),
                                int(bdf_order), float(dtau), float(tol), int(max_iter),
                                int(check_every), float(stall), ctypes.byref(it),
                                ctypes.byref(res), _stream(stream))
    if not (st == FR_OK or (allow_noconv and st == FR_ENOCONV)):
        _check(st, "fr_pseudo_solve")
    return st, it.value, res.value


def fr_pmg_create(ctx, coarsest_order=1):
    out = ctypes.c_void_p()
    _check(_lib().fr_pmg_create(ctypes.c_void_p(ctx), int(coarsest_order), ctypes.byref(out)),
           "fr_pmg_create")
    return out.value


def fr_pmg_destroy(pmg):
    _lib().fr_pmg_destroy(ctypes.c_void_p(pmg))


def fr_pmg_set_cycle(pmg, schedule):
    """schedule: list of (order, iterations)."""
    n = len(schedule)
    orders = (ctypes.c_int * n)(*[int(o) for o, _ in schedule])
    iters = (ctypes.c_int * n)(*[int(k) for _, k in schedule])
    _check(_lib().fr_pmg_set_cycle(ctypes.c_void_p(pmg), n, orders, iters), "fr_pmg_set_cycle")


def fr_pmg_set_dtau(pmg, factors=None, implicit=True):
    """factors: {order: multiplier} or None (keep)."""
    arr = None
    if factors is not None:
        vals = [1.0] * 8
        for q, f in factors.items():
            vals[int(q)] = float(f)
        arr = (ctypes.c_double * 8)(*vals)
    _check(_lib().fr_pmg_set_dtau(ctypes.c_void_p(pmg), arr, int(bool(implicit))),
           "fr_pmg_set_dtau")


def fr_pmg_set_anderson(pmg, memory):
    _check(_lib().fr_pmg_set_anderson(ctypes.c_void_p(pmg), int(memory)), "fr_pmg_set_anderson")


def fr_pmg_solve(pmg, U, V, Vn, Vnm1, dt, bdf_order, dtau, tol, max_cycles, stall=0.0,
                 stream=None, allow_noconv=False):
    """Returns (status, cycles, residual)."""
    cyc, res = ctypes.c_int(), ctypes.c_double()
    st = _lib().fr_pmg_solve(ctypes.c_void_p(pmg), _ptr(U), _ptr(V), _ptr(Vn),
                             _ptr(Vnm1) if Vnm1 is not None else None, float(dt), int(bdf_order),
                             float(dtau), float(tol), int(max_cycles), float(stall),
                             ctypes.byref(cyc), ctypes.byref(res), _stream(stream))
    if not (st == FR_OK or (allow_noconv and st == FR_ENOCONV)):
        _check(st, "fr_pmg_solve")
    return st, cyc.value, res.value


def fr_dual_init(ctx, U, stream=None):
    _check(_lib().fr_dual_init(ctypes.c_void_p(ctx), _ptr(U), _stream(stream)), "fr_dual_init")


def fr_dual_step(ctx, U, dt, dtau, tol, max_iter, check_every=1, guess=FR_GUESS_EXTRAPOLATE,
                 refine=None, U_refine=None, tol_switch=0.0, mlp=None, stream=None,
                 allow_noconv=False, pmg=None, refine_pmg=None):
    """Returns (status, fr_dual_stats)."""
    opts = fr_dual_opts(float(dt), float(dtau), float(tol), int(max_iter), int(check_every),
                        int(guess), refine, U_refine.data_ptr() if U_refine is not None else None,
                        float(tol_switch), mlp, pmg, refine_pmg)
    stats = fr_dual_stats()
    st = _lib().fr_dual_step(ctypes.c_void_p(ctx), _ptr(U), ctypes.byref(opts),
                             ctypes.byref(stats), _stream(stream))
    if not (st == FR_OK or (allow_noconv and st == FR_ENOCONV)):
        _check(st, "fr_dual_step")
    return st, stats


def fr_dual_copy(dst, src, stream=None):
    _check(_lib().fr_dual_copy(ctypes.c_void_p(dst), ctypes.c_void_p(src), _stream(stream)),
           "fr_dual_copy")


def fr_dual_velocity(ctx, V, stream=None):
    _check(_lib().fr_dual_velocity(ctypes.c_void_p(ctx), _ptr(V), _stream(stream)),
           "fr_dual_velocity")


def new_velocity(ctx, dim, order, device="cuda"):
    """FP64 velocity rows of a state: d * (p+1)^d rows of elem_stride."""
    import torch
    stride, _, _ = fr_layout(ctx)
    return torch.zeros((dim * (order + 1) ** dim, stride), dtype=torch.float64, device=device)


def velocity_rows(U, dim, npts):
    """The velocity rows of a packed state tensor (a view)."""
    return U[npts:(1 + dim) * npts]


def fr_mlp_create(ctx, hidden, capacity, seed):
    out = ctypes.c_void_p()
    _check(_lib().fr_mlp_create(ctypes.c_void_p(ctx), int(hidden), int(capacity), int(seed),
                                ctypes.byref(out)), "fr_mlp_create")
    return out.value


def fr_mlp_destroy(mlp):
    _lib().fr_mlp_destroy(ctypes.c_void_p(mlp))


def fr_mlp_info(mlp):
    """(n_in, hidden, n_out, n_samples, n_params)"""
    a, b_, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    e = ctypes.c_size_t()
    _check(_lib().fr_mlp_info(ctypes.c_void_p(mlp), ctypes.byref(a), ctypes.byref(b_),
                              ctypes.byref(c), ctypes.byref(d), ctypes.byref(e)), "fr_mlp_info")
    return a.value, b_.value, c.value, d.value, e.value


def fr_mlp_collect(mlp, count, seed, stream=None):
    """Returns the sampled element indices (numpy int32)."""
    el = np.zeros(count, dtype=np.int32)
    _check(_lib().fr_mlp_collect(ctypes.c_void_p(mlp), int(count), int(seed),
                                 el.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _stream(stream)),
           "fr_mlp_collect")
    return el


def fr_mlp_loss_grad(mlp, stream=None):
    loss = ctypes.c_double()
    _check(_lib().fr_mlp_loss_grad(ctypes.c_void_p(mlp), ctypes.byref(loss), _stream(stream)),
           "fr_mlp_loss_grad")
    return loss.value


def fr_mlp_train(mlp, epochs, lr, stream=None):
    loss = ctypes.c_double()
    _check(_lib().fr_mlp_train(ctypes.c_void_p(mlp), int(epochs), float(lr), ctypes.byref(loss),
                               _stream(stream)), "fr_mlp_train")
    return loss.value


def fr_mlp_set_training(mlp, n_val=0, weight_decay=0.0):
    _check(_lib().fr_mlp_set_training(ctypes.c_void_p(mlp), int(n_val), float(weight_decay)),
           "fr_mlp_set_training")


def fr_mlp_validation_loss(mlp, stream=None):
    loss = ctypes.c_double()
    _check(_lib().fr_mlp_validation_loss(ctypes.c_void_p(mlp), ctypes.byref(loss),
                                         _stream(stream)), "fr_mlp_validation_loss")
    return loss.value


def fr_mlp_train_step(mlp, lr, stream=None):
    loss = ctypes.c_double()
    _check(_lib().fr_mlp_train_step(ctypes.c_void_p(mlp), float(lr), ctypes.byref(loss),
                                    _stream(stream)), "fr_mlp_train_step")
    return loss.value


def fr_mlp_save(mlp, path):
    _check(_lib().fr_mlp_save(ctypes.c_void_p(mlp), os.fsencode(path)), "fr_mlp_save")


def fr_mlp_load(ctx, path, capacity=1):
    out = ctypes.c_void_p()
    _check(_lib().fr_mlp_load(ctypes.c_void_p(ctx), os.fsencode(path), int(capacity),
                              ctypes.byref(out)), "fr_mlp_load")
    return out.value


def fr_mlp_predict(mlp, U, V, stream=None):
    _check(_lib().fr_mlp_predict(ctypes.c_void_p(mlp), _ptr(U), _ptr(V), _stream(stream)),
           "fr_mlp_predict")


def fr_mlp_predict_for(mlp, ctx, U, V, stream=None):
    _check(_lib().fr_mlp_predict_for(ctypes.c_void_p(mlp), ctypes.c_void_p(ctx), _ptr(U), _ptr(V),
                                     _stream(stream)), "fr_mlp_predict_for")


def fr_mlp_params(mlp, which, values=None, count=None):
    """Get (values None) or set the parameters (0), gradients (1) or scales (2)."""
    if values is None:
        out = np.zeros(int(count), dtype=np.float32)
        _check(_lib().fr_mlp_params(ctypes.c_void_p(mlp), int(which),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size, 0),
               "fr_mlp_params")
        return out
    v = np.ascontiguousarray(values, dtype=np.float32)
    _check(_lib().fr_mlp_params(ctypes.c_void_p(mlp), int(which),
                                v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), v.size, 1),
           "fr_mlp_params")


def fr_gemm_bf16(amode, bmode, N, M, K, A, lda, B, ldb, C, ldc, stream=None):
    _check(_lib().fr_gemm_bf16(int(amode), int(bmode), int(N), int(M), int(K), _ptr(A), int(lda),
                               _ptr(B), int(ldb), _ptr(C), int(ldc), _stream(stream)),
           "fr_gemm_bf16")


def fr_mlp_set_output_degree(mlp, degree):
    _check(_lib().fr_mlp_set_output_degree(ctypes.c_void_p(mlp), int(degree)),
           "fr_mlp_set_output_degree")


FR_GEMM_AUTO, FR_GEMM_MMA_SYNC = 0, 1


def fr_gemm_set_kernel(kind):
    _check(_lib().fr_gemm_set_kernel(int(kind)), "fr_gemm_set_kernel")


def fr_gemm_check(stream=None):
    _check(_lib().fr_gemm_check(_stream(stream)), "fr_gemm_check")


def fr_fma_probe(precision, iters, out, stream=None):
    """Launches the FMA peak probe; returns the FLOPs the launch performs."""
    flops = ctypes.c_double()
    _check(_lib().fr_fma_probe(int(precision), int(iters), _ptr(out), ctypes.byref(flops),
                               _stream(stream)), "fr_fma_probe")
    return flops.value


def fr_check(ctx, stream=None):
    _check(_lib().fr_check(ctypes.c_void_p(ctx), _stream(stream)), "fr_check")


def fr_strerror(status):
    return _lib().fr_strerror(int(status)).decode()


# ---------------------------------------------------------------------------
# layout marshalling (padding of the element axis only)
# ---------------------------------------------------------------------------

def torch_dtype(precision):
    import torch
    return torch.float32 if precision == FR_F32 else torch.float64


def new_state(ctx, precision, device="cuda", fill=0.0):
    import torch
    stride, ne, nbytes = fr_layout(ctx)
    esz = 4 if precision == FR_F32 else 8
    rows = nbytes // (esz * stride)
    return torch.full((rows, stride), fill, dtype=torch_dtype(precision), device=device)


def pack_state(ctx, U, precision, device="cuda"):
    """[nv, npts, ne] numpy -> padded [nv*npts, stride] torch tensor on device."""
    import torch
    stride, ne, _ = fr_layout(ctx)
    nv, npts, ne_in = U.shape
    assert ne_in == ne
    host = np.zeros((nv * npts, stride), dtype=np.float32 if precision == FR_F32 else np.float64)
    host[:, :ne] = U.reshape(nv * npts, ne)
    return torch.from_numpy(host).to(device)


def unpack_state(ctx, T, nv):
    """padded device tensor -> [nv, npts, ne] numpy FP64."""
    stride, ne, _ = fr_layout(ctx)
    A = T.detach().cpu().numpy().astype(np.float64)
    return A[:, :ne].reshape(nv, -1, ne)
