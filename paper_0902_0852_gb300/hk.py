"""Thin Python binding of libhk (include/hk.h): argument marshalling only.

Every step of the factorisation and of inverse iteration runs in the CUDA
library; this module converts Python integers / numpy arrays / torch tensors to
the flat C-ABI arrays and back.  It raises ``HKError`` for any non-zero status
and ``RuntimeError`` when the compiled library is missing — there is no
fallback.

Values are exchanged as pairs ``(n, e)`` of Python ints meaning ``n * 2**e``
(|n| a P-bit mantissa or 0), the same convention as the oracle.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HK_CHECKED=1 selects the diagnosis build (device bounds checks, a
# synchronisation after every launch); see build.py
_LIB_PATH = os.path.join(_HERE, "libhk_checked.so" if os.environ.get("HK_CHECKED") == "1" else "libhk.so")
_lib = None

HK_OK, HK_ERR_ARG, HK_ERR_NOT_PD, HK_ERR_CUDA, HK_ERR_OOM, HK_ERR_TIMEOUT, HK_ERR_STATE, HK_ERR_RANGE = range(8)

EXPORTS = [
    "hk_create", "hk_destroy", "hk_strerror", "hk_workspace_bytes", "hk_set_workspace",
    "hk_load_moments", "hk_load_moments_flat", "hk_factor", "hk_get_R", "hk_get_R_flat",
    "hk_smallest_eig", "hk_get_history_flat", "hk_get_timings", "hk_get_stats", "hk_selftest_mp",
    "hk_probe_int_peaks", "hk_mp_op_noalloc", "hk_set_update_path",
    "hk_set_option", "hk_batch_solve",
    "hk_mlp_workspace_bytes", "hk_mlp_forward", "hk_mlp_loss_grad", "hk_mlp_adam", "hk_mlp_train",
    "hk_set_predictor", "hk_predict", "hk_update_plan", "hk_selftest_wait",
    "hk_ldlt_det", "hk_get_ldlt_flat", "hk_secant", "hk_get_secant_flat", "hk_secant_verify",
    "hk_time_update_slice", "hk_selftest_scalar",
]


class HKError(RuntimeError):
    def __init__(self, code, what, extra=None):
        self.code = code
        self.extra = extra
        msg = lib().hk_strerror(code).decode()
        super().__init__(f"{what}: {msg} (status {code})" + (f" [{extra}]" if extra is not None else ""))


class HkMp(ctypes.Structure):
    _fields_ = [("sign", ctypes.c_int32), ("exp", ctypes.c_int64), ("limbs", ctypes.POINTER(ctypes.c_uint32))]


def lib():
    """The loaded libhk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libhk.so not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        P32, P64, PU32 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint32)
        L.hk_create.argtypes = [ctypes.POINTER(vp), i32, vp]
        L.hk_destroy.argtypes = [vp]
        L.hk_destroy.restype = None
        L.hk_strerror.argtypes = [i32]
        L.hk_strerror.restype = ctypes.c_char_p
        L.hk_workspace_bytes.argtypes = [i32, i32, ctypes.POINTER(sz)]
        L.hk_set_workspace.argtypes = [vp, vp, sz]
        L.hk_load_moments.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(HkMp)]
        L.hk_load_moments_flat.argtypes = [vp, i32, i32, i32, i32, vp, vp, vp, i32]
        L.hk_factor.argtypes = [vp, ctypes.POINTER(i32)]
        L.hk_get_R.argtypes = [vp, ctypes.POINTER(HkMp)]
        L.hk_get_R_flat.argtypes = [vp, vp, vp, vp]
        L.hk_smallest_eig.argtypes = [vp, i32, ctypes.POINTER(HkMp), ctypes.POINTER(i32)]
        L.hk_get_history_flat.argtypes = [vp, i32, vp, vp, vp]
        L.hk_get_timings.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
        L.hk_get_stats.argtypes = [vp, P64, i32]
        L.hk_selftest_mp.argtypes = [i32, i32, PU32, i32, i64, PU32, i32, i64, PU32, P64]
        L.hk_probe_int_peaks.argtypes = [i32, ctypes.POINTER(ctypes.c_double), i32]
        L.hk_mp_op_noalloc.argtypes = [i32, i32, vp, i32, i64, vp, i32, i64, vp, vp, vp]
        L.hk_set_update_path.argtypes = [vp, i32]
        L.hk_set_option.argtypes = [vp, i32, i64]
        L.hk_batch_solve.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp]
        f32 = ctypes.c_float
        L.hk_mlp_workspace_bytes.argtypes = [i32]
        L.hk_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
        L.hk_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, sz, vp]
        L.hk_mlp_adam.argtypes = [vp, vp, vp, vp, i32, i32, f32, f32, f32, f32, vp]
        L.hk_mlp_train.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, f32, f32, f32, f32, vp, vp, sz, vp]
        L.hk_set_predictor.argtypes = [vp, vp, vp]
        L.hk_predict.argtypes = [vp, i32, vp, vp, vp]
        L.hk_update_plan.argtypes = [i32, i32, P64, P32, P32, P32, P32, i64, P32]
        L.hk_selftest_wait.argtypes = [vp]
        L.hk_ldlt_det.argtypes = [vp, ctypes.POINTER(HkMp), ctypes.POINTER(HkMp), ctypes.POINTER(i32),
                                  ctypes.POINTER(i32)]
        L.hk_get_ldlt_flat.argtypes = [vp, i32, vp, vp, vp]
        L.hk_secant.argtypes = [vp, i32, ctypes.POINTER(HkMp), ctypes.POINTER(i32)]
        L.hk_get_secant_flat.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp]
        L.hk_secant_verify.argtypes = [vp, ctypes.POINTER(HkMp), i32, i32, ctypes.POINTER(i32)]
        L.hk_time_update_slice.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.hk_selftest_scalar.argtypes = [i32, i32, ctypes.POINTER(HkMp), ctypes.POINTER(HkMp), ctypes.POINTER(HkMp),
                                         ctypes.POINTER(i32)]
        for name in EXPORTS:
            getattr(L, name).restype = getattr(L, name).restype if name in ("hk_destroy", "hk_strerror") else i32
        L.hk_mlp_workspace_bytes.restype = sz
        _lib = L
    return _lib


def _check(code, what, extra=None):
    if code != HK_OK:
        raise HKError(code, what, extra)


# ---------------------------------------------------------------------------
# marshalling of P-bit values
# ---------------------------------------------------------------------------

def pack(values, P):
    """(n, e) pairs -> (sign int32[k], exp int64[k], limbs uint32[k, L])."""
    L = P // 32
    k = len(values)
    sign = np.zeros(k, dtype=np.int32)
    exp = np.zeros(k, dtype=np.int64)
    buf = bytearray(4 * L * k)
    for idx, (n, e) in enumerate(values):
        if n == 0:
            continue
        a = -n if n < 0 else n
        if a.bit_length() != P:
            raise ValueError("mantissa is not normalised to P bits")
        sign[idx] = 1 if n < 0 else 0
        exp[idx] = e
        buf[4 * L * idx: 4 * L * (idx + 1)] = a.to_bytes(4 * L, "little")
    limbs = np.frombuffer(bytes(buf), dtype=np.uint32).reshape(k, L).copy()
    return sign, exp, limbs


def unpack(sign, exp, limbs):
    """Inverse of ``pack``."""
    limbs = np.ascontiguousarray(limbs, dtype=np.uint32)
    out = []
    raw = limbs.tobytes()
    L = limbs.shape[-1]
    for idx in range(len(sign)):
        a = int.from_bytes(raw[4 * L * idx: 4 * L * (idx + 1)], "little")
        if a == 0:
            out.append((0, 0))
        else:
            out.append((-a if sign[idx] else a, int(exp[idx])))
    return out


def _ptr(a):
    if hasattr(a, "data_ptr"):  # torch tensor (device memory)
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# C-ABI mirrors
# ---------------------------------------------------------------------------

def hk_create(device=0, stream=None):
    """``hk_create``; ``stream`` is a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    h = ctypes.c_void_p()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    _check(lib().hk_create(ctypes.byref(h), device, ctypes.c_void_p(s)), "hk_create")
    return h


def hk_destroy(ctx):
    lib().hk_destroy(ctx)


def hk_workspace_bytes(N, P):
    b = ctypes.c_size_t()
    _check(lib().hk_workspace_bytes(N, P, ctypes.byref(b)), "hk_workspace_bytes")
    return b.value


def hk_set_workspace(ctx, tensor):
    """Use a caller-owned device buffer (e.g. a torch uint8 CUDA tensor)."""
    _check(lib().hk_set_workspace(ctx, ctypes.c_void_p(tensor.data_ptr()), tensor.numel() * tensor.element_size()),
           "hk_set_workspace")


def hk_load_moments_flat(ctx, N, beta, P, sign, exp, limbs, on_device=False):
    p, q = beta
    _check(lib().hk_load_moments_flat(ctx, N, p, q, P, _ptr(sign), _ptr(exp), _ptr(limbs), 1 if on_device else 0),
           "hk_load_moments_flat")


def hk_load_moments(ctx, N, beta, P, moments):
    """Host moments as (n, e) pairs through the struct-array entry point."""
    sign, exp, limbs = pack(moments, P)
    arr = (HkMp * len(moments))()
    for k in range(len(moments)):
        arr[k].sign = int(sign[k])
        arr[k].exp = int(exp[k])
        arr[k].limbs = limbs[k].ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    p, q = beta
    _check(lib().hk_load_moments(ctx, N, p, q, P, arr), "hk_load_moments")


def hk_factor(ctx):
    bad = ctypes.c_int(-1)
    code = lib().hk_factor(ctx, ctypes.byref(bad))
    if code == HK_ERR_NOT_PD:
        raise HKError(code, "hk_factor", extra={"bad_row": bad.value})
    _check(code, "hk_factor")


def hk_get_R_flat(ctx, N, P):
    L = P // 32
    nt = N * (N + 1) // 2
    sign = np.zeros(nt, dtype=np.int32)
    exp = np.zeros(nt, dtype=np.int64)
    limbs = np.zeros((nt, L), dtype=np.uint32)
    _check(lib().hk_get_R_flat(ctx, _ptr(sign), _ptr(exp), _ptr(limbs)), "hk_get_R_flat")
    return sign, exp, limbs


def hk_get_R(ctx, N, P):
    """R as rows of (n, e): ``R[t][j - t]`` = R_tj, like the oracle."""
    vals = unpack(*hk_get_R_flat(ctx, N, P))
    rows, k = [], 0
    for t in range(N):
        rows.append(vals[k:k + N - t])
        k += N - t
    return rows


def hk_smallest_eig(ctx, P, iters):
    L = P // 32
    limbs = np.zeros(L, dtype=np.uint32)
    m = HkMp(0, 0, limbs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    used = ctypes.c_int(0)
    _check(lib().hk_smallest_eig(ctx, iters, ctypes.byref(m), ctypes.byref(used)), "hk_smallest_eig")
    return unpack(np.array([m.sign]), np.array([m.exp]), limbs.reshape(1, L))[0], used.value


def hk_get_history_flat(ctx, count, P):
    L = P // 32
    sign = np.zeros(count, dtype=np.int32)
    exp = np.zeros(count, dtype=np.int64)
    limbs = np.zeros((count, L), dtype=np.uint32)
    _check(lib().hk_get_history_flat(ctx, count, _ptr(sign), _ptr(exp), _ptr(limbs)), "hk_get_history_flat")
    return unpack(sign, exp, limbs)


def hk_get_timings(ctx):
    out = (ctypes.c_double * 5)()
    _check(lib().hk_get_timings(ctx, out, 5), "hk_get_timings")
    keys = ["update_ms", "panel_ms", "solve_ms", "factor_ms", "eig_ms"]
    return dict(zip(keys, list(out)))


def hk_get_stats(ctx):
    out = (ctypes.c_int64 * 11)()
    _check(lib().hk_get_stats(ctx, out, 11), "hk_get_stats")
    return {"launches": out[0], "W": out[1], "widenings": out[2], "karatsuba_levels": out[3],
            "limbprod_per_mac": out[4], "converged": out[5], "solve_wv_max": out[6], "solve_wv_mean": out[7],
            "resumes": out[8], "solve_prepared_used": out[9], "solve_prepared_dropped": out[10]}


def hk_selftest_mp(op, L, x, ex=0, y=None, ey=0):
    """Run one device multiprecision operation on Python-int operands.
    op 0: x*y; 1: floor(2^(2P+1)/x); 2: RNE sqrt(x 2^ex); 3: RNE (x 2^ex)/(y 2^ey);
    4: RNE(x 2^ex) (x an nx-limb integer).  Returns an int, or (mantissa, exp)."""
    def limbs_of(v, n):
        return np.frombuffer(v.to_bytes(4 * n, "little"), dtype=np.uint32).copy()
    nx = max(1, (x.bit_length() + 31) // 32) if op in (0, 4) else L
    xa = limbs_of(x, nx)
    ny = 0
    ya = np.zeros(1, dtype=np.uint32)
    if y is not None:
        ny = max(1, (y.bit_length() + 31) // 32) if op == 0 else L
        ya = limbs_of(y, ny)
    nout = {0: nx + ny + 2, 1: L + 2}.get(op, L)
    out = np.zeros(max(nout, 1) + 8, dtype=np.uint32)
    eo = np.zeros(2, dtype=np.int64)
    PU32 = ctypes.POINTER(ctypes.c_uint32)
    code = lib().hk_selftest_mp(op, L, xa.ctypes.data_as(PU32), nx, ex, ya.ctypes.data_as(PU32), ny, ey,
                                out.ctypes.data_as(PU32), eo.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    _check(code, "hk_selftest_mp")
    if eo[1]:
        raise HKError(HK_ERR_TIMEOUT, "hk_selftest_mp correction did not settle")
    val = int.from_bytes(out[:nout].tobytes(), "little")
    if op in (0, 1):
        return val
    return val, int(eo[0])


def hk_probe_int_peaks(device=0):
    """Measured integer rates per clock per SM (see include/hk.h)."""
    out = (ctypes.c_double * 6)()
    _check(lib().hk_probe_int_peaks(device, out, 6), "hk_probe_int_peaks")
    return {"imad_per_clk_sm": out[0], "imad_mhz": out[1], "limbprod_per_clk_sm": out[2],
            "limbprod_mhz": out[3], "mma_u8_mac_per_clk_sm": out[4], "mma_mhz": out[5]}


def hk_mp_op_noalloc(op, L, x, ex, y, ey, out, eo, stream=None):
    """Allocation-free device operation: x, y, out, eo are CUDA tensors
    (uint32 limbs viewed as int32, eo int64[2]); asynchronous on ``stream``."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    nx = x.numel()
    ny = 0 if y is None else y.numel()
    yp = ctypes.c_void_p(y.data_ptr()) if y is not None else ctypes.c_void_p(0)
    _check(lib().hk_mp_op_noalloc(op, L, ctypes.c_void_p(x.data_ptr()), nx, ex, yp, ny, ey,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(eo.data_ptr()),
                                  ctypes.c_void_p(s)), "hk_mp_op_noalloc")


(HK_OPT_UPDATE_PATH, HK_OPT_KARATSUBA, HK_OPT_GRAPH, HK_OPT_AUTOTUNE, HK_OPT_PANEL_ROWS, HK_OPT_MAX_ITERS,
 HK_OPT_WAIT_NS, HK_OPT_LOOKAHEAD) = range(8)


def hk_set_option(ctx, option, value):
    _check(lib().hk_set_option(ctx, option, int(value)), "hk_set_option")


def hk_selftest_wait(ctx):
    """Status of the bounded-wait self-test (HK_ERR_TIMEOUT when the wait ran
    out as designed); returned, not raised."""
    return lib().hk_selftest_wait(ctx)


def hk_batch_solve(ctx, instances, iters=0, nthreads=16):
    """instances: list of (N, (p, q), P, moments).  Returns a list of
    (status, lambda (n, e) or None, iterations used)."""
    count = len(instances)
    Ns = np.array([x[0] for x in instances], dtype=np.int32)
    bn = np.array([x[1][0] for x in instances], dtype=np.int32)
    bd = np.array([x[1][1] for x in instances], dtype=np.int32)
    Ps = np.array([x[2] for x in instances], dtype=np.int32)
    keep = []
    mom_ptrs = (ctypes.POINTER(HkMp) * count)()
    lam = (HkMp * count)()
    lam_limbs = []
    for k, (N, beta, P, moments) in enumerate(instances):
        sign, exp, limbs = pack(moments, P)
        arr = (HkMp * len(moments))()
        for i in range(len(moments)):
            arr[i].sign = int(sign[i])
            arr[i].exp = int(exp[i])
            arr[i].limbs = limbs[i].ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        keep.append((limbs, arr))
        mom_ptrs[k] = ctypes.cast(arr, ctypes.POINTER(HkMp))
        ll = np.zeros(P // 32, dtype=np.uint32)
        lam_limbs.append(ll)
        lam[k].limbs = ll.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    status = np.zeros(count, dtype=np.int32)
    used = np.zeros(count, dtype=np.int32)
    _check(lib().hk_batch_solve(ctx, count, _ptr(Ns), _ptr(bn), _ptr(bd), _ptr(Ps),
                                ctypes.cast(mom_ptrs, ctypes.c_void_p), iters, nthreads,
                                ctypes.cast(lam, ctypes.c_void_p), _ptr(status), _ptr(used)), "hk_batch_solve")
    out = []
    for k in range(count):
        if status[k] == HK_OK:
            v = unpack(np.array([lam[k].sign]), np.array([lam[k].exp]), lam_limbs[k].reshape(1, -1))[0]
        else:
            v = None
        out.append((int(status[k]), v, int(used[k])))
    return out


def _mp_in(v, P):
    """(n, e) -> HkMp with its limbs array (kept alive by the caller)."""
    L = P // 32
    n, e = v
    a = -n if n < 0 else n
    limbs = np.frombuffer(a.to_bytes(4 * L, "little"), dtype=np.uint32).copy()
    return HkMp(1 if n < 0 else 0, e if n else 0, limbs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), limbs


def _mp_out(P):
    L = P // 32
    limbs = np.zeros(L, dtype=np.uint32)
    return HkMp(0, 0, limbs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), limbs


def _mp_val(m, limbs):
    n = int.from_bytes(limbs.tobytes(), "little")
    return (0, 0) if n == 0 else ((-n if m.sign else n), int(m.exp))


def hk_time_update_slice(ctx, tsteps):
    """(device ms, MACs) of the update contributions of the first tsteps rows."""
    ms, macs = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().hk_time_update_slice(ctx, tsteps, ctypes.byref(ms), ctypes.byref(macs)), "hk_time_update_slice")
    return ms.value, macs.value


def hk_selftest_scalar(op, P, a, b):
    """Scalar operation of the Secant step on the device: op 0 RNE(a - b),
    1 RNE(a b), 2 RNE(a / b) -> (n, e); op 3 -> comparison -1/0/1."""
    am, al = _mp_in(a, P)
    bm, bl = _mp_in(b, P)
    om, ol = _mp_out(P)
    cmp = ctypes.c_int(0)
    _check(lib().hk_selftest_scalar(op, P // 32, ctypes.byref(am), ctypes.byref(bm), ctypes.byref(om),
                                    ctypes.byref(cmp)), "hk_selftest_scalar")
    return cmp.value if op == 3 else _mp_val(om, ol)


def hk_ldlt_det(ctx, P, x):
    """P(x) = det(M - xI): returns (det (n, e), negative pivots, first zero
    pivot or -1)."""
    xm, xl = _mp_in(x, P)
    dm, dl = _mp_out(P)
    neg, zr = ctypes.c_int(0), ctypes.c_int(-1)
    _check(lib().hk_ldlt_det(ctx, ctypes.byref(xm), ctypes.byref(dm), ctypes.byref(neg), ctypes.byref(zr)),
           "hk_ldlt_det")
    return _mp_val(dm, dl), neg.value, zr.value


def hk_get_ldlt(ctx, which, N, P):
    """which 0: the N pivots; 1: C rows as R rows; 2: CDivDiag rows."""
    n = N if which == 0 else N * (N + 1) // 2
    L = P // 32
    sign = np.zeros(n, dtype=np.int32)
    exp = np.zeros(n, dtype=np.int64)
    limbs = np.zeros((n, L), dtype=np.uint32)
    _check(lib().hk_get_ldlt_flat(ctx, which, _ptr(sign), _ptr(exp), _ptr(limbs)), "hk_get_ldlt_flat")
    vals = unpack(sign, exp, limbs)
    if which == 0:
        return vals
    rows, k = [], 0
    for t in range(N):
        rows.append(vals[k:k + N - t])
        k += N - t
    return rows


def hk_secant(ctx, P, max_steps=200):
    """The Secant root of P(x): returns (root (n, e), determinants used)."""
    rm, rl = _mp_out(P)
    used = ctypes.c_int(0)
    _check(lib().hk_secant(ctx, max_steps, ctypes.byref(rm), ctypes.byref(used)), "hk_secant")
    return _mp_val(rm, rl), used.value


def hk_get_secant(ctx, count, P):
    """Iterates and determinants of the last hk_secant: two lists of (n, e)."""
    L = P // 32
    arrs = [np.zeros(count, dtype=np.int32), np.zeros(count, dtype=np.int64), np.zeros((count, L), dtype=np.uint32),
            np.zeros(count, dtype=np.int32), np.zeros(count, dtype=np.int64), np.zeros((count, L), dtype=np.uint32)]
    _check(lib().hk_get_secant_flat(ctx, count, *[_ptr(a) for a in arrs]), "hk_get_secant_flat")
    return unpack(*arrs[:3]), unpack(*arrs[3:])


def hk_secant_verify(ctx, P, x, bits=130, P2=None):
    """Inertia on both sides of x: (negatives below, negatives above, det sign
    below, det sign above)."""
    if P2 is None:
        P2 = (P + bits + 1 + 31) // 32 * 32
    xm, xl = _mp_in(x, P)
    out = (ctypes.c_int * 4)()
    _check(lib().hk_secant_verify(ctx, ctypes.byref(xm), bits, P2, out), "hk_secant_verify")
    return tuple(out)


class Hankel:
    """Convenience wrapper: one context, one problem."""

    def __init__(self, device=0, stream=None):
        self.ctx = hk_create(device, stream)
        self.N = self.P = None

    def close(self):
        if self.ctx is not None:
            hk_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load(self, N, beta, P, moments):
        self.N, self.P = N, P
        sign, exp, limbs = pack(moments, P)
        hk_load_moments_flat(self.ctx, N, beta, P, sign, exp, limbs)

    def load_device(self, N, beta, P, sign, exp, limbs):
        """Moments already resident in device memory (torch CUDA tensors)."""
        self.N, self.P = N, P
        hk_load_moments_flat(self.ctx, N, beta, P, sign, exp, limbs, on_device=True)

    def factor(self):
        hk_factor(self.ctx)

    def set_option(self, option, value):
        hk_set_option(self.ctx, option, value)

    def set_update_path(self, path):
        """0: IMAD product scanning (default), 1: INT8 tensor instruction."""
        _check(lib().hk_set_update_path(self.ctx, path), "hk_set_update_path")

    def R(self):
        return hk_get_R(self.ctx, self.N, self.P)

    def smallest_eig(self, iters):
        return hk_smallest_eig(self.ctx, self.P, iters)

    def history(self, count):
        return hk_get_history_flat(self.ctx, count, self.P)

    def timings(self):
        return hk_get_timings(self.ctx)

    def stats(self):
        return hk_get_stats(self.ctx)


HK_MLP_NPARAMS = 4547


def _dp(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))


def hk_mlp_workspace_bytes(B):
    return int(lib().hk_mlp_workspace_bytes(B))


def hk_mlp_forward(params, x, y, stream=None):
    """params float32[HK_MLP_NPARAMS], x float32[B, 2], y float32[B, 3]: CUDA tensors."""
    _check(lib().hk_mlp_forward(_dp(params), _dp(x), x.shape[0], _dp(y), _stream(stream)), "hk_mlp_forward")


def hk_mlp_loss_grad(params, x, t, w, grad, loss, work, stream=None):
    _check(lib().hk_mlp_loss_grad(_dp(params), _dp(x), _dp(t), _dp(w), x.shape[0], _dp(grad), _dp(loss),
                                  _dp(work), work.numel() * work.element_size(), _stream(stream)),
           "hk_mlp_loss_grad")


def hk_mlp_adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().hk_mlp_adam(_dp(params), _dp(grad), _dp(m), _dp(v), params.numel(), step, lr, beta1, beta2,
                             eps, _stream(stream)), "hk_mlp_adam")


def hk_mlp_train(params, m, v, grad, x, t, w, steps, step0, lr, work, loss_hist=None, beta1=0.9, beta2=0.999,
                 eps=1e-8, stream=None):
    _check(lib().hk_mlp_train(_dp(params), _dp(m), _dp(v), _dp(grad), _dp(x), _dp(t), _dp(w), x.shape[0], steps,
                              step0, lr, beta1, beta2, eps, _dp(loss_hist), _dp(work),
                              work.numel() * work.element_size(), _stream(stream)), "hk_mlp_train")


def hk_update_plan(W, levels=-1, with_units=True):
    """Host-side plan of the exact update for a window of W limbs (no GPU):
    the Karatsuba depth, pieces (offset, width), their (offset, sign) terms,
    split points, the (stripe, chunk) schedule, the unit table and the
    per-block operand windows -- what hk_factor launches for that window."""
    L = lib()
    info = (ctypes.c_int64 * 9)()
    splits = (ctypes.c_int32 * 40)()
    pieces = (ctypes.c_int32 * (3 * 81))()
    terms = (ctypes.c_int32 * (2 * 16 * 81))()
    _check(L.hk_update_plan(W, levels, info, splits, pieces, terms, None, 0, None), "hk_update_plan")
    n, nunits, nxb = info[1], info[6], info[7]
    units = win = None
    if with_units:
        ub = (ctypes.c_int32 * (2 * nunits))()
        wb = (ctypes.c_int32 * (2 * 64))()
        _check(L.hk_update_plan(W, levels, info, None, None, None, ub, nunits, wb), "hk_update_plan")
        # (piece, first column, first p, p-steps); stripe-8 units carry their own
        # length (groups of eight in bits 16..23 of the start), others the chunk
        units = []
        for u in range(nunits):
            q, d0, pw = ub[2 * u] >> 24, ub[2 * u] & 0xFFFFFF, ub[2 * u + 1]
            if info[4] == 8:
                units.append((q, d0, pw & 0xFFFF, ((pw >> 16) & 0xFF) * 8))
            else:
                units.append((q, d0, pw, info[5]))
        win = [(wb[2 * b], wb[2 * b + 1]) for b in range(nxb)]
    return {
        "levels": info[0], "npieces": n, "stride": info[2], "gap": info[3], "uc": info[4], "upc": info[5],
        "nunits": nunits, "nxb": nxb, "C": info[8],
        "m1": splits[0], "m2": list(splits[1:4]), "m3": list(splits[4:13]), "m4": list(splits[13:40]),
        "pieces": [(pieces[3 * k], pieces[3 * k + 1]) for k in range(n)],
        "terms": [[(terms[2 * (16 * k + t)], terms[2 * (16 * k + t) + 1]) for t in range(pieces[3 * k + 2])]
                  for k in range(n)],
        "units": units, "windows": win,
    }


def hk_set_predictor(ctx, params, x_mean, x_std, y_mean, y_std):
    """Load a trained network (host float32[HK_MLP_NPARAMS]) and its scalings."""
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    sc = np.ascontiguousarray(np.concatenate([x_mean, x_std, y_mean, y_std]).astype(np.float64))
    _check(lib().hk_set_predictor(ctx, p.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p)),
           "hk_set_predictor")


def hk_predict(ctx, Ns, betas):
    """(bits, log2 lambda_min, iterations) per (N, beta) from the loaded network."""
    n = len(Ns)
    N = np.ascontiguousarray(np.asarray(Ns, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
    out = np.zeros((n, 3), dtype=np.float32)
    _check(lib().hk_predict(ctx, n, N.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                            out.ctypes.data_as(ctypes.c_void_p)), "hk_predict")
    return out
