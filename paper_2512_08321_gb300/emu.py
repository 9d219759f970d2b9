"""Thin ctypes binding of the C ABI in include/ozaki2_emu.h.

Argument marshalling only: every step of the emulation runs in the CUDA
library.  The functions keep the C names; device buffers are passed as
integer addresses (``tensor.data_ptr()``) and streams as ``cudaStream_t``
handles (``torch.cuda.current_stream().cuda_stream``).  There is no CPU
fallback: loading fails loudly when the library has not been built.
"""
import ctypes
import os

import torch  # loads the CUDA runtime the library links against

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libozaki2emu.so")

EMU_OK = 0
EMU_ERR_INVALID_ARG = 1
EMU_ERR_K_TOO_LARGE = 2
EMU_ERR_MODULI_RANGE = 3
EMU_ERR_ALLOC = 4
EMU_ERR_CUDA = 5
EMU_ERR_TIMEOUT = 6
EMU_ERR_UNSUPPORTED = 7
EMU_ERR_WORKSPACE = 8
EMU_ERR_SIZE_LIMIT = 9
STATUS_NAMES = {0: "EMU_OK", 1: "EMU_ERR_INVALID_ARG", 2: "EMU_ERR_K_TOO_LARGE",
                3: "EMU_ERR_MODULI_RANGE", 4: "EMU_ERR_ALLOC", 5: "EMU_ERR_CUDA",
                6: "EMU_ERR_TIMEOUT", 7: "EMU_ERR_UNSUPPORTED", 8: "EMU_ERR_WORKSPACE",
                9: "EMU_ERR_SIZE_LIMIT"}
EMU_STATIC_EXP_MAX_ROWS = 65536

OPS = {"N": 0, "T": 1, "C": 2}
EMU_ENGINE_AUTO, EMU_ENGINE_F16, EMU_ENGINE_I8 = 0, 1, 2
EMU_EXP_NONFINITE = -32768
EMU_MIN_MODULI, EMU_MAX_MODULI = 2, 24

_c_i64 = ctypes.c_int64
_c_ptr = ctypes.c_void_p
_c_int = ctypes.c_int

# (name, restype, argtypes) of every exported function
_SIGS = [
    ("emu_zgemm", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_double),
                           _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_double), _c_ptr,
                           _c_i64, _c_int, _c_ptr]),
    ("emu_cgemm", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_float),
                           _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_float), _c_ptr,
                           _c_i64, _c_int, _c_ptr]),
    ("emu_dgemm", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_double),
                           _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_double), _c_ptr,
                           _c_i64, _c_int, _c_ptr]),
    ("emu_sgemm", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_float),
                           _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_float), _c_ptr,
                           _c_i64, _c_int, _c_ptr]),
    ("emu_zgemm_host", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_double),
                                _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_double), _c_ptr,
                                _c_i64, _c_int, _c_ptr]),
    ("emu_cgemm_host", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_float),
                                _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_float), _c_ptr,
                                _c_i64, _c_int, _c_ptr]),
    ("emu_dgemm_host", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_double),
                                _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_double), _c_ptr,
                                _c_i64, _c_int, _c_ptr]),
    ("emu_sgemm_host", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_float),
                                _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_float), _c_ptr,
                                _c_i64, _c_int, _c_ptr]),
    ("emu_grouped_create", _c_int, [_c_int, _c_int, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                    _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_int, _c_int,
                                    ctypes.POINTER(_c_ptr)]),
    ("emu_grouped_run", _c_int, [_c_ptr, _c_ptr]),
    ("emu_grouped_tile", _c_int, [_c_ptr]),
    ("emu_grouped_kernels", _c_int, [_c_ptr]),
    ("emu_grouped_destroy", _c_int, [_c_ptr]),
    ("emu_grouped_phase_times", _c_int, [_c_ptr, ctypes.POINTER(ctypes.c_float), _c_ptr]),
    ("emu_zgemm_grouped", _c_int, [_c_int, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                   _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_int, _c_ptr]),
    ("emu_cgemm_grouped", _c_int, [_c_int, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr,
                                   _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_int, _c_ptr]),
    ("emu_zgemm_tol", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_double),
                               _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_double), _c_ptr, _c_i64,
                               ctypes.c_double, ctypes.POINTER(_c_int), _c_ptr]),
    ("emu_cgemm_tol", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_float),
                               _c_ptr, _c_i64, _c_ptr, _c_i64, ctypes.POINTER(ctypes.c_float), _c_ptr, _c_i64,
                               ctypes.c_double, ctypes.POINTER(_c_int), _c_ptr]),
    ("emu_moduli_apriori", _c_int, [_c_int, _c_i64, ctypes.c_double]),
    ("emu_mlp_param_count", _c_int, []),
    ("emu_mlp_set_weights", _c_int, [ctypes.POINTER(ctypes.c_float), _c_int]),
    ("emu_moduli_features", _c_int, [_c_int, _c_int, _c_int, _c_i64, _c_i64, _c_i64, _c_ptr, _c_i64, _c_ptr,
                                     _c_i64, ctypes.c_double, _c_ptr, _c_ptr]),
    ("emu_mlp_forward", _c_int, [_c_ptr, _c_ptr, _c_int, _c_ptr, _c_ptr]),
    ("emu_mlp_backward", _c_int, [_c_ptr, _c_ptr, _c_ptr, _c_int, _c_ptr, _c_ptr, _c_ptr]),
    ("emu_mlp_adam", _c_int, [_c_ptr, _c_ptr, _c_ptr, _c_ptr, _c_int, ctypes.c_float, _c_ptr]),
    ("emu_mlp_choose", _c_int, [_c_ptr, _c_ptr, ctypes.c_float, _c_ptr, _c_ptr]),
    ("emu_workspace_bytes", ctypes.c_size_t, [_c_int, _c_i64, _c_i64, _c_i64, _c_int]),
    ("emu_set_workspace", _c_int, [_c_ptr, ctypes.c_size_t]),
    ("emu_set_engine", _c_int, [_c_int, _c_int]),
    ("emu_set_crt_mode", _c_int, [_c_int]),
    ("emu_set_tuning", _c_int, [_c_int, _c_int]),
    ("emu_get_tuning", _c_int, [_c_int]),
    ("emu_tuned_value", _c_int, [_c_int, _c_int, _c_i64, _c_i64, _c_i64, _c_int]),
    ("emu_autotune_gemm", _c_int, [_c_int, _c_i64, _c_i64, _c_i64, _c_int, ctypes.POINTER(_c_int)]),
    ("emu_autotune_clear", _c_int, []),
    ("emu_set_scaling", _c_int, [_c_int]),
    ("emu_get_scaling", _c_int, []),
    ("emu_plan_exponent_accu", _c_int, [_c_int, ctypes.c_uint64]),
    ("emu_stage_exponents", _c_int, [_c_int, _c_int, _c_int, _c_i64, _c_i64, _c_i64, _c_ptr, _c_i64,
                                     _c_ptr, _c_i64, _c_int, _c_ptr, _c_ptr, _c_ptr]),
    ("emu_stage_exponents_static", _c_int, [_c_int, _c_int, _c_int, _c_i64, _c_i64, _c_i64, _c_ptr, _c_i64,
                                            _c_ptr, _c_i64, _c_int, _c_ptr, _c_ptr, _c_ptr]),
    ("emu_stage_split", _c_int, [_c_int, _c_int, _c_int, _c_i64, _c_i64, _c_i64, _c_ptr, _c_i64,
                                 _c_ptr, _c_i64, _c_int, _c_ptr, _c_ptr, _c_int, _c_i64, _c_ptr,
                                 _c_ptr, _c_ptr]),
    ("emu_stage_residue_gemm", _c_int, [_c_int, _c_i64, _c_i64, _c_i64, _c_int, _c_ptr, _c_ptr,
                                        _c_ptr, _c_i64, _c_ptr]),
    ("emu_stage_crt", _c_int, [_c_int, _c_i64, _c_i64, _c_int, _c_ptr, _c_i64, _c_ptr, _c_ptr,
                               _c_ptr, _c_ptr, _c_ptr, _c_i64, _c_ptr]),
    ("emu_plan_info", _c_int, [_c_int, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)]),
    ("emu_plan_exponent", _c_int, [_c_int, ctypes.c_uint64]),
    ("emu_last_bad_param", _c_int, []),
    ("emu_stream_status", _c_int, [_c_ptr]),
    ("emu_selftest_bounded_wait", _c_int, [_c_i64, _c_ptr]),
    ("emu_set_phase_events", _c_int, [ctypes.POINTER(_c_ptr), _c_int]),
    ("emu_kernel_launches", ctypes.c_uint64, []),
    ("emu_host_trace_enable", _c_int, [_c_int]),
    ("emu_host_trace_read", _c_int, [ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float), _c_int]),
    ("emu_version", ctypes.c_char_p, []),
]

_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return [s[0] for s in _SIGS]


class EmuError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        bp = lib().emu_last_bad_param() if status == EMU_ERR_INVALID_ARG else 0
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}" + (f" (argument {bp})" if bp else ""))


def check(status, where):
    if status != EMU_OK:
        raise EmuError(status, where)
    return status


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _op(op):
    return OPS[op.upper()] if isinstance(op, str) else int(op)


# ------------------------------------------------------------ C-named calls
def emu_zgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a = (ctypes.c_double * 2)(float(alpha.real), float(alpha.imag))
    b = (ctypes.c_double * 2)(float(beta.real), float(beta.imag))
    return lib().emu_zgemm(_op(transa), _op(transb), m, n, k, a, A, lda, B, ldb, b, C, ldc,
                           num_moduli, _stream(stream))


def emu_cgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a = (ctypes.c_float * 2)(float(alpha.real), float(alpha.imag))
    b = (ctypes.c_float * 2)(float(beta.real), float(beta.imag))
    return lib().emu_cgemm(_op(transa), _op(transb), m, n, k, a, A, lda, B, ldb, b, C, ldc,
                           num_moduli, _stream(stream))


def emu_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a, b = ctypes.c_double(float(alpha)), ctypes.c_double(float(beta))
    return lib().emu_dgemm(_op(transa), _op(transb), m, n, k, ctypes.byref(a), A, lda, B, ldb, ctypes.byref(b),
                           C, ldc, num_moduli, _stream(stream))


def emu_sgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a, b = ctypes.c_float(float(alpha)), ctypes.c_float(float(beta))
    return lib().emu_sgemm(_op(transa), _op(transb), m, n, k, ctypes.byref(a), A, lda, B, ldb, ctypes.byref(b),
                           C, ldc, num_moduli, _stream(stream))


def emu_zgemm_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a = (ctypes.c_double * 2)(float(alpha.real), float(alpha.imag))
    b = (ctypes.c_double * 2)(float(beta.real), float(beta.imag))
    return lib().emu_zgemm_host(_op(transa), _op(transb), m, n, k, a, A, lda, B, ldb, b, C, ldc,
                                num_moduli, _stream(stream))


def emu_cgemm_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a = (ctypes.c_float * 2)(float(alpha.real), float(alpha.imag))
    b = (ctypes.c_float * 2)(float(beta.real), float(beta.imag))
    return lib().emu_cgemm_host(_op(transa), _op(transb), m, n, k, a, A, lda, B, ldb, b, C, ldc,
                                num_moduli, _stream(stream))


def emu_dgemm_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a, b = ctypes.c_double(float(alpha)), ctypes.c_double(float(beta))
    return lib().emu_dgemm_host(_op(transa), _op(transb), m, n, k, ctypes.byref(a), A, lda, B, ldb,
                                ctypes.byref(b), C, ldc, num_moduli, _stream(stream))


def emu_sgemm_host(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, num_moduli, stream=None):
    a, b = ctypes.c_float(float(alpha)), ctypes.c_float(float(beta))
    return lib().emu_sgemm_host(_op(transa), _op(transb), m, n, k, ctypes.byref(a), A, lda, B, ldb,
                                ctypes.byref(b), C, ldc, num_moduli, _stream(stream))


class GroupedArgs:
    """Host arrays describing a grouped call (kept alive with the plan)."""

    def __init__(self, problems, num_moduli):
        # problems: list of dicts with transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc
        c = len(problems)
        I64 = ctypes.c_int64 * max(c, 1)
        OPS_ = ctypes.c_int * max(c, 1)
        P = ctypes.c_void_p * max(c, 1)
        D = ctypes.c_double * max(2 * c, 2)
        self.count = c
        self.ta = OPS_(*[_op(p["transa"]) for p in problems])
        self.tb = OPS_(*[_op(p["transb"]) for p in problems])
        self.m = I64(*[p["m"] for p in problems])
        self.n = I64(*[p["n"] for p in problems])
        self.k = I64(*[p["k"] for p in problems])
        self.lda = I64(*[p["lda"] for p in problems])
        self.ldb = I64(*[p["ldb"] for p in problems])
        self.ldc = I64(*[p["ldc"] for p in problems])
        self.A = P(*[p["A"] for p in problems])
        self.B = P(*[p["B"] for p in problems])
        self.C = P(*[p["C"] for p in problems])
        al, be = [], []
        for p in problems:
            a, b = complex(p.get("alpha", 1.0)), complex(p.get("beta", 0.0))
            al += [a.real, a.imag]
            be += [b.real, b.imag]
        self.alpha = D(*al) if al else D()
        self.beta = D(*be) if be else D()
        self.N = num_moduli

    def argv(self):
        c = ctypes.cast
        return (self.count, c(self.ta, _c_ptr), c(self.tb, _c_ptr), c(self.m, _c_ptr), c(self.n, _c_ptr),
                c(self.k, _c_ptr), c(self.alpha, _c_ptr), c(self.A, _c_ptr), c(self.lda, _c_ptr),
                c(self.B, _c_ptr), c(self.ldb, _c_ptr), c(self.beta, _c_ptr), c(self.C, _c_ptr),
                c(self.ldc, _c_ptr))


def emu_grouped_create(is_single, args, tile_n=0):
    """Returns (status, plan handle)."""
    h = _c_ptr()
    st = lib().emu_grouped_create(int(is_single), *args.argv(), args.N, int(tile_n), ctypes.byref(h))
    return st, h


EMU_GROUPED_TILE_PER_PROBLEM = -1


def emu_grouped_run(plan, stream=None):
    return lib().emu_grouped_run(plan, _stream(stream))


def emu_grouped_tile(plan):
    return lib().emu_grouped_tile(plan)


def emu_grouped_kernels(plan):
    return lib().emu_grouped_kernels(plan)


def emu_grouped_phase_times(plan, stream=None):
    """(status, [exponents, split, residue products, CRT] milliseconds)."""
    ms = (ctypes.c_float * 4)()
    st = lib().emu_grouped_phase_times(plan, ms, _stream(stream))
    return st, list(ms)


def emu_grouped_destroy(plan):
    return lib().emu_grouped_destroy(plan)


def emu_zgemm_grouped(args, stream=None):
    return lib().emu_zgemm_grouped(*args.argv(), args.N, _stream(stream))


def emu_cgemm_grouped(args, stream=None):
    return lib().emu_cgemm_grouped(*args.argv(), args.N, _stream(stream))


def emu_zgemm_tol(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, target, stream=None):
    """Returns (status, N used)."""
    a = (ctypes.c_double * 2)(float(complex(alpha).real), float(complex(alpha).imag))
    b = (ctypes.c_double * 2)(float(complex(beta).real), float(complex(beta).imag))
    nu = _c_int(0)
    st = lib().emu_zgemm_tol(_op(transa), _op(transb), m, n, k, a, A, lda, B, ldb, b, C, ldc, float(target),
                             ctypes.byref(nu), _stream(stream))
    return st, nu.value


def emu_cgemm_tol(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, target, stream=None):
    a = (ctypes.c_float * 2)(float(complex(alpha).real), float(complex(alpha).imag))
    b = (ctypes.c_float * 2)(float(complex(beta).real), float(complex(beta).imag))
    nu = _c_int(0)
    st = lib().emu_cgemm_tol(_op(transa), _op(transb), m, n, k, a, A, lda, B, ldb, b, C, ldc, float(target),
                             ctypes.byref(nu), _stream(stream))
    return st, nu.value


def emu_moduli_apriori(is_single, k, target):
    return lib().emu_moduli_apriori(int(is_single), int(k), float(target))


def emu_mlp_param_count():
    return lib().emu_mlp_param_count()


def emu_mlp_set_weights(params):
    """params: sequence of floats (or None to unload)."""
    if params is None:
        return lib().emu_mlp_set_weights(None, 0)
    arr = (ctypes.c_float * len(params))(*[float(v) for v in params])
    return lib().emu_mlp_set_weights(arr, len(params))


def emu_moduli_features(is_single, transa, transb, m, n, k, A, lda, B, ldb, target, features, stream=None):
    return lib().emu_moduli_features(int(is_single), _op(transa), _op(transb), m, n, k, A, lda, B, ldb,
                                     float(target), features, _stream(stream))


def emu_mlp_forward(theta, X, batch, logits, stream=None):
    return lib().emu_mlp_forward(theta, X, batch, logits, _stream(stream))


def emu_mlp_backward(theta, X, Y, batch, grad, loss, stream=None):
    return lib().emu_mlp_backward(theta, X, Y, batch, grad, loss, _stream(stream))


def emu_mlp_adam(theta, grad, m, v, step, lr, stream=None):
    return lib().emu_mlp_adam(theta, grad, m, v, int(step), float(lr), _stream(stream))


def emu_mlp_choose(theta, features, threshold, n_out, stream=None):
    return lib().emu_mlp_choose(theta, features, float(threshold), n_out, _stream(stream))


EMU_DTYPE_Z, EMU_DTYPE_C, EMU_DTYPE_D, EMU_DTYPE_S = 0, 1, 2, 3


def emu_workspace_bytes(dtype, m, n, k, num_moduli):
    return lib().emu_workspace_bytes(int(dtype), m, n, k, num_moduli)


def emu_set_workspace(ptr, nbytes):
    return lib().emu_set_workspace(ptr, nbytes)


def emu_set_engine(engine, chunk_k=0):
    return lib().emu_set_engine(int(engine), int(chunk_k))


EMU_CRT_EXACT, EMU_CRT_PAPER_FP64 = 0, 1
EMU_TUNE_TILE_N, EMU_TUNE_GROUP, EMU_TUNE_CHUNK_K, EMU_TUNE_CRT_ROWS, EMU_TUNE_SPLIT_ELEMS = 1, 2, 3, 4, 5
EMU_TUNE_NBLOCK = 6
EMU_TUNE_OVERLAP = 7
EMU_TUNE_ORDER, EMU_TUNE_PAIRING, EMU_TUNE_KDIR, EMU_TUNE_BAND = 8, 9, 10, 11
EMU_TUNE_CRT_ENGINE = 12
EMU_TUNE_CTA_PAIR = 13
EMU_TUNE_BOUND_PAIR = 14
SCHEDULE_KNOBS = {"order": EMU_TUNE_ORDER, "pairing": EMU_TUNE_PAIRING, "kdir": EMU_TUNE_KDIR,
                  "band": EMU_TUNE_BAND, "cta_pair": EMU_TUNE_CTA_PAIR}


def emu_set_tuning(key, value):
    return lib().emu_set_tuning(int(key), int(value))


def emu_get_tuning(key):
    return lib().emu_get_tuning(int(key))


def emu_tuned_value(dtype, num_moduli, m, n, k, key):
    return lib().emu_tuned_value(int(dtype), int(num_moduli), m, n, k, int(key))


def emu_autotune_gemm(dtype, m, n, k, num_moduli):
    """Returns (status, [tile_n, group, chunk_k, crt_rows, split_elems]); dtype
    is an EMU_DTYPE_* code (0/1 = complex128/complex64)."""
    best = (_c_int * 5)()
    st = lib().emu_autotune_gemm(int(dtype), m, n, k, num_moduli, best)
    return st, list(best)


def emu_autotune_clear():
    return lib().emu_autotune_clear()


EMU_SCALING_FAST, EMU_SCALING_ACCURATE = 0, 1


def emu_set_scaling(mode):
    return lib().emu_set_scaling(int(mode))


def emu_get_scaling():
    return lib().emu_get_scaling()


def emu_plan_exponent_accu(num_moduli, M):
    return lib().emu_plan_exponent_accu(int(num_moduli), int(M))


def emu_set_crt_mode(mode):
    return lib().emu_set_crt_mode(int(mode))


def emu_stage_exponents(is_single, transa, transb, m, n, k, A, lda, B, ldb, num_moduli, x, y, stream=None):
    return lib().emu_stage_exponents(int(is_single), _op(transa), _op(transb), m, n, k, A, lda, B, ldb,
                                     num_moduli, x, y, _stream(stream))


def emu_stage_exponents_static(is_single, transa, transb, m, n, k, A, lda, B, ldb, num_moduli, x, y,
                               stream=None):
    """Allocation-free exponent phase (fixed scratch inside the library)."""
    return lib().emu_stage_exponents_static(int(is_single), _op(transa), _op(transb), m, n, k, A, lda, B, ldb,
                                            num_moduli, x, y, _stream(stream))


def emu_stage_split(is_single, transa, transb, m, n, k, A, lda, B, ldb, num_moduli, x, y, plane_fp16,
                    kpad, planesA, planesB, stream=None):
    return lib().emu_stage_split(int(is_single), _op(transa), _op(transb), m, n, k, A, lda, B, ldb,
                                 num_moduli, x, y, int(plane_fp16), kpad, planesA, planesB, _stream(stream))


def emu_stage_residue_gemm(engine, m, n, kpad, num_moduli, planesA, planesB, residues, ldr, stream=None):
    return lib().emu_stage_residue_gemm(int(engine), m, n, kpad, num_moduli, planesA, planesB, residues,
                                        ldr, _stream(stream))


def emu_stage_crt(is_single, m, n, num_moduli, residues, ldr, x, y, alpha, beta, C, ldc, stream=None):
    T = ctypes.c_float if is_single else ctypes.c_double
    a = (T * 2)(float(alpha.real), float(alpha.imag))
    b = (T * 2)(float(beta.real), float(beta.imag))
    return lib().emu_stage_crt(int(is_single), m, n, num_moduli, residues, ldr, x, y,
                               ctypes.cast(a, _c_ptr), ctypes.cast(b, _c_ptr), C, ldc, _stream(stream))


def emu_plan_info(num_moduli):
    """(status, moduli, q, P as int, crt limb count) computed by the library."""
    mod = (ctypes.c_int32 * EMU_MAX_MODULI)()
    q = (ctypes.c_int32 * EMU_MAX_MODULI)()
    limbs = (ctypes.c_uint32 * 8)()
    L = ctypes.c_int32()
    st = lib().emu_plan_info(num_moduli, mod, q, limbs, ctypes.byref(L))
    P = sum(int(limbs[t]) << (32 * t) for t in range(8))
    return st, list(mod[:num_moduli]), list(q[:num_moduli]), P, L.value


def emu_plan_exponent(num_moduli, S):
    return lib().emu_plan_exponent(num_moduli, int(S))


def emu_last_bad_param():
    return lib().emu_last_bad_param()


def emu_stream_status(stream=None):
    return lib().emu_stream_status(_stream(stream))


def emu_selftest_bounded_wait(limit_cycles, stream=None):
    return lib().emu_selftest_bounded_wait(int(limit_cycles), _stream(stream))


def emu_set_phase_events(events):
    """events: five torch.cuda.Event(enable_timing=True), or None to stop."""
    if not events:
        return lib().emu_set_phase_events(None, 0)
    for e in events:
        if not e.cuda_event:        # torch creates the CUDA event on first record
            e.record()
    arr = (_c_ptr * 5)(*[e.cuda_event for e in events])
    return lib().emu_set_phase_events(arr, 5)


def emu_kernel_launches():
    return lib().emu_kernel_launches()


(EMU_TRACE_START, EMU_TRACE_A_IN, EMU_TRACE_B_IN, EMU_TRACE_BLOCK_START, EMU_TRACE_BLOCK_CRT, EMU_TRACE_C_OUT,
 EMU_TRACE_END) = range(7)
EMU_TRACE_MAX = 64
TRACE_NAMES = ["start", "a_in", "b_in", "block_start", "block_crt", "c_out", "end"]


def emu_host_trace_enable(on):
    return lib().emu_host_trace_enable(int(bool(on)))


def emu_host_trace_read():
    """[(label name, ms after the call's start)] of the latest traced host-buffer call."""
    labels = (_c_int * EMU_TRACE_MAX)()
    ms = (ctypes.c_float * EMU_TRACE_MAX)()
    cnt = lib().emu_host_trace_read(labels, ms, EMU_TRACE_MAX)
    if cnt < 0:
        raise EmuError(EMU_ERR_CUDA, "emu_host_trace_read")
    return [(TRACE_NAMES[labels[i]], float(ms[i])) for i in range(cnt)]


def emu_version():
    return lib().emu_version().decode()


# ------------------------------------------------- torch tensor conveniences
def gemm(A_store, B_store, C_store, m, n, k, num_moduli, transa="N", transb="N",
         alpha=1.0, beta=0.0, lda=None, ldb=None, ldc=None, stream=None):
    """Emulated GEMM on column-major matrices held as C-contiguous (cols x ld)
    torch tensors (complex128 -> ZGEMM, complex64 -> CGEMM, float64 -> DGEMM,
    float32 -> SGEMM).  Raises on error."""
    f = {torch.complex128: emu_zgemm, torch.complex64: emu_cgemm,
         torch.float64: emu_dgemm, torch.float32: emu_sgemm}[A_store.dtype]
    lda = lda if lda is not None else A_store.shape[-1]
    ldb = ldb if ldb is not None else B_store.shape[-1]
    ldc = ldc if ldc is not None else C_store.shape[-1]
    real = not A_store.dtype.is_complex
    st = f(transa, transb, m, n, k, float(alpha) if real else complex(alpha), A_store.data_ptr(), lda,
           B_store.data_ptr(), ldb, float(beta) if real else complex(beta), C_store.data_ptr(), ldc, num_moduli,
           stream)
    return check(st, f.__name__)
