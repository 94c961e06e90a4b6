"""ctypes loader and signatures of libfk.so (the C ABI declared in include/fk.h)."""
import ctypes
import os
import threading

from . import build as _build

P = ctypes.c_void_p
I = ctypes.c_int
U = ctypes.c_uint
SZ = ctypes.c_size_t
U64 = ctypes.c_uint64
PP = ctypes.POINTER(ctypes.c_void_p)

# name -> argtypes; every function returns int except the string getters.
SIGNATURES = {
    "fk_version": [],
    "fk_device_status": [I],
    "fk_wait_selftest": [I],
    "fk_debug_status": [I, P, P],
    "fk_debug_selftest": [],
    "fk_table_create_dis": [P, I, P, I, I, P, I, U, PP],
    "fk_table_create_had": [P, I, P, P, I, I, P, I, U, PP],
    "fk_table_destroy": [P],
    "fk_table_info": [P, P, P, P, P, P, P, P],
    "fk_dis_conv": [P, P, I, P, I, I, P],
    "fk_had_conv": [P, P, I, P, I, I, P],
    "fk_had_conv_noalloc": [P, P, I, P, I, I, P],
    "fk_table_create_dense": [P, I, ctypes.c_longlong, U, PP],
    "fk_dense_conv": [P, P, I, P, I, I, P],
    "fk_luminosity": [P, P, I, P, I, P],
    "fk_conv_backward": [P, P, P, I, I, P, I, I, P],
    "fk_saved_size": [P, I, I, ctypes.POINTER(SZ)],
    "fk_had_conv_save": [P, P, I, P, I, P, SZ, I, P],
    "fk_conv_backward_saved": [P, P, P, I, I, P, SZ, P, I, I, P],
    "fk_grad_sum": [P, I, ctypes.c_longlong, P, I, I, P],
    "fk_cov_create": [P, P, I, PP],
    "fk_cov_destroy": [P],
    "fk_cov_size": [P],
    "fk_chi2": [P, P, P, I, P, P, I, P],
    "fk_chi2_white": [P, I, P, I, I, P, P, I, I, P],
    "fk_pdf_eval": [P, I, P, I, P, I, P],
    "fk_pdf_grad": [P, P, I, P, I, P, I, P],
    "fk_adam_step": [P, P, P, P, ctypes.c_longlong, I, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_double, I, P],
    "fk_fma_probe": [I, I, I, P, P],
    "fk_mma_probe": [I, I, I, P, P],
    "fk_serve_create": [SZ, I, PP],
    "fk_serve_add_table": [P, P, P],
    "fk_serve_submit": [P, I, P, I, I, ctypes.POINTER(U64)],
    "fk_serve_poll": [P, U64, P, P],
    "fk_serve_wait": [P, U64, P, I],
    "fk_serve_stats": [P, P, P, P, P, P],
    "fk_serve_cancel": [P, U64],
    "fk_serve_inject": [P, I, I],
    "fk_serve_destroy": [P],
}
U64_FUNCS = {"fk_kernel_launches": []}
STRING_FUNCS = {"fk_strerror": [I], "fk_last_error_message": []}

_lib = None
_lock = threading.Lock()


def debug() -> bool:
    """True when FK_DEBUG=1: the debug build libfk_debug.so is loaded."""
    return os.environ.get("FK_DEBUG") == "1"


def path() -> str:
    return _build.LIB_DEBUG if debug() else _build.LIB


def load():
    """Loads libfk.so (libfk_debug.so when FK_DEBUG=1), building it first if
    the sources are newer and nvcc is present.  Raises if the library cannot
    be loaded: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        dbg = debug()
        if not _build.up_to_date(dbg):
            try:
                _build.build(debug=dbg)
            except (OSError, RuntimeError) as e:
                if not os.path.exists(path()):
                    raise RuntimeError(f"{os.path.basename(path())} is missing and could not be built: {e}") from e
        lib = ctypes.CDLL(path())
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = I
        for name, args in U64_FUNCS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = U64
        for name, args in STRING_FUNCS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p
        _lib = lib
        return lib


class FKError(RuntimeError):
    def __init__(self, func, status, lib):
        self.status = status
        msg = lib.fk_strerror(status).decode()
        detail = lib.fk_last_error_message().decode()
        super().__init__(f"{func}: {msg}" + (f" ({detail})" if detail else ""))


def call(name, *args):
    lib = load()
    rc = getattr(lib, name)(*args)
    if rc != 0:
        raise FKError(name, rc, lib)
    return rc


# status codes and precisions (include/fk.h)
FK_OK, FK_EINVAL, FK_ENOMEM, FK_EBUDGET, FK_EPENDING, FK_ETIMEDOUT, FK_ECUDA, FK_ENOTFOUND, \
    FK_EUNSUPPORTED, FK_ECANCELED = range(10)
FK_FAULT_PINNED, FK_FAULT_DEVICE, FK_FAULT_LAUNCH, FK_FAULT_DROP = range(1, 5)
# forward-formulation flags of fk_table_create_had (include/fk.h)
FK_TABLE_FACTORED, FK_TABLE_LUMI = 1 << 16, 1 << 17
FK_FP64, FK_FP32, FK_BF16, FK_BF16X3, FK_TF32, FK_FP64_TC = range(6)
PRECS = {"fp64": FK_FP64, "fp32": FK_FP32, "bf16": FK_BF16, "bf16x3": FK_BF16X3, "tf32": FK_TF32,
         "fp64tc": FK_FP64_TC}
