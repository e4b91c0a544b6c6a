"""ctypes binding of libqrmc (include/qr.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays and torch tensors to pointers and raises on error statuses. There is
no CPU fallback: if the library is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqrmc.so")

QR_OK, QR_EINVAL, QR_ENOMEM, QR_ECUDA, QR_ETIMEOUT, QR_ENONFINITE, QR_ENOTIMPL = range(7)
QR_NU_LOMAX, QR_NU_STUDENT2, QR_NU_CAUCHY = range(3)
QR_G_LINF, QR_G_L1, QR_G_HYP, QR_G_FULL_N, QR_G_TOTAL_N, QR_G_HYP_N = range(6)
QR_F_ZERO, QR_F_LINEAR, QR_F_CUBIC_MANUF, QR_F_PAPER_MIN = range(4)
QR_FAULT_NONE, QR_FAULT_ALLOC, QR_FAULT_LAUNCH, QR_FAULT_NAN = range(4)
QR_GT_COS, QR_GT_TRIGPOLY, QR_GT_PAPER_SIN = range(3)
QR_FP64, QR_FP32 = 0, 1
QR_U_PHILOX, QR_U_LATTICE = 0, 1
QR_HOST, QR_DEVICE = 0, 1
QR_PEAK_FP32, QR_PEAK_FP32X2, QR_PEAK_FP64, QR_PEAK_FP32MIX = range(4)

# every symbol declared in include/qr.h
EXPORTS = [
    "qr_init", "qr_picard_step", "qr_backward_sweep", "qr_eval", "qr_gamma_size", "qr_gamma_list",
    "qr_get_coefs", "qr_set_coefs", "qr_get_responses", "qr_set_profiling", "qr_get_stats",
    "qr_last_error", "qr_status_string", "qr_destroy", "qr_philox_words", "qr_sample", "qr_sample_normals_tree", "qr_project_static", "qr_test_points",
    "qr_selftest_wait_timeout",
    "qr_inject_fault",
    "qr_tree_layout",
    "qr_mlp_create", "qr_mlp_num_params", "qr_mlp_get_params", "qr_mlp_set_params", "qr_mlp_forward",
    "qr_mlp_gradients", "qr_mlp_train_step", "qr_mlp_last_error", "qr_mlp_destroy",
    "qr_batch_create", "qr_batch_picard_step", "qr_batch_info", "qr_batch_set_grouping", "qr_batch_groups",
    "qr_batch_last_error", "qr_batch_destroy", "qr_fma_peak", "qr_tc_selftest",
    "qr_shard_plan", "qr_shard", "qr_shard_groups", "qr_picard_begin", "qr_picard_finish",
]


class QrNu(C.Structure):
    _fields_ = [("kind", C.c_int), ("mu", C.c_double)]


class QrGamma(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int)]


class QrFn(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.POINTER(C.c_double)), ("n_params", C.c_int)]


class QrOpts(C.Structure):
    _fields_ = [
        ("M", C.c_longlong),
        ("seed", C.c_ulonglong),
        ("precision", C.c_int),
        ("clamp_L", C.c_double),
        ("stream", C.c_void_p),
        ("uniform_source", C.c_int),
        ("lattice_n", C.c_int),
        ("instance", C.c_int),
        ("path_kernel", C.c_int),
        ("damping_q", C.c_double),
        ("dev_alloc", C.c_void_p),
        ("dev_free", C.c_void_p),
        ("alloc_user", C.c_void_p),
    ]


# device allocator callbacks of qr_opts (dev_alloc / dev_free)
DEV_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
DEV_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


def _torch_alloc(nbytes, stream, user):
    try:
        import torch

        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # noqa: BLE001  (the library reports QR_ENOMEM)
        return None


def _torch_free(ptr, stream, user):
    try:
        import torch

        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:  # noqa: BLE001  (interpreter shutdown: the memory goes with the process)
        pass


TORCH_ALLOC = DEV_ALLOC(_torch_alloc)
TORCH_FREE = DEV_FREE(_torch_free)


def torch_allocator():
    """(dev_alloc, dev_free) pointers for qr_opts: PyTorch's caching allocator
    on the context's stream."""
    return C.cast(TORCH_ALLOC, C.c_void_p), C.cast(TORCH_FREE, C.c_void_p)


class QrStats(C.Structure):
    _fields_ = [
        ("iterations", C.c_longlong),
        ("clamp_hits", C.c_longlong),
        ("nonfinite", C.c_longlong),
        ("ms_paths", C.c_double),
        ("ms_project", C.c_double),
        ("ms_reduce", C.c_double),
        ("launches_paths", C.c_longlong),
        ("launches_project", C.c_longlong),
        ("launches_reduce", C.c_longlong),
    ]


class QrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("qr status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libqrmc.so (built in-tree by paper_2407_21084_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libqrmc.so is not built (run python -m paper_2407_21084_b300.build)")
    L = C.CDLL(p)
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    L.qr_init.restype = C.c_int
    L.qr_init.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_double, C.POINTER(QrNu), C.POINTER(QrGamma), dp, dp,
                          C.POINTER(QrFn), C.POINTER(QrFn), C.POINTER(QrOpts)]
    L.qr_picard_step.restype = C.c_int
    L.qr_picard_step.argtypes = [vp, C.c_int, dp]
    L.qr_backward_sweep.restype = C.c_int
    L.qr_backward_sweep.argtypes = [vp]
    L.qr_eval.restype = C.c_int
    L.qr_eval.argtypes = [vp, C.c_int, vp, C.c_longlong, vp, C.c_int]
    L.qr_gamma_size.restype = C.c_int
    L.qr_gamma_size.argtypes = [vp, C.POINTER(C.c_int)]
    L.qr_gamma_list.restype = C.c_int
    L.qr_gamma_list.argtypes = [vp, C.POINTER(C.c_int)]
    L.qr_get_coefs.restype = C.c_int
    L.qr_get_coefs.argtypes = [vp, dp]
    L.qr_set_coefs.restype = C.c_int
    L.qr_set_coefs.argtypes = [vp, dp]
    L.qr_get_responses.restype = C.c_int
    L.qr_get_responses.argtypes = [vp, C.c_int, dp]
    L.qr_set_profiling.restype = C.c_int
    L.qr_set_profiling.argtypes = [vp, C.c_int]
    L.qr_get_stats.restype = C.c_int
    L.qr_get_stats.argtypes = [vp, C.POINTER(QrStats)]
    L.qr_last_error.restype = C.c_char_p
    L.qr_last_error.argtypes = [vp]
    L.qr_status_string.restype = C.c_char_p
    L.qr_status_string.argtypes = [C.c_int]
    L.qr_destroy.restype = None
    L.qr_destroy.argtypes = [vp]
    L.qr_philox_words.restype = C.c_int
    L.qr_philox_words.argtypes = [C.POINTER(C.c_uint32), C.c_longlong, C.POINTER(C.c_uint32)]
    L.qr_sample.restype = C.c_int
    L.qr_sample.argtypes = [C.c_int, C.POINTER(QrNu), C.c_ulonglong, C.c_int, C.c_int, C.c_longlong, C.c_longlong,
                            C.c_int, C.c_int, dp, dp, dp]
    L.qr_sample_normals_tree.restype = C.c_int
    L.qr_sample_normals_tree.argtypes = [C.c_int, C.c_ulonglong, C.c_int, C.c_int, C.c_longlong, C.c_longlong,
                                         C.c_int, dp]
    fp = C.POINTER(C.c_float)
    L.qr_mlp_create.restype = C.c_int
    L.qr_mlp_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, vp]
    L.qr_mlp_num_params.restype = C.c_longlong
    L.qr_mlp_num_params.argtypes = [vp]
    L.qr_mlp_get_params.restype = C.c_int
    L.qr_mlp_get_params.argtypes = [vp, fp]
    L.qr_mlp_set_params.restype = C.c_int
    L.qr_mlp_set_params.argtypes = [vp, fp]
    L.qr_mlp_forward.restype = C.c_int
    L.qr_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
    L.qr_mlp_gradients.restype = C.c_int
    L.qr_mlp_gradients.argtypes = [vp, vp, vp, C.c_int, fp, fp]
    L.qr_mlp_train_step.restype = C.c_int
    L.qr_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, fp]
    L.qr_mlp_last_error.restype = C.c_char_p
    L.qr_mlp_last_error.argtypes = [vp]
    L.qr_mlp_destroy.restype = None
    L.qr_mlp_destroy.argtypes = [vp]
    L.qr_batch_create.restype = C.c_int
    L.qr_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int]
    L.qr_batch_picard_step.restype = C.c_int
    L.qr_batch_picard_step.argtypes = [vp, C.c_int, dp]
    L.qr_batch_info.restype = C.c_int
    L.qr_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
    L.qr_selftest_wait_timeout.restype = C.c_int
    L.qr_selftest_wait_timeout.argtypes = [vp]
    L.qr_inject_fault.restype = C.c_int
    L.qr_inject_fault.argtypes = [vp, C.c_int]
    L.qr_tree_layout.restype = C.c_int
    L.qr_tree_layout.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), dp]
    L.qr_batch_set_grouping.restype = C.c_int
    L.qr_batch_set_grouping.argtypes = [vp, C.c_int]
    L.qr_batch_groups.restype = C.c_int
    L.qr_batch_groups.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.qr_batch_last_error.restype = C.c_char_p
    L.qr_batch_last_error.argtypes = [vp]
    L.qr_batch_destroy.restype = None
    L.qr_batch_destroy.argtypes = [vp]
    L.qr_test_points.restype = C.c_int
    L.qr_test_points.argtypes = [vp, C.c_int, C.c_longlong, dp]
    L.qr_project_static.restype = C.c_int
    L.qr_project_static.argtypes = [vp, vp, C.c_int, C.c_int, vp]
    L.qr_fma_peak.restype = C.c_int
    L.qr_fma_peak.argtypes = [C.c_int, C.c_double, vp, dp, dp, C.POINTER(C.c_int)]
    ip = C.POINTER(C.c_int)
    L.qr_shard_plan.restype = C.c_int
    L.qr_shard_plan.argtypes = [C.c_int, C.c_int, C.c_int, ip, ip, ip, ip]
    L.qr_shard.restype = C.c_int
    L.qr_shard.argtypes = [vp, C.c_int, C.c_int]
    L.qr_shard_groups.restype = C.c_int
    L.qr_shard_groups.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_longlong), ip, ip]
    L.qr_picard_begin.restype = C.c_int
    L.qr_picard_begin.argtypes = [vp]
    L.qr_picard_finish.restype = C.c_int
    L.qr_picard_finish.argtypes = [vp, dp]
    L.qr_tc_selftest.restype = C.c_int
    L.qr_tc_selftest.argtypes = [C.POINTER(C.c_uint16), C.POINTER(C.c_uint16), C.POINTER(C.c_float)]
    _lib = L
    return L


def check(status: int, ctx=None):
    if status != QR_OK:
        L = load()
        msg = L.qr_last_error(ctx).decode() if ctx else L.qr_status_string(status).decode()
        raise QrError(status, msg or L.qr_status_string(status).decode())


def fma_peak(kind: int, ms: float, stream: int | None = None) -> dict:
    """Measured FMA throughput of the current device (qr_fma_peak):
    {"tflops", "ms", "sm_count"}."""
    L = load()
    tf, el, sms = C.c_double(), C.c_double(), C.c_int()
    check(L.qr_fma_peak(kind, ms, C.c_void_p(stream or 0), C.byref(tf), C.byref(el), C.byref(sms)))
    return {"tflops": tf.value, "ms": el.value, "sm_count": sms.value}


def tc_selftest(A_bits, B_bits):
    """qr_tc_selftest: D = A B^T (128x64 and 32x64 BF16 bit patterns) on the tensor cores."""
    import numpy as np

    L = load()
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    if A.shape != (128, 64) or B.shape != (32, 64):
        raise ValueError("A must be 128x64 and B 32x64")
    D = np.zeros((128, 32), dtype=np.float32)
    check(L.qr_tc_selftest(A.ctypes.data_as(C.POINTER(C.c_uint16)), B.ctypes.data_as(C.POINTER(C.c_uint16)),
                           D.ctypes.data_as(C.POINTER(C.c_float))))
    return D


def shard_plan(n_chunks: int, rank: int, world: int) -> dict:
    """qr_shard_plan: chunk and group ranges of a rank (host arithmetic)."""
    L = load()
    v = [C.c_int() for _ in range(4)]
    check(L.qr_shard_plan(n_chunks, rank, world, *[C.byref(x) for x in v]))
    return {"c_lo": v[0].value, "c_hi": v[1].value, "g_lo": v[2].value, "g_hi": v[3].value}
