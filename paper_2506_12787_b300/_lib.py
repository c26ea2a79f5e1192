"""ctypes view of the C ABI in include/wrf.h (argument marshalling only).

The shared library ``libwrf.so`` is built in-tree by ``build.py``.  Loading
fails loudly when it is missing: there is no CPU or PyTorch fallback for any
step of the path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwrf.so")

WRF_OK, WRF_EINVAL, WRF_ENOSPC, WRF_ECUDA, WRF_ETIMEOUT, WRF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
WRF_FP32, WRF_BF16, WRF_BF16X3 = 0, 1, 2
MAX_LAYERS = 8
PAPER_MAX_LAYERS, PAPER_MAX_WIDTH = 9, 160
REC_FLOATS = 8

STATUS_NAMES = {0: "WRF_OK", -1: "WRF_EINVAL", -2: "WRF_ENOSPC", -3: "WRF_ECUDA",
                -4: "WRF_ETIMEOUT", -5: "WRF_EUNSUPPORTED"}

# Every symbol include/wrf.h declares (checked by the CPU test suite).
EXPORTS = (
    "wrf_deform_workspace_size", "wrf_deform", "wrf_deform_acts", "wrf_project",
    "wrf_deform_project",
    "wrf_bin_workspace_size", "wrf_bin", "wrf_bin_noalloc", "wrf_render", "wrf_render_backward",
    "wrf_project_backward", "wrf_deform_backward_workspace_size", "wrf_deform_backward",
    "wrf_status_read", "wrf_last_error", "wrf_version", "wrf_selftest_wait", "wrf_rssi",
    "wrf_loss_workspace_size", "wrf_loss", "wrf_adam", "wrf_render_complex",
    "wrf_paper_workspace_size", "wrf_paper_deform_project", "wrf_measure_alu_peaks",
    "wrf_anneal_tx", "wrf_multi_set_size", "wrf_multi_set_prepare", "wrf_multi_workspace_size",
    "wrf_deform_project_multi", "wrf_bin_multi", "wrf_render_multi",
    "wrf_pipeline_create", "wrf_pipeline_step", "wrf_pipeline_wait", "wrf_pipeline_destroy",
)


class WrfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Scene(C.Structure):
    _fields_ = [("n", C.c_int32), ("channels", C.c_int32), ("mean", C.c_void_p),
                ("log_scale", C.c_void_p), ("rot", C.c_void_p), ("opacity_logit", C.c_void_p),
                ("amp", C.c_void_p)]


class Mlp(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("dims", C.c_int32 * (MAX_LAYERS + 1)),
                ("W", C.c_void_p * MAX_LAYERS), ("b", C.c_void_p * MAX_LAYERS),
                ("L_mean", C.c_int32), ("L_tx", C.c_int32), ("room_min", C.c_float * 3),
                ("room_size", C.c_float * 3), ("precision", C.c_int32)]


class PaperScene(C.Structure):
    _fields_ = [("n", C.c_int32), ("mu", C.c_void_p), ("chol", C.c_void_p),
                ("attn_logit", C.c_void_p), ("psi", C.c_void_p)]


class PaperMlp(C.Structure):
    _fields_ = [("n_hidden", C.c_int32), ("width", C.c_int32),
                ("W", C.c_void_p * PAPER_MAX_LAYERS), ("b", C.c_void_p * PAPER_MAX_LAYERS),
                ("L_mean", C.c_int32), ("L_tx", C.c_int32), ("room_min", C.c_float * 3),
                ("room_size", C.c_float * 3), ("precision", C.c_int32)]


class AdamGroup(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p),
                ("v", C.c_void_p), ("n", C.c_int64), ("lr", C.c_float)]


class Grid(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("q_cut", C.c_float), ("wrap_x", C.c_int32),
                ("px_per_thread", C.c_int32), ("batch_factor", C.c_int32),
                ("tma_staging", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libwrf.so and declare every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_2506_12787_b300.build` (nvcc, sm_103a)")
    L = C.CDLL(path)
    P, S, I32, I64, F = C.c_void_p, C.c_size_t, C.c_int32, C.c_int64, C.c_float
    sp, mp, gp = C.POINTER(Scene), C.POINTER(Mlp), C.POINTER(Grid)
    sig = {
        "wrf_deform_workspace_size": (S, [I32, I32, mp]),
        "wrf_deform": (I32, [sp, mp, gp, P, I32, P, P, S, P]),
        "wrf_deform_acts": (I32, [sp, mp, gp, P, I32, P, P, P, S, P]),
        "wrf_project": (I32, [sp, P, I32, gp, P, P, P]),
        "wrf_deform_project": (I32, [sp, mp, gp, P, I32, P, P, P, S, P]),
        "wrf_bin_workspace_size": (S, [I32, I32, gp]),
        "wrf_bin": (I32, [P, I32, I32, gp, P, I64, P, P, P, S, P]),
        "wrf_bin_noalloc": (I32, [P, I32, I32, gp, P, I64, P, P, P]),
        "wrf_render": (I32, [P, P, P, P, I64, I32, I32, gp, P, P]),
        "wrf_render_backward": (I32, [P, P, P, P, I64, I32, I32, gp, P, P, P]),
        "wrf_project_backward": (I32, [sp, P, I32, P, P, P, P, P, P, P, P]),
        "wrf_deform_backward_workspace_size": (S, [I32, I32, mp]),
        "wrf_deform_backward": (I32, [sp, mp, gp, P, I32, P, P, P, P, P, I32, P, S, P]),
        "wrf_status_read": (I32, [P]),
        "wrf_last_error": (C.c_char_p, []),
        "wrf_version": (I32, []),
        "wrf_selftest_wait": (I32, [I64, P, P]),
        "wrf_rssi": (I32, [sp, mp, gp, P, I32, P, P, P, S, P]),
        "wrf_loss_workspace_size": (S, [I32, I32, I32]),
        "wrf_loss": (I32, [P, P, I32, I32, I32, F, P, P, P, S, P]),
        "wrf_adam": (I32, [C.POINTER(AdamGroup), I32, I32, F, F, F, P]),
        "wrf_render_complex": (I32, [P, P, P, P, I64, I32, I32, gp, P, P]),
        "wrf_anneal_tx": (I32, [P, P, I32, P, I32, I32, F, I32, C.POINTER(C.c_float), P, P]),
        "wrf_multi_set_size": (S, [sp, mp, I32]),
        "wrf_multi_set_prepare": (I32, [sp, mp, I32, gp, P, S, P]),
        "wrf_multi_workspace_size": (S, [I32]),
        "wrf_deform_project_multi": (I32, [sp, mp, I32, P, P, P, I32, gp, P, I64, P, P, S, P]),
        "wrf_bin_multi": (I32, [P, P, I32, I32, gp, P, I64, P, P, P, S, P]),
        "wrf_render_multi": (I32, [P, P, P, P, P, I64, I32, gp, P, P]),
        "wrf_pipeline_create": (I32, [sp, mp, gp, I32, F, C.POINTER(P)]),
        "wrf_pipeline_step": (I32, [P, P, P]),
        "wrf_pipeline_wait": (I32, [P]),
        "wrf_pipeline_destroy": (I32, [P]),
        "wrf_paper_workspace_size": (S, [I32, I32]),
        "wrf_measure_alu_peaks": (I32, [C.POINTER(C.c_double)] * 3 + [P]),
        "wrf_paper_deform_project": (I32, [C.POINTER(PaperScene), C.POINTER(PaperMlp), gp, P, I32,
                                           P, P, S, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int) -> None:
    if status != WRF_OK:
        msg = load().wrf_last_error().decode(errors="replace")
        raise WrfError(int(status), msg)
