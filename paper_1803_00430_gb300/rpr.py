"""ctypes binding of the C ABI declared in include/rpr.h.

Argument marshalling only: every step of the computation runs in the CUDA library
(``_build/librpr.so``, built by ``paper_1803_00430_gb300.build``).  Loading fails
loudly when the library is missing; there is no CPU fallback.

The raw entry points keep their C names (``rp_create``, ``rp_trace`` ...).  The
small classes below pass torch CUDA tensors (device memory) or numpy arrays (host
memory) through them.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref
from dataclasses import dataclass

import numpy as np

from . import build as _build

MAX_BANDS = 8
MAX_SH_ORDER = 3
MAX_SH = 16
MAX_SOURCES = 4096

RP_OK = 0
STATUS = {
    0: "RP_OK", -1: "RP_ERR_INVALID_ARG", -2: "RP_ERR_CUDA", -3: "RP_ERR_OOM", -4: "RP_ERR_CAPACITY",
    -5: "RP_ERR_STACK_OVERFLOW", -6: "RP_ERR_TIMEOUT", -7: "RP_ERR_NAN_INPUT", -8: "RP_ERR_EMPTY_SCENE",
    -9: "RP_ERR_NO_DEVICE", -10: "RP_ERR_TOO_LARGE", -11: "RP_ERR_BOUNDS",
}
RP_ERR = {v: k for k, v in STATUS.items()}
RP_MEM_HOST, RP_MEM_DEVICE = 0, 1
RP_FLAG_RAY_HASH, RP_FLAG_COUNT_VISITS, RP_FLAG_DEVICE_POSITIONS, RP_FLAG_FP32_PATHS = 1, 2, 4, 8
RP_FLAG_SHADOW_PACKETS, RP_FLAG_SHADOW_LANES = 16, 32
RP_MLP_FLAG_LEGACY_GEMM = 1


class rp_mesh_desc(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("tris", C.c_void_p), ("tri_material", C.c_void_p),
                ("absorption", C.c_void_p), ("scattering", C.c_void_p), ("num_verts", C.c_int32),
                ("num_tris", C.c_int32), ("num_materials", C.c_int32), ("num_bands", C.c_int32),
                ("memory", C.c_int32), ("ray_epsilon", C.c_float)]


class rp_scene_info(C.Structure):
    _fields_ = [("num_tris", C.c_int32), ("num_nodes", C.c_int32), ("max_depth", C.c_int32),
                ("num_bands", C.c_int32), ("bounds_lo", C.c_float * 3), ("bounds_hi", C.c_float * 3),
                ("ray_epsilon", C.c_float), ("build_ms", C.c_float), ("refit_ms", C.c_float)]


class rp_trace_params(C.Structure):
    _fields_ = [("num_rays", C.c_uint64), ("seed", C.c_uint64), ("first_ray", C.c_uint64), ("max_order", C.c_int32),
                ("sh_order", C.c_int32), ("num_bins", C.c_int32), ("min_order", C.c_int32),
                ("ir_rate_hz", C.c_float), ("speed_of_sound", C.c_float), ("source_radius", C.c_float),
                ("scene_id", C.c_uint32), ("budget_refill", C.c_int32), ("flags", C.c_int32)]


class rp_direct(C.Structure):
    _fields_ = [("visible", C.c_int32), ("bin", C.c_int32), ("dist", C.c_float), ("time", C.c_float),
                ("energy", C.c_float), ("sh", C.c_float * MAX_SH)]


class rp_trace_stats(C.Structure):
    _fields_ = [("escaped", C.c_double * MAX_BANDS), ("absorbed", C.c_double * MAX_BANDS),
                ("remaining", C.c_double * MAX_BANDS), ("late", C.c_double * MAX_BANDS),
                ("mfp_sum", C.c_double), ("mfp_sum_np", C.c_double), ("mfp_count", C.c_uint64),
                ("mfp_count_np", C.c_uint64), ("segments", C.c_uint64), ("shadow_rays", C.c_uint64),
                ("primaries", C.c_uint64), ("contributions", C.c_uint64), ("sphere_hits", C.c_uint64),
                ("waves", C.c_uint64), ("node_visits", C.c_uint64 * 2), ("tri_tests", C.c_uint64 * 2),
                ("hits_stored", C.c_uint64), ("fp64_reruns", C.c_uint64), ("packet_walks", C.c_uint64),
                ("packet_steps", C.c_uint64), ("error", C.c_int32),
                ("reserved", C.c_int32)]


class rp_estimate_params(C.Structure):
    _fields_ = [("ir_rate_hz", C.c_double), ("dt_update", C.c_double), ("tau", C.c_double)]


class rp_reverb_params(C.Structure):
    _fields_ = [("rt60_raw", C.c_double), ("rt60_smoothed", C.c_double), ("fit_hi_db", C.c_double),
                ("fit_lo_db", C.c_double), ("fit_r2", C.c_double), ("slope_db_per_s", C.c_double),
                ("intercept_db", C.c_double), ("i_total", C.c_double), ("g_reverb", C.c_double),
                ("e_direct", C.c_double), ("drr_db", C.c_double), ("predelay_s", C.c_double),
                ("range_kind", C.c_int32), ("n_fit", C.c_int32), ("fit_j0", C.c_int32),
                ("fit_j1", C.c_int32), ("xbar", C.c_double * MAX_SH)]


class rp_batch_item(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("listener", C.c_void_p), ("sources", C.c_void_p),
                ("num_sources", C.c_int32), ("scene_id", C.c_uint32), ("num_rays", C.c_uint64),
                ("first_ray", C.c_uint64)]


class rp_batch_tuning(C.Structure):
    _fields_ = [("chunk_rays", C.c_int32), ("shadow_steps", C.c_int32), ("paths_blocks_per_sm", C.c_int32),
                ("shadow_blocks_per_sm", C.c_int32), ("shadow_mode", C.c_int32)]


class rp_batch_info(C.Structure):
    _fields_ = [("num_items", C.c_int32), ("total_sources", C.c_int32), ("num_groups", C.c_int32),
                ("reserved", C.c_int32), ("total_rays", C.c_uint64), ("max_group_reflections", C.c_uint64)]


class rp_mlp_config(C.Structure):
    _fields_ = [("in_dim", C.c_int32), ("hidden", C.c_int32), ("layers", C.c_int32), ("out_dim", C.c_int32),
                ("max_batch", C.c_int32), ("flags", C.c_int32), ("seed", C.c_uint64)]


class rp_er_path(C.Structure):
    _fields_ = [("source", C.c_int32), ("order", C.c_int32), ("tri", C.c_int32 * 2), ("delay_s", C.c_double),
                ("energy", C.c_double * MAX_BANDS), ("sh", (C.c_double * MAX_SH) * MAX_BANDS)]


class rp_er_params(C.Structure):
    _fields_ = [("dt_update", C.c_double), ("tau_er", C.c_double), ("prune", C.c_double),
                ("hearing_threshold", C.c_double), ("n_er", C.c_int32), ("reserved", C.c_int32)]


N_COMB = 8


class rp_reverberator(C.Structure):
    _fields_ = [("mean_delay_s", C.c_double), ("generation", C.c_uint32), ("resampled", C.c_int32),
                ("t_comb", C.c_double * N_COMB), ("g_comb", (C.c_double * MAX_BANDS) * N_COMB),
                ("dir", (C.c_double * 3) * N_COMB), ("comb_in", (C.c_float * MAX_SH) * N_COMB),
                ("rot", ((C.c_float * 3) * 3) * N_COMB), ("J", ((C.c_float * MAX_SH) * MAX_SH) * N_COMB),
                ("D", ((C.c_float * MAX_SH) * MAX_SH) * MAX_BANDS)]


class rp_reverb_render_config(C.Structure):
    _fields_ = [("sample_rate", C.c_double), ("crossover_hz", C.c_double * (MAX_BANDS - 1)),
                ("max_delay_samples", C.c_int32), ("max_predelay_samples", C.c_int32)]


class rp_debug_limits(C.Structure):
    _fields_ = [("iter_cap", C.c_int32), ("spec_slots", C.c_int32), ("hit_cap", C.c_uint64),
                ("record_cap", C.c_uint64)]


class rp_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


# (name, argtypes) of every exported entry point, in header order
_SIGS = {
    "rp_status_string": ([C.c_int], C.c_char_p),
    "rp_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p], C.c_int),
    "rp_destroy": ([C.c_void_p], C.c_int),
    "rp_set_stream": ([C.c_void_p, C.c_void_p], C.c_int),
    "rp_scene_create": ([C.c_void_p, C.POINTER(rp_mesh_desc), C.POINTER(C.c_void_p)], C.c_int),
    "rp_scene_destroy": ([C.c_void_p], C.c_int),
    "rp_scene_info_get": ([C.c_void_p, C.POINTER(rp_scene_info)], C.c_int),
    "rp_scene_refit": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_int32], C.c_int),
    "rp_trace_reserve": ([C.c_void_p, C.POINTER(rp_trace_params), C.c_int32], C.c_int),
    "rp_trace": ([C.c_void_p, C.POINTER(rp_trace_params), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "rp_estimate": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                     C.POINTER(rp_estimate_params), C.c_void_p, C.c_void_p], C.c_int),
    "rp_update": ([C.c_void_p, C.POINTER(rp_trace_params), C.POINTER(rp_estimate_params), C.c_void_p,
                   C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                  C.c_int),
    "rp_reverb_configure": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                             C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_void_p], C.c_int),
    "rp_reverb_state_bytes": ([C.c_int32, C.c_int32, C.c_int32, C.POINTER(rp_reverb_render_config),
                               C.POINTER(C.c_int64)], C.c_int),
    "rp_reverb_render": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                          C.POINTER(rp_reverb_render_config), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p],
                         C.c_int),
    "rp_er_cache_create": ([C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)], C.c_int),
    "rp_er_cache_destroy": ([C.c_void_p], C.c_int),
    "rp_er_cache_reset": ([C.c_void_p], C.c_int),
    "rp_er_cache_read": ([C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "rp_trace_er": ([C.c_void_p, C.POINTER(rp_trace_params), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                     C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(rp_er_params), C.c_void_p, C.c_void_p], C.c_int),
    "rp_ir_cache_update": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_int32],
                           C.c_int),
    "rp_batch_create": ([C.c_void_p, C.POINTER(rp_batch_item), C.c_int32, C.POINTER(rp_trace_params),
                         C.POINTER(rp_estimate_params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.POINTER(C.c_void_p)], C.c_int),
    "rp_batch_destroy": ([C.c_void_p], C.c_int),
    "rp_batch_run": ([C.c_void_p, C.c_uint64, C.c_int], C.c_int),
    "rp_batch_set_tuning": ([C.c_void_p, C.POINTER(rp_batch_tuning)], C.c_int),
    "rp_batch_get_tuning": ([C.c_void_p, C.POINTER(rp_batch_tuning)], C.c_int),
    "rp_batch_info_get": ([C.c_void_p, C.POINTER(rp_batch_info)], C.c_int),
    "rp_batch_autotune": ([C.c_void_p, C.c_uint64, C.c_char_p, C.POINTER(rp_batch_tuning),
                           C.POINTER(C.c_double)], C.c_int),
    "rp_scene_features": ([C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "rp_mlp_features": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_void_p,
                         C.c_int32, C.c_void_p], C.c_int),
    "rp_mlp_create": ([C.c_void_p, C.POINTER(rp_mlp_config), C.POINTER(C.c_void_p)], C.c_int),
    "rp_mlp_destroy": ([C.c_void_p], C.c_int),
    "rp_mlp_param_count": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "rp_mlp_get_params": ([C.c_void_p, C.c_void_p], C.c_int),
    "rp_mlp_set_params": ([C.c_void_p, C.c_void_p], C.c_int),
    "rp_mlp_get_adam_state": ([C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)], C.c_int),
    "rp_mlp_set_adam_state": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32], C.c_int),
    "rp_mlp_set_normalization": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "rp_mlp_prepare": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "rp_mlp_forward": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32], C.c_int),
    "rp_mlp_loss_grad": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p],
                         C.c_int),
    "rp_mlp_train_step": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_float,
                           C.c_void_p], C.c_int),
    "rp_trace_noalloc": ([C.c_void_p, C.POINTER(rp_trace_params), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                          C.c_void_p, C.c_void_p], C.c_int),
    "rp_set_debug_limits": ([C.c_void_p, C.POINTER(rp_debug_limits)], C.c_int),
    "rp_measure_pipe_peaks": ([C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "rp_sync_status": ([C.c_void_p], C.c_int),
    "rp_profile_enable": ([C.c_void_p, C.c_int], C.c_int),
    "rp_profile_reset": ([C.c_void_p], C.c_int),
    "rp_profile_read": ([C.c_void_p, C.POINTER(rp_kernel_time), C.c_int32, C.POINTER(C.c_int32)], C.c_int),
}

_lib = None
_live = weakref.WeakSet()   # contexts and scenes still holding library objects
_closed = False


def _close_all():
    """Release library objects while the CUDA runtime is still alive (interpreter
    exit runs Python's atexit handlers before the C runtime's)."""
    global _closed
    for obj in sorted(list(_live), key=lambda o: 0 if isinstance(o, (Batch, MLP, ERCache)) else 1 if isinstance(o, Scene)
                      else 2):
        try:
            obj.close()
        except Exception:
            pass
    _closed = True


atexit.register(_close_all)


def checked_requested() -> bool:
    """RPR_CHECKED=1 in the environment selects the bounds-checked build of the library
    (compiled with RP_CHECKED: every node, triangle, reflection, record, key and
    histogram index is tested before use; a violation is reported as RP_ERR_BOUNDS)."""
    return os.environ.get("RPR_CHECKED", "0") not in ("", "0")


def library_path() -> str:
    return _build.lib_path(checked_requested())


def load(build_if_missing: bool = False):
    """Load librpr.so (optionally building it).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    checked = checked_requested()
    path = _build.lib_path(checked)
    if build_if_missing and not _build.up_to_date(checked):
        _build.build(checked=checked)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run python -m paper_1803_00430_gb300.build)")
    lib = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


class RprError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({load().rp_status_string(status).decode()})")


def check(status: int, what: str = "rp call"):
    if status != RP_OK:
        raise RprError(status, what)
    return status


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


@dataclass
class TraceParams:
    num_rays: int = 10000
    max_order: int = 20
    sh_order: int = 1
    num_bins: int = 1000
    min_order: int = 1
    ir_rate_hz: float = 1000.0
    speed_of_sound: float = 343.0
    source_radius: float = 0.5
    seed: int = 0xC0FFEE
    scene_id: int = 0
    budget_refill: int = 0
    flags: int = 0
    first_ray: int = 0

    def c(self) -> rp_trace_params:
        return rp_trace_params(int(self.num_rays), int(self.seed) & 0xFFFFFFFFFFFFFFFF, int(self.first_ray),
                               int(self.max_order),
                               int(self.sh_order), int(self.num_bins), int(self.min_order),
                               float(self.ir_rate_hz), float(self.speed_of_sound), float(self.source_radius),
                               int(self.scene_id) & 0xFFFFFFFF, int(self.budget_refill), int(self.flags))

    @property
    def K(self) -> int:
        return (self.sh_order + 1) ** 2


class Context:
    """rp_ctx on one device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = C.c_void_p()
        check(self.lib.rp_create(C.byref(h), int(device), _stream_handle(stream)), "rp_create")
        self.h = h
        self.device = device
        self.scenes = weakref.WeakSet()   # objects that hold library handles of this context
        self.deps = weakref.WeakSet()
        _live.add(self)

    def set_stream(self, stream):
        check(self.lib.rp_set_stream(self.h, _stream_handle(stream)), "rp_set_stream")

    def set_debug_limits(self, iter_cap: int = 0, hit_cap: int = 0, record_cap: int = 0, spec_slots: int = 0):
        """Lower limits that exercise the error paths (all zero: the normal limits);
        spec_slots limits the refill planner's speculative slots (-1: no store passes)."""
        lim = rp_debug_limits(iter_cap, spec_slots, hit_cap, record_cap)
        check(self.lib.rp_set_debug_limits(self.h, C.byref(lim)), "rp_set_debug_limits")

    def pipe_peaks(self) -> tuple:
        """(FP32 FMA instructions/s, FP32 min/max instructions/s) measured on the device."""
        f, m = C.c_double(), C.c_double()
        check(self.lib.rp_measure_pipe_peaks(self.h, C.byref(f), C.byref(m)), "rp_measure_pipe_peaks")
        return f.value, m.value

    def sync_status(self) -> int:
        return self.lib.rp_sync_status(self.h)

    def profile(self, enable: bool = True):
        check(self.lib.rp_profile_enable(self.h, int(enable)), "rp_profile_enable")

    def profile_reset(self):
        check(self.lib.rp_profile_reset(self.h), "rp_profile_reset")

    def profile_read(self) -> dict:
        n = C.c_int32()
        buf = (rp_kernel_time * 64)()
        check(self.lib.rp_profile_read(self.h, buf, 64, C.byref(n)), "rp_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                for i in range(min(n.value, 64))}

    def close(self):
        if getattr(self, "h", None) and not _closed:
            for d in list(self.deps):  # batches and networks before the scenes they use
                d.close()
            for sc in list(self.scenes):
                sc.close()
            self.lib.rp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """rp_scene: the mesh and its device BVH.  Arrays may be numpy (host) or torch
    CUDA tensors (device)."""

    def __init__(self, ctx: Context, verts, tris, tri_material, absorption, scattering,
                 ray_epsilon: float = 0.0):
        self.ctx = ctx
        self.lib = ctx.lib
        on_dev = hasattr(verts, "is_cuda") and verts.is_cuda
        if on_dev:
            import torch
            arrs = [verts.float().contiguous(), tris.int().contiguous(), tri_material.int().contiguous(),
                    absorption.float().contiguous(), scattering.float().contiguous()]
            assert all(isinstance(a, torch.Tensor) and a.is_cuda for a in arrs)
        else:
            arrs = [np.ascontiguousarray(verts, np.float32), np.ascontiguousarray(tris, np.int32),
                    np.ascontiguousarray(tri_material, np.int32), np.ascontiguousarray(absorption, np.float32),
                    np.ascontiguousarray(scattering, np.float32)]
        self._keep = arrs
        v, t, m, a, s = arrs
        B = int(a.shape[1]) if len(a.shape) == 2 else 1
        d = rp_mesh_desc(_ptr(v), _ptr(t), _ptr(m), _ptr(a), _ptr(s), int(v.shape[0]), int(t.shape[0]),
                         int(a.shape[0]), B, RP_MEM_DEVICE if on_dev else RP_MEM_HOST, float(ray_epsilon))
        self.B = B
        h = C.c_void_p()
        check(self.lib.rp_scene_create(ctx.h, C.byref(d), C.byref(h)), "rp_scene_create")
        self.h = h
        self._keep = None
        ctx.scenes.add(self)
        _live.add(self)

    @classmethod
    def from_scene(cls, ctx: Context, sc, **kw):
        return cls(ctx, sc.verts, sc.tris, sc.tri_material, sc.absorption, sc.scattering, **kw)

    def info(self) -> rp_scene_info:
        out = rp_scene_info()
        check(self.lib.rp_scene_info_get(self.h, C.byref(out)), "rp_scene_info_get")
        return out

    def refit(self, verts):
        """rp_scene_refit: new vertex positions (same triangles), BVH refitted on the device."""
        if hasattr(verts, "is_cuda") and verts.is_cuda:
            v = verts.float().contiguous()
            check(self.lib.rp_scene_refit(self.h, _ptr(v), v.shape[0], RP_MEM_DEVICE), "rp_scene_refit")
        else:
            v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
            check(self.lib.rp_scene_refit(self.h, _ptr(v), v.shape[0], RP_MEM_HOST), "rp_scene_refit")

    def close(self):
        if getattr(self, "h", None) and not _closed and getattr(self.ctx, "h", None):
            self.lib.rp_scene_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _struct_array(raw: bytes, ctype, n: int):
    arr = (ctype * n).from_buffer_copy(raw)
    return arr


def stats_to_dict(st: rp_trace_stats, B: int) -> dict:
    out = {k: np.array(getattr(st, k)[:B]) for k in ("escaped", "absorbed", "remaining", "late")}
    for k in ("mfp_sum", "mfp_sum_np", "mfp_count", "mfp_count_np", "segments", "shadow_rays", "primaries",
              "contributions", "sphere_hits", "waves", "hits_stored", "fp64_reruns", "packet_walks", "packet_steps",
              "error"):
        out[k] = getattr(st, k)
    out["node_visits"] = list(st.node_visits)
    out["tri_tests"] = list(st.tri_tests)
    out["mean_free_path"] = st.mfp_sum / st.mfp_count if st.mfp_count else float("nan")
    out["mean_free_path_np"] = st.mfp_sum_np / st.mfp_count_np if st.mfp_count_np else float("nan")
    return out


def direct_to_dict(raw, S: int, K: int) -> dict:
    arr = _struct_array(bytes(raw), rp_direct, S)
    return {"visible": np.array([a.visible for a in arr], bool), "bin": np.array([a.bin for a in arr]),
            "dist": np.array([a.dist for a in arr]), "time": np.array([a.time for a in arr]),
            "energy": np.array([a.energy for a in arr]),
            "sh": np.array([list(a.sh)[:K] for a in arr]).reshape(S, K)}


EP_FIELDS = ["rt60_raw", "rt60_smoothed", "fit_hi_db", "fit_lo_db", "fit_r2", "slope_db_per_s",
             "intercept_db", "i_total", "g_reverb", "e_direct", "drr_db", "predelay_s", "range_kind",
             "n_fit", "fit_j0", "fit_j1"]


def params_to_dict(raw, S: int, B: int, K: int) -> dict:
    arr = _struct_array(bytes(raw), rp_reverb_params, S * B)
    out = {f: np.array([getattr(a, f) for a in arr]).reshape(S, B) for f in EP_FIELDS}
    out["xbar"] = np.array([list(a.xbar)[:K] for a in arr]).reshape(S, B, K)
    return out


class DeviceTrace:
    """Device outputs of rp_trace: H (torch float32 [S,B,K,T] on cuda), direct
    (rp_direct[S] bytes), stats (rp_trace_stats bytes), optional ray hashes."""

    def __init__(self, S, B, K, T, want_hash=0, device="cuda"):
        import torch
        self.S, self.B, self.K, self.T = S, B, K, T
        self.H = torch.empty((S, B, K, T), dtype=torch.float32, device=device)
        self.direct = torch.zeros(max(S, 1) * C.sizeof(rp_direct), dtype=torch.uint8, device=device)
        self.stats = torch.zeros(C.sizeof(rp_trace_stats), dtype=torch.uint8, device=device)
        self.ray_hash = torch.zeros(max(want_hash, 1), dtype=torch.int64, device=device) if want_hash else None

    def stats_dict(self) -> dict:
        st = rp_trace_stats.from_buffer_copy(bytes(self.stats.cpu().numpy()))
        return stats_to_dict(st, self.B)

    def direct_dict(self) -> dict:
        return direct_to_dict(self.direct.cpu().numpy()[: self.S * C.sizeof(rp_direct)], self.S, self.K)

    def hashes(self) -> np.ndarray:
        return self.ray_hash.cpu().numpy().view(np.uint64)


def trace(scene: Scene, p: TraceParams, listener, sources, out: DeviceTrace | None = None,
          sync: bool = True) -> DeviceTrace:
    """One rp_trace with host positions; returns the device outputs."""
    lis = np.ascontiguousarray(listener, np.float32).reshape(3)
    src = np.ascontiguousarray(sources, np.float32).reshape(-1, 3)
    S = src.shape[0]
    if out is None:
        out = DeviceTrace(S, scene.B, p.K, p.num_bins,
                          want_hash=p.num_rays if p.flags & RP_FLAG_RAY_HASH else 0)
    cp = p.c()
    check(scene.lib.rp_trace(scene.h, C.byref(cp), _ptr(lis), _ptr(src), S, _ptr(out.H), _ptr(out.direct),
                             _ptr(out.stats), _ptr(out.ray_hash)), "rp_trace")
    if sync:
        check(scene.ctx.sync_status(), "rp_trace (device)")
    return out


def trace_noalloc(scene: Scene, p: TraceParams, listener, sources, out: DeviceTrace | None = None,
                  sync: bool = True) -> DeviceTrace:
    """rp_trace_noalloc (no memory allocation inside the call); host positions."""
    lis = np.ascontiguousarray(listener, np.float32).reshape(3)
    src = np.ascontiguousarray(sources, np.float32).reshape(-1, 3)
    S = src.shape[0]
    if out is None:
        out = DeviceTrace(S, scene.B, p.K, p.num_bins)
    cp = p.c()
    check(scene.lib.rp_trace_noalloc(scene.h, C.byref(cp), _ptr(lis), _ptr(src), S, _ptr(out.H),
                                     _ptr(out.direct), _ptr(out.stats)), "rp_trace_noalloc")
    if sync:
        check(scene.ctx.sync_status(), "rp_trace_noalloc (device)")
    return out


def reverb_configure(ctx: Context, H, params, S: int, B: int, K: int, ir_rate_hz: float, mean_free_path: float,
                     seed: int, rev=None, speed_of_sound: float = 343.0):
    """rp_reverb_configure; params: the device buffer rp_estimate filled; rev: the
    device state (a zeroed buffer is made when None).  Returns (rev, list of dicts)."""
    import torch
    T = H.shape[-1]
    if rev is None:
        rev = torch.zeros(S * C.sizeof(rp_reverberator), dtype=torch.uint8, device="cuda")
    check(ctx.lib.rp_reverb_configure(ctx.h, _ptr(H), _ptr(params), S, B, K, T, ir_rate_hz, mean_free_path,
                                      speed_of_sound, seed, _ptr(rev)), "rp_reverb_configure")
    check(ctx.sync_status(), "rp_reverb_configure (device)")
    arr = (rp_reverberator * S).from_buffer_copy(rev.cpu().numpy().tobytes())
    out = []
    for s in range(S):
        r = arr[s]
        out.append({"mean_delay": r.mean_delay_s, "generation": r.generation, "resampled": bool(r.resampled),
                    "t_comb": np.array(r.t_comb[:]), "g_comb": np.array([r.g_comb[i][:B] for i in range(N_COMB)]),
                    "dir": np.array([r.dir[i][:] for i in range(N_COMB)]),
                    "comb_in": np.array([r.comb_in[i][:K] for i in range(N_COMB)]),
                    "rot": np.array([[r.rot[i][p][:] for p in range(3)] for i in range(N_COMB)]),
                    "J": np.array([[r.J[i][k][:K] for k in range(K)] for i in range(N_COMB)]),
                    "D": np.array([[r.D[b][k][:K] for k in range(K)] for b in range(B)])})
    return rev, out


class Reverberator:
    """rp_reverb_render: the SH-domain Schroeder reverberators of S sources with their
    render state (device), rendering blocks of mono input."""

    def __init__(self, ctx: Context, S: int, B: int, K: int, crossover_hz, sample_rate: float = 48000.0,
                 max_delay_samples: int = 1 << 14, max_predelay_samples: int = 1 << 14):
        import torch
        self.ctx, self.S, self.B, self.K = ctx, S, B, K
        xo = list(crossover_hz) + [0.0] * (MAX_BANDS - 1 - len(crossover_hz))
        self.cfg = rp_reverb_render_config(sample_rate, (C.c_double * (MAX_BANDS - 1))(*xo), max_delay_samples,
                                           max_predelay_samples)
        n = C.c_int64()
        check(ctx.lib.rp_reverb_state_bytes(S, B, K, C.byref(self.cfg), C.byref(n)), "rp_reverb_state_bytes")
        self.state = torch.zeros(max(n.value, 1), dtype=torch.uint8, device="cuda")

    def render(self, rev, params, x):
        """x: device float32 [S][N] -> device float32 [S][K][N]."""
        import torch
        x = x.float().contiguous()
        N = x.shape[1]
        out = torch.empty((self.S, self.K, N), dtype=torch.float32, device="cuda")
        check(self.ctx.lib.rp_reverb_render(self.ctx.h, _ptr(rev), _ptr(params), self.S, self.B, self.K,
                                            C.byref(self.cfg), _ptr(x), N, _ptr(out), _ptr(self.state)),
              "rp_reverb_render")
        return out


def _er_paths_to_dict(raw: bytes, n: int, B: int, K: int) -> dict:
    arr = (rp_er_path * max(n, 1)).from_buffer_copy(raw) if n else []
    return {"source": np.array([arr[i].source for i in range(n)], np.int64),
            "order": np.array([arr[i].order for i in range(n)], np.int64),
            "tri1": np.array([arr[i].tri[0] for i in range(n)], np.int64),
            "tri2": np.array([arr[i].tri[1] for i in range(n)], np.int64),
            "delay": np.array([arr[i].delay_s for i in range(n)]),
            "energy": np.array([list(arr[i].energy)[:B] for i in range(n)]).reshape(n, B),
            "sh": np.array([[list(arr[i].sh[b])[:K] for b in range(B)] for i in range(n)]).reshape(n, B, K)}


class ERCache:
    """rp_er_cache: the early-reflection path cache of the temporal coherence (Section 5)."""

    def __init__(self, ctx: Context, num_bands: int, sh_order: int):
        self.ctx = ctx
        self.lib = ctx.lib
        self.B, self.K = num_bands, (sh_order + 1) ** 2
        h = C.c_void_p()
        check(self.lib.rp_er_cache_create(ctx.h, num_bands, sh_order, C.byref(h)), "rp_er_cache_create")
        self.h = h
        ctx.deps.add(self)
        _live.add(self)

    def reset(self):
        check(self.lib.rp_er_cache_reset(self.h), "rp_er_cache_reset")

    def read(self) -> dict:
        import torch
        n = C.c_int64()
        check(self.lib.rp_er_cache_read(self.h, None, 0, C.byref(n)), "rp_er_cache_read")
        buf = torch.empty(max(n.value, 1) * C.sizeof(rp_er_path), dtype=torch.uint8, device="cuda")
        check(self.lib.rp_er_cache_read(self.h, _ptr(buf), n.value, C.byref(n)), "rp_er_cache_read")
        torch.cuda.synchronize()
        return _er_paths_to_dict(buf.cpu().numpy().tobytes(), n.value, self.B, self.K)

    def trace(self, scene: "Scene", p: TraceParams, listener, sources, dt_update=0.0, tau_er=1.0, prune=0.0,
              hearing_threshold=0.0, n_er=100):
        """rp_trace_er with host positions: (DeviceTrace, rendered paths dict)."""
        import torch
        lis = np.ascontiguousarray(listener, np.float32).reshape(3)
        src = np.ascontiguousarray(sources, np.float32).reshape(-1, 3)
        S = src.shape[0]
        out = DeviceTrace(S, scene.B, p.K, p.num_bins)
        ep = rp_er_params(dt_update, tau_er, prune, hearing_threshold, n_er, 0)
        ren = torch.empty(max(n_er, 1) * C.sizeof(rp_er_path), dtype=torch.uint8, device="cuda")
        nr = torch.zeros(1, dtype=torch.int32, device="cuda")
        check(self.lib.rp_trace_er(scene.h, C.byref(p.c()), _ptr(lis), _ptr(src), S, _ptr(out.H), _ptr(out.direct),
                                   _ptr(out.stats), self.h, C.byref(ep), _ptr(ren), _ptr(nr)), "rp_trace_er")
        check(self.ctx.sync_status(), "rp_trace_er (device)")
        n = int(nr.item())
        return out, _er_paths_to_dict(ren.cpu().numpy().tobytes()[: max(n, 1) * C.sizeof(rp_er_path)], n, self.B,
                                      self.K)

    def close(self):
        if getattr(self, "h", None) and not _closed:
            self.lib.rp_er_cache_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ir_cache_update(ctx: Context, H, C_, dt_update: float, tau: float, first: bool):
    """rp_ir_cache_update: C_ = (1 - alpha) C_ + alpha H in place (device tensors)."""
    check(ctx.lib.rp_ir_cache_update(ctx.h, _ptr(H), _ptr(C_), H.numel(), dt_update, tau, int(first)),
          "rp_ir_cache_update")


class Batch:
    """rp_batch: many scenes traced and estimated in the same launches.  `items` is a
    list of (Scene, listener[3], sources[S,3], num_rays, scene_id).  Outputs are torch
    CUDA tensors owned by this object; item i's sources start at self.offsets[i]."""

    def __init__(self, ctx: Context, items, p: TraceParams, est_tau: float = 0.0, est_dt: float = 0.0,
                 estimate: bool = True):
        import torch
        self.ctx = ctx
        self.lib = ctx.lib
        self.p = p
        self._keep = []
        arr = (rp_batch_item * len(items))()
        self.offsets = []
        S_total = 0
        B = None
        for i, (scene, lis, src, rays, sid) in enumerate(items):
            lis = np.ascontiguousarray(lis, np.float32).reshape(3)
            src = np.ascontiguousarray(src, np.float32).reshape(-1, 3)
            self._keep += [lis, src]
            arr[i] = rp_batch_item(scene.h, lis.ctypes.data, src.ctypes.data, src.shape[0], int(sid),
                                   int(rays), 0)
            self.offsets.append(S_total)
            S_total += src.shape[0]
            B = scene.B
        self.S, self.B, self.K, self.T = S_total, B, p.K, p.num_bins
        dev = "cuda"
        self.H = torch.empty((S_total, B, p.K, p.num_bins), dtype=torch.float32, device=dev)
        self.direct = torch.zeros(max(S_total, 1) * C.sizeof(rp_direct), dtype=torch.uint8, device=dev)
        self.params = (torch.zeros(max(S_total * B, 1) * C.sizeof(rp_reverb_params), dtype=torch.uint8,
                                   device=dev) if estimate else None)
        self.stats = torch.zeros(C.sizeof(rp_trace_stats), dtype=torch.uint8, device=dev)
        ep = rp_estimate_params(float(p.ir_rate_hz), float(est_dt), float(est_tau))
        cp = p.c()
        h = C.c_void_p()
        check(self.lib.rp_batch_create(ctx.h, arr, len(items), C.byref(cp), C.byref(ep), _ptr(self.H),
                                       _ptr(self.direct), _ptr(self.params), _ptr(self.stats), C.byref(h)),
              "rp_batch_create")
        self.h = h
        self._keep = None
        ctx.deps.add(self)
        _live.add(self)

    def run(self, seed: int, use_graph: bool = False, sync: bool = True):
        check(self.lib.rp_batch_run(self.h, int(seed) & 0xFFFFFFFFFFFFFFFF, int(use_graph)), "rp_batch_run")
        if sync:
            check(self.ctx.sync_status(), "rp_batch_run (device)")

    def tuning(self) -> rp_batch_tuning:
        t = rp_batch_tuning()
        check(self.lib.rp_batch_get_tuning(self.h, C.byref(t)), "rp_batch_get_tuning")
        return t

    def set_tuning(self, t: rp_batch_tuning):
        check(self.lib.rp_batch_set_tuning(self.h, C.byref(t)), "rp_batch_set_tuning")

    def info(self) -> rp_batch_info:
        i = rp_batch_info()
        check(self.lib.rp_batch_info_get(self.h, C.byref(i)), "rp_batch_info_get")
        return i

    def autotune(self, seed: int, cache_path: str | None = None):
        t = rp_batch_tuning()
        ms = C.c_double()
        check(self.lib.rp_batch_autotune(self.h, int(seed), cache_path.encode() if cache_path else None,
                                         C.byref(t), C.byref(ms)), "rp_batch_autotune")
        return t, ms.value

    def stats_dict(self) -> dict:
        st = rp_trace_stats.from_buffer_copy(bytes(self.stats.cpu().numpy()))
        return stats_to_dict(st, self.B)

    def params_dict(self) -> dict:
        return params_to_dict(self.params.cpu().numpy().tobytes()[: self.S * self.B * C.sizeof(rp_reverb_params)],
                              self.S, self.B, self.K)

    def direct_dict(self) -> dict:
        return direct_to_dict(self.direct.cpu().numpy()[: self.S * C.sizeof(rp_direct)], self.S, self.K)

    def close(self):
        if getattr(self, "h", None) and not _closed and getattr(self.ctx, "h", None):
            self.lib.rp_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scene_features(scene: Scene) -> np.ndarray:
    out = (C.c_float * 10)()
    check(scene.lib.rp_scene_features(scene.h, out), "rp_scene_features")
    return np.array(list(out), np.float32)


def mlp_features(ctx: Context, H, scene_feats, ir_rate_hz: float, in_dim: int = 528):
    """Raw MLP features [S, in_dim] (torch float32 on the device) of H [S, B, K, T]:
    per band the windowed decay curve and the window length, then scene features."""
    import torch
    S, B, K, T = H.shape
    sf = torch.as_tensor(np.ascontiguousarray(scene_feats, np.float32).reshape(S, 10), device=H.device)
    X = torch.empty((S, in_dim), dtype=torch.float32, device=H.device)
    check(ctx.lib.rp_mlp_features(ctx.h, _ptr(H), S, B, K, T, float(ir_rate_hz), _ptr(sf), in_dim, _ptr(X)),
          "rp_mlp_features")
    return X


class MLP:
    """rp_mlp: the learned estimator (BF16 tensor-core GEMMs, FP32 masters, AdamW)."""

    def __init__(self, ctx: Context, in_dim=528, hidden=256, layers=3, out_dim=16, max_batch=4096, seed=1,
                 legacy_gemm: bool = False):
        self.ctx = ctx
        self.lib = ctx.lib
        self.cfg = rp_mlp_config(in_dim, hidden, layers, out_dim, max_batch,
                                 RP_MLP_FLAG_LEGACY_GEMM if legacy_gemm else 0, seed)
        h = C.c_void_p()
        check(self.lib.rp_mlp_create(ctx.h, C.byref(self.cfg), C.byref(h)), "rp_mlp_create")
        self.h = h
        n = C.c_int64()
        check(self.lib.rp_mlp_param_count(h, C.byref(n)), "rp_mlp_param_count")
        self.nparams = n.value
        ctx.deps.add(self)
        _live.add(self)

    def params(self):
        import torch
        p = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        check(self.lib.rp_mlp_get_params(self.h, _ptr(p)), "rp_mlp_get_params")
        torch.cuda.synchronize()
        return p

    def set_params(self, p):
        import torch
        p = torch.as_tensor(p, dtype=torch.float32, device="cuda").contiguous()
        check(self.lib.rp_mlp_set_params(self.h, _ptr(p)), "rp_mlp_set_params")
        torch.cuda.synchronize()

    def adam_state(self):
        import torch
        m = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        v = torch.empty_like(m)
        step = C.c_int32()
        check(self.lib.rp_mlp_get_adam_state(self.h, _ptr(m), _ptr(v), C.byref(step)), "rp_mlp_get_adam_state")
        torch.cuda.synchronize()
        return m, v, step.value

    def set_adam_state(self, m, v, step):
        check(self.lib.rp_mlp_set_adam_state(self.h, _ptr(m), _ptr(v), int(step)), "rp_mlp_set_adam_state")

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        a = [np.ascontiguousarray(x, np.float32) for x in (in_mean, in_std, out_mean, out_std)]
        check(self.lib.rp_mlp_set_normalization(self.h, *[x.ctypes.data_as(C.c_void_p) for x in a]),
              "rp_mlp_set_normalization")

    def prepare(self, X):
        import torch
        Xb = torch.empty(X.shape, dtype=torch.bfloat16, device="cuda")
        check(self.lib.rp_mlp_prepare(self.h, _ptr(X), X.shape[0], _ptr(Xb)), "rp_mlp_prepare")
        return Xb

    def forward(self, Xb, destandardize=True):
        import torch
        Y = torch.empty((Xb.shape[0], self.cfg.out_dim), dtype=torch.float32, device="cuda")
        check(self.lib.rp_mlp_forward(self.h, _ptr(Xb), Xb.shape[0], _ptr(Y), int(destandardize)), "rp_mlp_forward")
        return Y

    def loss_grad(self, Xb, T, mask):
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        check(self.lib.rp_mlp_loss_grad(self.h, _ptr(Xb), _ptr(T), _ptr(mask), Xb.shape[0], _ptr(loss), _ptr(g)),
              "rp_mlp_loss_grad")
        return loss, g

    def train_step(self, Xb, T, mask, lr, weight_decay=0.0, loss=None):
        check(self.lib.rp_mlp_train_step(self.h, _ptr(Xb), _ptr(T), _ptr(mask), Xb.shape[0], float(lr),
                                         float(weight_decay), _ptr(loss)), "rp_mlp_train_step")

    def close(self):
        if getattr(self, "h", None) and not _closed and getattr(self.ctx, "h", None):
            self.lib.rp_mlp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate(ctx: Context, H, direct, ir_rate_hz: float, dt_update: float = 0.0, tau: float = 0.0,
             state=None, out=None, sync: bool = True):
    """rp_estimate on device H [S,B,K,T]; returns (raw rp_reverb_params bytes tensor)."""
    import torch
    S, B, K, T = H.shape
    if out is None:
        out = torch.empty(max(S * B, 1) * C.sizeof(rp_reverb_params), dtype=torch.uint8, device=H.device)
    ep = rp_estimate_params(float(ir_rate_hz), float(dt_update), float(tau))
    check(ctx.lib.rp_estimate(ctx.h, _ptr(H), _ptr(direct), S, B, K, T, C.byref(ep), _ptr(out), _ptr(state)),
          "rp_estimate")
    if sync:
        check(ctx.sync_status(), "rp_estimate (device)")
    return out


def update(scene: Scene, p: TraceParams, ir_rate_hz: float, listener, sources, dt_update: float = 0.0,
           tau: float = 0.0, state=None, H_host=None, want=("H", "params", "direct", "stats")):
    """rp_update: host buffers in and out (copies inside the call)."""
    lis = np.ascontiguousarray(listener, np.float32).reshape(3)
    src = np.ascontiguousarray(sources, np.float32).reshape(-1, 3)
    S, B, K, T = src.shape[0], scene.B, p.K, p.num_bins
    H = H_host if H_host is not None else (np.empty((S, B, K, T), np.float32) if "H" in want else None)
    prm = (rp_reverb_params * max(S * B, 1))() if "params" in want else None
    dr = (rp_direct * max(S, 1))() if "direct" in want else None
    st = rp_trace_stats() if "stats" in want else None
    cp = p.c()
    ep = rp_estimate_params(float(ir_rate_hz), float(dt_update), float(tau))
    check(scene.lib.rp_update(scene.h, C.byref(cp), C.byref(ep), _ptr(lis), _ptr(src), S, _ptr(H),
                              prm, dr, C.byref(st) if st is not None else None, _ptr(state)), "rp_update")
    res = {"H": H}
    if prm is not None:
        res["params"] = params_to_dict(bytes(prm), S, B, K)
    if dr is not None:
        res["direct"] = direct_to_dict(bytes(dr), S, K)
    if st is not None:
        res["stats"] = stats_to_dict(st, B)
    return res
