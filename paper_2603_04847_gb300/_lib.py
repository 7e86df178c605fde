"""ctypes binding of libgs (include/gs.h).  Argument marshalling only: every
step of the path runs in the library's CUDA kernels.  Importing works
without a GPU; calling a compute entry point without the built library or a
GPU raises.  There is no CPU fallback."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs.so")

c_int32, c_int64, c_float, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                  ctypes.c_void_p, ctypes.c_size_t)

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_NONFINITE, GS_ERR_UNSUPPORTED = range(6)
GS_FLAG_CAPACITY = 1
GS_FLAG_NONFINITE = 2
GS_FLAG_SORT_STALL = 4
GS_FLAG_NOT_SPD = 8
GS_MAX_BATCH = 64
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
                4: "GS_ERR_NONFINITE", 5: "GS_ERR_UNSUPPORTED"}


class gs_gaussians(ctypes.Structure):
    _fields_ = [("n", c_int32), ("sh_degree", c_int32), ("mean", c_void_p), ("log_scale", c_void_p),
                ("quat", c_void_p), ("opacity_logit", c_void_p), ("sh", c_void_p)]


class gs_gaussian_grads(ctypes.Structure):
    _fields_ = [("mean", c_void_p), ("log_scale", c_void_p), ("quat", c_void_p),
                ("opacity_logit", c_void_p), ("sh", c_void_p)]


class gs_cameras(ctypes.Structure):
    _fields_ = [("n_cams", c_int32), ("wh", c_void_p), ("K", c_void_p), ("Rt", c_void_p),
                ("near_plane", c_float), ("far_plane", c_float)]


class gs_batch(ctypes.Structure):
    _fields_ = [("B", c_int32), ("tile", c_int32), ("views", c_void_p), ("px_offset", c_void_p),
                ("tile_offset", c_void_p), ("n_pixels", c_int64), ("n_tiles", c_int32),
                ("_pad", c_int32)]


class gs_projected(ctypes.Structure):
    _fields_ = [("splat", c_void_p), ("rect", c_void_p), ("n_tiles", c_void_p), ("depth_key", c_void_p)]


class gs_adam(ctypes.Structure):
    _fields_ = [("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("step", c_void_p)]


class gs_tuning(ctypes.Structure):
    _fields_ = [("render_fwd_batch", c_int32), ("render_bwd_batch", c_int32), ("sort_blocks_per_sm", c_int32),
                ("sort_spin_limit", c_int32)]


class gs_adam_group(ctypes.Structure):
    _fields_ = [("p", c_void_p), ("g", c_void_p), ("m", c_void_p), ("v", c_void_p), ("n", c_int64),
                ("lr", c_float), ("_pad", c_int32)]


class gs_gaussians_f64(ctypes.Structure):
    _fields_ = gs_gaussians._fields_


class gs_gaussian_grads_f64(ctypes.Structure):
    _fields_ = gs_gaussian_grads._fields_


class gs_cameras_f64(ctypes.Structure):
    _fields_ = [("n_cams", c_int32), ("wh", c_void_p), ("K", c_void_p), ("Rt", c_void_p),
                ("near_plane", ctypes.c_double), ("far_plane", ctypes.c_double)]


class gs_projected_f64(ctypes.Structure):
    _fields_ = gs_projected._fields_


STRUCTS = [gs_gaussians, gs_gaussian_grads, gs_cameras, gs_batch, gs_projected, gs_adam, gs_tuning, gs_adam_group,
           gs_gaussians_f64, gs_gaussian_grads_f64, gs_cameras_f64, gs_projected_f64]

# name -> (restype, argtypes)
PROTOTYPES = {
    "gs_abi_version": (ctypes.c_int, []),
    "gs_last_error": (ctypes.c_char_p, []),
    "gs_struct_size": (c_size_t, [ctypes.c_int]),
    "gs_device_sm_count": (ctypes.c_int, []),
    "gs_set_tuning": (ctypes.c_int, [c_void_p]),
    "gs_get_tuning": (ctypes.c_int, [c_void_p]),
    "gs_adam_update_groups": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p]),
    "gs_project": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_sort_tiles_workspace": (ctypes.c_int, [c_int32, c_void_p, c_size_t, ctypes.POINTER(c_size_t)]),
    "gs_sort_tiles": (ctypes.c_int, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "gs_render_fwd": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_render_bwd_workspace": (ctypes.c_int, [c_int32, c_void_p, ctypes.POINTER(c_size_t)]),
    "gs_render_bwd": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_raster_bwd": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p,
                                     c_void_p, c_size_t, c_void_p]),
    "gs_raster_bwd_zeroed": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p,
                                            c_void_p, c_size_t, c_void_p]),
    "gs_project_bwd": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_size_t, c_void_p]),
    "gs_project_bwd_clearing": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                               c_void_p, c_size_t, c_void_p]),
    "gs_render_bwd_det_workspace": (ctypes.c_int, [c_int32, c_void_p, c_size_t, ctypes.POINTER(c_size_t)]),
    "gs_raster_bwd_det": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float,
                                         c_void_p, c_size_t, c_void_p, c_size_t, c_void_p]),
    "gs_render_bwd_det": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float,
                                         c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "track_reproj_workspace": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "track_reproj_fwd_bwd": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_size_t, c_void_p]),
    "track_reproj_fwd_bwd_det": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                                c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p,
                                                c_void_p, c_void_p, c_size_t, c_void_p]),
    "track_reproj_fwd_bwd_static": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                                   c_void_p, c_void_p, c_float, c_float, c_void_p, c_void_p,
                                                   c_void_p, c_void_p, c_void_p]),
    "pose_se3_update": (ctypes.c_int, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p]),
    "gs_adam_update": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "gs_step_advance": (ctypes.c_int, [c_void_p, c_void_p]),
    "gs_zero": (ctypes.c_int, [c_void_p, c_size_t, c_void_p]),
    "gs_batch_layout": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_gather_view_pixels": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "gs_photo_loss_workspace": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "gs_mcmc_workspace": (ctypes.c_int, [c_int32, ctypes.POINTER(c_size_t)]),
    "gs_mcmc_relocate": (ctypes.c_int, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_mcmc_noise": (ctypes.c_int, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float,
                                     c_void_p]),
    "gs_mcmc_grow": (ctypes.c_int, [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_mcmc_reset_moments": (ctypes.c_int, [c_int32, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p]),
    "sfm_ba_schur": (ctypes.c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, ctypes.c_double, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    "sfm_ba_pair_lists": (ctypes.c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sfm_ba_schur_pairs_workspace": (ctypes.c_int, [c_int64, c_int32, c_void_p]),
    "sfm_ba_schur_pairs": (ctypes.c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                          c_void_p, c_int32, ctypes.c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_size_t, c_void_p]),
    "sfm_ba_lm_accept": (ctypes.c_int, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "sfm_ba_objective": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                        c_float, c_void_p, c_void_p]),
    "sfm_ba_apply_step": (ctypes.c_int, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p]),
    "sfm_ba_solve_cameras": (ctypes.c_int, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sfm_ba_back_substitute": (ctypes.c_int, [c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                              c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sfm_ba_assemble": (ctypes.c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                       c_float, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p]),
    "gs_photo_loss": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_float, c_void_p,
                                     c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_project_f64": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_sort_tiles_f64": (ctypes.c_int, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                         c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "gs_render_fwd_f64": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_render_bwd_workspace_f64": (ctypes.c_int, [c_int32, c_void_p, ctypes.POINTER(c_size_t)]),
    "gs_raster_bwd_f64": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_double,
                                         c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_project_bwd_f64": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_size_t, c_void_p]),
    "gs_render_bwd_f64": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_double,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "pose_se3_update_f64": (ctypes.c_int, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                           c_void_p, c_void_p, c_void_p]),
}

_lib = None


class GsError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Loads libgs.so (built by paper_2603_04847_gb300.build); raises if
    it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise GsError("libgs.so is not built (%s); run paper_2603_04847_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    for i, s in enumerate(STRUCTS):
        if lib.gs_struct_size(i) != ctypes.sizeof(s):
            raise GsError("ABI mismatch for %s: C %d vs ctypes %d" % (s.__name__, lib.gs_struct_size(i),
                                                                      ctypes.sizeof(s)))
    if lib.gs_abi_version() != 5:
        raise GsError("unexpected libgs ABI version")
    _lib = lib
    return lib


def check(status: int, what: str):
    if status != GS_OK:
        msg = load().gs_last_error().decode(errors="replace")
        raise GsError("%s failed: %s (%s)" % (what, STATUS_NAMES.get(status, status), msg))
