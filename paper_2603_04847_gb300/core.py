"""Tensor containers and thin wrappers over the C ABI, one per entry point,
with the entry points' names.  PyTorch supplies device memory and streams;
every computation runs in libgs kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check

TILE = 16


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("libgs arguments must be contiguous CUDA tensors")


@dataclass
class Gaussians:
    """Raw Gaussian parameters (float32, CUDA): mean [N,3], log_scale [N,3],
    quat [N,4] (w,x,y,z), opacity_logit [N], sh [N,K,3]."""
    mean: torch.Tensor
    log_scale: torch.Tensor
    quat: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor

    @property
    def n(self):
        return self.mean.shape[0]

    @property
    def sh_degree(self):
        return int(round(self.sh.shape[1] ** 0.5)) - 1

    def tensors(self):
        return [self.mean, self.log_scale, self.quat, self.opacity_logit, self.sh]

    @property
    def f64(self) -> bool:
        """float64 parameters: the FP64 instantiation of the kernels."""
        return self.mean.dtype == torch.float64

    def _check_dtype(self):
        dt = self.mean.dtype
        if dt not in (torch.float32, torch.float64) or any(t.dtype != dt for t in self.tensors()):
            raise ValueError("Gaussian parameters must all be float32 or all float64")

    def c(self):
        _need_cuda(*self.tensors())
        self._check_dtype()
        cls = _lib.gs_gaussians_f64 if self.f64 else _lib.gs_gaussians
        return cls(self.n, self.sh_degree, self.mean.data_ptr(), self.log_scale.data_ptr(),
                   self.quat.data_ptr(), self.opacity_logit.data_ptr(), self.sh.data_ptr())

    def grads_c(self):
        _need_cuda(*self.tensors())
        self._check_dtype()
        cls = _lib.gs_gaussian_grads_f64 if self.f64 else _lib.gs_gaussian_grads
        return cls(self.mean.data_ptr(), self.log_scale.data_ptr(), self.quat.data_ptr(),
                   self.opacity_logit.data_ptr(), self.sh.data_ptr())

    @staticmethod
    def zeros_like(g: "Gaussians") -> "Gaussians":
        return Gaussians(*[torch.zeros_like(t) for t in g.tensors()])

    @staticmethod
    def from_numpy(d: dict, device="cuda", dtype=torch.float32) -> "Gaussians":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device).contiguous()
        return Gaussians(f(d["mean"]), f(d["log_scale"]), f(d["quat"]), f(d["opacity_logit"]).reshape(-1),
                         f(d["sh"]))


@dataclass
class Cameras:
    """All cameras: wh [V,2] int32, K [V,4] (fx,fy,cx,cy), Rt [V,12]
    world-to-camera (R row-major, t)."""
    wh: torch.Tensor
    K: torch.Tensor
    Rt: torch.Tensor
    near: float = 0.01
    far: float = 1e10
    wh_host: np.ndarray = None

    def __post_init__(self):
        if self.wh_host is None:
            self.wh_host = self.wh.detach().cpu().numpy().astype(np.int64)

    @property
    def V(self):
        return self.wh.shape[0]

    def c(self, Rt: torch.Tensor = None, f64: bool = False):
        """The C struct; f64: gs_cameras_f64 with the intrinsics in double
        and Rt (if given) float64."""
        if f64:
            if getattr(self, "_K64", None) is None:
                self._K64 = self.K.to(torch.float64).contiguous()
            Rt = self.Rt.to(torch.float64).contiguous() if Rt is None else Rt
            if Rt.dtype != torch.float64:
                raise ValueError("the FP64 path needs float64 poses")
            self._Rt64_keep = Rt
            _need_cuda(self.wh, self._K64, Rt)
            return _lib.gs_cameras_f64(self.V, self.wh.data_ptr(), self._K64.data_ptr(), Rt.data_ptr(),
                                       float(self.near), float(self.far))
        Rt = self.Rt if Rt is None else Rt
        _need_cuda(self.wh, self.K, Rt)
        return _lib.gs_cameras(self.V, self.wh.data_ptr(), self.K.data_ptr(), Rt.data_ptr(),
                               float(self.near), float(self.far))

    @staticmethod
    def from_numpy(wh, K, Rt, near=0.01, far=1e10, device="cuda") -> "Cameras":
        return Cameras(torch.as_tensor(np.asarray(wh), dtype=torch.int32, device=device).contiguous(),
                       torch.as_tensor(np.asarray(K), dtype=torch.float32, device=device).contiguous(),
                       torch.as_tensor(np.asarray(Rt), dtype=torch.float32, device=device).contiguous(),
                       near, far, np.asarray(wh).astype(np.int64))


def _layout_host(wh: np.ndarray, tile: int):
    """Pixel and tile offsets [B+1] of views of sizes wh [B,2]."""
    W, H = wh[:, 0].astype(np.int64), wh[:, 1].astype(np.int64)
    px = np.zeros(len(W) + 1, dtype=np.int64)
    px[1:] = np.cumsum(W * H)
    to = np.zeros(len(W) + 1, dtype=np.int64)
    to[1:] = np.cumsum(((W + tile - 1) // tile) * ((H + tile - 1) // tile))
    return px, to


class Batch:
    """A batch of views rendered together; per-slot images packed in slot
    order (pixel offsets) and tiles numbered globally (tile offsets).

    capacity=None sizes the batch's buffers for exactly these views.  With
    capacity=(n_pixels, n_tiles) the buffers hold any views whose totals fit,
    and the offsets are recomputed on the device from the device copy of the
    view ids (gs_batch_layout): views of other sizes can then be swapped in
    without re-allocating, including between replays of a captured step."""

    def __init__(self, cams: Cameras, views, tile: int = TILE, device="cuda", capacity=None):
        views = np.asarray(views, dtype=np.int64).reshape(-1)
        if not 1 <= len(views) <= _lib.GS_MAX_BATCH:
            raise ValueError("batch size must be 1..%d" % _lib.GS_MAX_BATCH)
        self.tile = tile
        self.B = len(views)
        self._set_host(cams, views)
        self.dynamic = capacity is not None
        if self.dynamic:
            self.n_pixels, self.n_tiles = int(capacity[0]), int(capacity[1])
            if self.pixels > self.n_pixels or int(self.tile_offset_host[-1]) > self.n_tiles:
                raise ValueError("views exceed the batch capacity")
        else:
            self.n_pixels = self.pixels
            self.n_tiles = int(self.tile_offset_host[-1])
        self.views = torch.as_tensor(views.astype(np.int32), device=device)
        self.px_offset = torch.as_tensor(self.px_offset_host, device=device)
        self.tile_offset = torch.as_tensor(self.tile_offset_host.astype(np.int32), device=device)

    def _set_host(self, cams: Cameras, views):
        wh = cams.wh_host[views]
        self.views_host = views
        self.W = wh[:, 0].copy()
        self.H = wh[:, 1].copy()
        self.px_offset_host, self.tile_offset_host = _layout_host(wh, self.tile)

    @property
    def pixels(self) -> int:
        """Pixels of the current views (n_pixels is the buffers' size)."""
        return int(self.px_offset_host[-1])

    @staticmethod
    def capacity_for(cams: Cameras, B: int, tile: int = TILE, views=None):
        """(n_pixels, n_tiles) that hold any B of `views` (default: all
        cameras): the sums over the B largest views."""
        wh = cams.wh_host if views is None else cams.wh_host[np.asarray(views, dtype=np.int64).reshape(-1)]
        W, H = wh[:, 0].astype(np.int64), wh[:, 1].astype(np.int64)
        px = np.sort(W * H)[::-1][:B].sum()
        tl = np.sort(((W + tile - 1) // tile) * ((H + tile - 1) // tile))[::-1][:B].sum()
        return int(px), int(tl)

    def fits(self, cams: "Cameras", views) -> bool:
        views = np.asarray(views, dtype=np.int64).reshape(-1)
        if len(views) != self.B:
            return False
        px, to = _layout_host(cams.wh_host[views], self.tile)
        return int(px[-1]) <= self.n_pixels and int(to[-1]) <= self.n_tiles

    def same_layout(self, cams: "Cameras", views) -> bool:
        """True when `views` can replace the current ones in place: any
        views within the capacity of a device-laid-out batch, else views of
        the current per-slot sizes."""
        if self.dynamic:
            return self.fits(cams, views)
        wh = cams.wh_host[np.asarray(views, dtype=np.int64).reshape(-1)]
        return len(wh) == self.B and np.array_equal(wh[:, 0], self.W) and np.array_equal(wh[:, 1], self.H)

    def set_views(self, cams: "Cameras", views, stream=None):
        """Replaces the batch's views in place on the device (buffers,
        kernels and captured graphs stay valid).  A device-laid-out batch
        recomputes its offsets on the stream; otherwise the views must have
        the current per-slot sizes."""
        if not self.same_layout(cams, views):
            raise ValueError("set_views: the views do not fit this batch's layout or capacity")
        views = np.asarray(views, dtype=np.int64).reshape(-1)
        self._set_host(cams, views)
        st = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(st):
            self.views.copy_(torch.as_tensor(views.astype(np.int32)), non_blocking=False)
            if self.dynamic:
                self.layout(cams, stream=st)

    def layout(self, cams: "Cameras", status: torch.Tensor = None, stream=None):
        """gs_batch_layout on this batch's own offset arrays."""
        lib = _lib.load()
        cc, bc = cams.c(), self.c()
        check(lib.gs_batch_layout(ctypes.byref(cc), ctypes.byref(bc), _p(self.px_offset), _p(self.tile_offset),
                                  _p(status), _stream(stream)), "gs_batch_layout")

    def c(self):
        return _lib.gs_batch(self.B, self.tile, self.views.data_ptr(), self.px_offset.data_ptr(),
                             self.tile_offset.data_ptr(), self.n_pixels, self.n_tiles, 0)

    def slot_image(self, buf: torch.Tensor, b: int) -> torch.Tensor:
        """View of slot b of a packed per-pixel buffer as [H, W, ...]."""
        a, e = int(self.px_offset_host[b]), int(self.px_offset_host[b + 1])
        return buf[a:e].reshape(int(self.H[b]), int(self.W[b]), *buf.shape[1:])


class Projected:
    """Per-(slot, Gaussian) records: splat [B*N,12] (float32, or float64 for
    the FP64 path), rect [B*N,4] u16, n_tiles [B*N] u32, depth_key [B*N]
    u32 (int16/int32 storage)."""

    def __init__(self, n: int, B: int, device="cuda", dtype=torch.float32):
        M = n * B
        self.splat = torch.empty((max(M, 1), 12), dtype=dtype, device=device)
        self.rect = torch.empty((max(M, 1), 4), dtype=torch.int16, device=device)
        self.n_tiles = torch.zeros((max(M, 1),), dtype=torch.int32, device=device)
        self.depth_key = torch.empty((max(M, 1),), dtype=torch.int32, device=device)

    @property
    def f64(self) -> bool:
        return self.splat.dtype == torch.float64

    def c(self):
        cls = _lib.gs_projected_f64 if self.f64 else _lib.gs_projected
        return cls(self.splat.data_ptr(), self.rect.data_ptr(), self.n_tiles.data_ptr(), self.depth_key.data_ptr())


class TileLists:
    """Sorted tile instances: tiles [cap] u32 (tile id), vals [cap] u32
    (record), ranges [2*n_tiles] u32, n_instances [1] u32, sort workspace."""

    def __init__(self, n: int, batch: Batch, capacity: int, device="cuda"):
        lib = _lib.load()
        self.capacity = int(capacity)
        self.tiles = torch.empty(self.capacity, dtype=torch.int32, device=device)
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=device)
        self.ranges = torch.zeros(max(2 * batch.n_tiles, 2), dtype=torch.int32, device=device)
        self.n_instances = torch.zeros(1, dtype=torch.int32, device=device)
        ws = ctypes.c_size_t(0)
        bc = batch.c()
        check(lib.gs_sort_tiles_workspace(n, ctypes.byref(bc), self.capacity, ctypes.byref(ws)),
              "gs_sort_tiles_workspace")
        self.ws = torch.empty(max(ws.value, 256), dtype=torch.uint8, device=device)


def new_status(device="cuda"):
    return torch.zeros(1, dtype=torch.int32, device=device)


# ---------------------------------------------------------------------------
# thin wrappers, same names as the C entry points


def _fn(lib, name, f64):
    """The entry point `name`, or its FP64 instantiation `name_f64`."""
    return getattr(lib, name + "_f64") if f64 else getattr(lib, name)


def gs_project(g: Gaussians, cams: Cameras, batch: Batch, proj: Projected, status: torch.Tensor,
               Rt: torch.Tensor = None, stream=None):
    lib = _lib.load()
    gc, cc, bc, pc = g.c(), cams.c(Rt, f64=g.f64), batch.c(), proj.c()
    check(_fn(lib, "gs_project", g.f64)(ctypes.byref(gc), ctypes.byref(cc), ctypes.byref(bc), ctypes.byref(pc),
                                        _p(status), _stream(stream)), "gs_project")


def gs_sort_tiles(n: int, cams: Cameras, batch: Batch, proj: Projected, tl: TileLists, status: torch.Tensor,
                  Rt: torch.Tensor = None, stream=None):
    lib = _lib.load()
    cc, bc, pc = cams.c(Rt, f64=proj.f64), batch.c(), proj.c()
    check(_fn(lib, "gs_sort_tiles", proj.f64)(n, ctypes.byref(cc), ctypes.byref(bc), ctypes.byref(pc), _p(tl.tiles),
                                              _p(tl.vals), tl.capacity, _p(tl.ranges), _p(tl.n_instances),
                                              _p(tl.ws), tl.ws.numel(), _p(status), _stream(stream)),
          "gs_sort_tiles")


def gs_render_fwd(batch: Batch, cams: Cameras, proj: Projected, tl: TileLists, bg: torch.Tensor,
                  image: torch.Tensor, T_final: torch.Tensor, n_contrib: torch.Tensor, Rt=None, stream=None,
                  n_added: torch.Tensor = None):
    lib = _lib.load()
    _need_cuda(bg, image, T_final, n_contrib, n_added)
    cc, bc, pc = cams.c(Rt, f64=proj.f64), batch.c(), proj.c()
    check(_fn(lib, "gs_render_fwd", proj.f64)(ctypes.byref(bc), ctypes.byref(cc), ctypes.byref(pc), _p(tl.vals),
                                              _p(tl.ranges), _p(bg), _p(image), _p(T_final), _p(n_contrib),
                                              _p(n_added), _stream(stream)),
          "gs_render_fwd")


def render_bwd_workspace_bytes(n: int, batch: Batch, f64: bool = False) -> int:
    lib = _lib.load()
    ws = ctypes.c_size_t(0)
    bc = batch.c()
    check(_fn(lib, "gs_render_bwd_workspace", f64)(n, ctypes.byref(bc), ctypes.byref(ws)), "gs_render_bwd_workspace")
    return ws.value


def render_bwd_det_workspace_bytes(n: int, batch: Batch, capacity: int) -> int:
    lib = _lib.load()
    ws = ctypes.c_size_t(0)
    bc = batch.c()
    check(lib.gs_render_bwd_det_workspace(n, ctypes.byref(bc), int(capacity), ctypes.byref(ws)),
          "gs_render_bwd_det_workspace")
    return ws.value


def gs_raster_bwd_det(g: Gaussians, cams: Cameras, batch: Batch, proj: Projected, tl: TileLists, bg, image,
                      T_final, n_contrib, v_image, target, l1_weight: float, loss, ws: torch.Tensor, Rt=None,
                      stream=None):
    """gs_raster_bwd with tile-order-independent results (gs_raster_bwd_det);
    ws from render_bwd_det_workspace_bytes(n, batch, tl.capacity)."""
    lib = _lib.load()
    if g.f64:
        raise _lib.GsError("gs_raster_bwd_det is FP32 only")
    _need_cuda(bg, T_final, n_contrib, ws, image, v_image, target, loss)
    gc, cc, bc, pc = g.c(), cams.c(Rt), batch.c(), proj.c()
    check(lib.gs_raster_bwd_det(ctypes.byref(gc), ctypes.byref(cc), ctypes.byref(bc), ctypes.byref(pc),
                                _p(tl.vals), _p(tl.ranges), _p(tl.n_instances), _p(bg), _p(image), _p(T_final),
                                _p(n_contrib), _p(v_image), _p(target), float(l1_weight), _p(loss), tl.capacity,
                                _p(ws), ws.numel(), _stream(stream)), "gs_raster_bwd_det")


def gs_render_bwd(g: Gaussians, cams: Cameras, batch: Batch, proj: Projected, tl: TileLists,
                  bg: torch.Tensor, image, T_final, n_contrib, v_image, target, l1_weight: float,
                  loss, dg: Gaussians, g_pose_tangent: torch.Tensor, ws: torch.Tensor, Rt=None, stream=None):
    lib = _lib.load()
    _need_cuda(bg, T_final, n_contrib, g_pose_tangent, ws, image, v_image, target, loss)
    gc, cc, bc, pc, dgc = g.c(), cams.c(Rt, f64=g.f64), batch.c(), proj.c(), dg.grads_c()
    check(_fn(lib, "gs_render_bwd", g.f64)(ctypes.byref(gc), ctypes.byref(cc), ctypes.byref(bc), ctypes.byref(pc),
                                           _p(tl.vals), _p(tl.ranges), _p(bg), _p(image), _p(T_final),
                                           _p(n_contrib), _p(v_image), _p(target), float(l1_weight), _p(loss),
                                           ctypes.byref(dgc), _p(g_pose_tangent), _p(ws), ws.numel(),
                                           _stream(stream)), "gs_render_bwd")


def gs_raster_bwd(g: Gaussians, cams: Cameras, batch: Batch, proj: Projected, tl: TileLists, bg, image,
                  T_final, n_contrib, v_image, target, l1_weight: float, loss, ws: torch.Tensor, Rt=None,
                  stream=None, records_zeroed: bool = False):
    """records_zeroed: the caller has zeroed the screen-space records at the
    start of ws (gs_raster_bwd_zeroed; FP32 only)."""
    lib = _lib.load()
    _need_cuda(bg, T_final, n_contrib, ws, image, v_image, target, loss)
    gc, cc, bc, pc = g.c(), cams.c(Rt, f64=g.f64), batch.c(), proj.c()
    if records_zeroed and g.f64:
        raise _lib.GsError("gs_raster_bwd_zeroed is FP32 only")
    fn = lib.gs_raster_bwd_zeroed if records_zeroed else _fn(lib, "gs_raster_bwd", g.f64)
    check(fn(ctypes.byref(gc), ctypes.byref(cc), ctypes.byref(bc), ctypes.byref(pc),
             _p(tl.vals), _p(tl.ranges), _p(bg), _p(image), _p(T_final),
             _p(n_contrib), _p(v_image), _p(target), float(l1_weight), _p(loss),
             _p(ws), ws.numel(), _stream(stream)), "gs_raster_bwd")


def gs_project_bwd(g: Gaussians, cams: Cameras, batch: Batch, proj: Projected, dg: Gaussians,
                   g_pose_tangent: torch.Tensor, ws: torch.Tensor, Rt=None, stream=None, clear_records: bool = False):
    """clear_records: gs_project_bwd_clearing, which leaves the screen-space
    records of ws zero behind it (FP32 only)."""
    lib = _lib.load()
    _need_cuda(g_pose_tangent, ws)
    if clear_records and g.f64:
        raise _lib.GsError("gs_project_bwd_clearing is FP32 only")
    gc, cc, bc, pc, dgc = g.c(), cams.c(Rt, f64=g.f64), batch.c(), proj.c(), dg.grads_c()
    fn = lib.gs_project_bwd_clearing if clear_records else _fn(lib, "gs_project_bwd", g.f64)
    check(fn(ctypes.byref(gc), ctypes.byref(cc), ctypes.byref(bc), ctypes.byref(pc), ctypes.byref(dgc),
             _p(g_pose_tangent), _p(ws), ws.numel(), _stream(stream)), "gs_project_bwd")


def photo_loss_workspace_bytes(batch: Batch) -> int:
    lib = _lib.load()
    bc = batch.c()
    ws = ctypes.c_size_t(0)
    check(lib.gs_photo_loss_workspace(ctypes.byref(bc), ctypes.byref(ws)), "gs_photo_loss_workspace")
    return ws.value


def gs_photo_loss(cams: Cameras, batch: Batch, image: torch.Tensor, target: torch.Tensor, l1_weight: float,
                  ssim_weight: float, loss, v_image: torch.Tensor, ws: torch.Tensor, Rt=None, stream=None):
    """Eq. 5 (L1 + SSIM) of every slot: loss (device double [1], may be
    None) += the batch's photometric loss; v_image [P,3] = dL/dimage."""
    lib = _lib.load()
    _need_cuda(image, target, v_image, ws, loss)
    cc, bc = cams.c(Rt), batch.c()
    check(lib.gs_photo_loss(ctypes.byref(cc), ctypes.byref(bc), _p(image), _p(target), float(l1_weight),
                            float(ssim_weight), _p(loss), _p(v_image), _p(ws), ws.numel() * ws.element_size(),
                            _stream(stream)), "gs_photo_loss")


def sfm_ba_assemble(X: torch.Tensor, cams: Cameras, obs_point: torch.Tensor, obs_cam: torch.Tensor,
                    obs_xy: torch.Tensor, delta: float, U, Vp, gc, gp, Wo, objective=None, Rt=None, stream=None):
    """The IRLS normal-equation blocks of one LM iteration of Eq. 4 (all
    float64 outputs, += except Wo): U [V,36], Vp [P,9], gc [V,6], gp [P,3],
    Wo [M,18], objective [1]."""
    lib = _lib.load()
    _need_cuda(X, obs_point, obs_cam, obs_xy, U, Vp, gc, gp, Wo, objective)
    cc = cams.c(Rt)
    check(lib.sfm_ba_assemble(_p(X), X.shape[0], ctypes.byref(cc), _p(obs_point), _p(obs_cam), _p(obs_xy),
                              obs_point.shape[0], float(delta), _p(U), _p(Vp), _p(gc), _p(gp), _p(Wo),
                              _p(objective), _stream(stream)), "sfm_ba_assemble")


def sfm_ba_schur(U, Vp, gc, gp, Wo, obs_cam, point_obs_offset, point_obs, lam, S, rhs, Vinv, stream=None):
    """Points eliminated from the damped LM system of Eq. 4: S [6V,6V], rhs
    [6V], Vinv [P,9] written (float64 device tensors).  lam: the damping, a
    float or a device double tensor [1] read on the device."""
    lib = _lib.load()
    _need_cuda(U, Vp, gc, gp, Wo, obs_cam, point_obs_offset, point_obs, S, rhs, Vinv)
    lam_dev = lam if isinstance(lam, torch.Tensor) else None
    _need_cuda(lam_dev)
    check(lib.sfm_ba_schur(U.shape[0], Vp.shape[0], obs_cam.shape[0], _p(U), _p(Vp), _p(gc), _p(gp), _p(Wo),
                           _p(obs_cam), _p(point_obs_offset), _p(point_obs), 0.0 if lam_dev is not None else float(lam),
                           _p(lam_dev), _p(S), _p(rhs), _p(Vinv), _stream(stream)), "sfm_ba_schur")


PAIR_CHUNK = 256


def sfm_ba_pair_lists(n_cams, n_points, obs_cam, point_obs_offset, point_obs, chunk=PAIR_CHUNK):
    """The host-side plan of the elimination by camera pairs
    (sfm_ba_pair_lists) from host arrays: dict of numpy arrays inc [n_inc,3],
    pair_cams [n_pairs,2], pair_chunks [n_pairs+1], chunk_start
    [n_chunks+1]."""
    lib = _lib.load()
    oc = np.ascontiguousarray(obs_cam, dtype=np.int32)
    off = np.ascontiguousarray(point_obs_offset, dtype=np.int64)
    ids = np.ascontiguousarray(point_obs, dtype=np.int32)
    hp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    n_inc, n_pairs, n_chunks = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    args = (int(n_cams), int(n_points), oc.shape[0], hp(oc), hp(off), hp(ids), int(chunk), ctypes.byref(n_inc),
            ctypes.byref(n_pairs), ctypes.byref(n_chunks))
    check(lib.sfm_ba_pair_lists(*args, None, None, None, None), "sfm_ba_pair_lists")
    out = dict(inc=np.zeros((n_inc.value, 3), np.int32), pair_cams=np.zeros((n_pairs.value, 2), np.int32),
               pair_chunks=np.zeros(n_pairs.value + 1, np.int32), chunk_start=np.zeros(n_chunks.value + 1, np.int64))
    check(lib.sfm_ba_pair_lists(*args, hp(out["inc"]), hp(out["pair_cams"]), hp(out["pair_chunks"]),
                                hp(out["chunk_start"])), "sfm_ba_pair_lists")
    return out


def sfm_ba_schur_pairs_workspace(n_obs, n_chunks):
    lib = _lib.load()
    b = ctypes.c_size_t()
    check(lib.sfm_ba_schur_pairs_workspace(int(n_obs), int(n_chunks), ctypes.byref(b)), "sfm_ba_schur_pairs_workspace")
    return b.value


def sfm_ba_schur_pairs(U, Vp, gc, gp, Wo, obs_cam, point_obs_offset, point_obs, plan, lam, S, rhs, Vinv, ws,
                       stream=None):
    """sfm_ba_schur's outputs summed by camera pairs (sfm_ba_schur_pairs):
    plan = the device copies (int32 / int64 tensors) of sfm_ba_pair_lists'
    arrays; ws a device workspace of sfm_ba_schur_pairs_workspace bytes."""
    lib = _lib.load()
    _need_cuda(U, Vp, gc, gp, Wo, obs_cam, point_obs_offset, point_obs, S, rhs, Vinv, ws, *plan.values())
    lam_dev = lam if isinstance(lam, torch.Tensor) else None
    _need_cuda(lam_dev)
    check(lib.sfm_ba_schur_pairs(U.shape[0], Vp.shape[0], obs_cam.shape[0], _p(U), _p(Vp), _p(gc), _p(gp), _p(Wo),
                                 _p(obs_cam), _p(point_obs_offset), _p(point_obs), _p(plan["inc"]),
                                 _p(plan["pair_cams"]), plan["pair_cams"].shape[0], _p(plan["pair_chunks"]),
                                 _p(plan["chunk_start"]), plan["chunk_start"].shape[0] - 1,
                                 0.0 if lam_dev is not None else float(lam), _p(lam_dev), _p(S), _p(rhs), _p(Vinv),
                                 _p(ws), ws.numel(), _stream(stream)), "sfm_ba_schur_pairs")


def sfm_ba_lm_accept(objective, lam, Rt, X, Rt_trial, X_trial, n_accepted=None, history=None, n_iter=None,
                     stream=None):
    """The LM accept / reject on the device (sfm_ba_lm_accept): objective
    [2] (current, trial) and lam [1] device doubles; Rt, X take the trial
    values when the trial objective is lower."""
    lib = _lib.load()
    _need_cuda(objective, lam, Rt, X, Rt_trial, X_trial, n_accepted, history, n_iter)
    check(lib.sfm_ba_lm_accept(Rt.shape[0], X.shape[0], _p(objective), _p(lam), _p(Rt), _p(X), _p(Rt_trial),
                               _p(X_trial), _p(n_accepted), _p(history),
                               0 if history is None else history.numel(), _p(n_iter), _stream(stream)),
          "sfm_ba_lm_accept")


def sfm_ba_objective(X, cams: Cameras, obs_point, obs_cam, obs_xy, delta: float, objective, Rt=None, stream=None):
    """objective (device double [1]) += the objective of Eq. 4."""
    lib = _lib.load()
    _need_cuda(X, obs_point, obs_cam, obs_xy, objective)
    cc = cams.c(Rt)
    check(lib.sfm_ba_objective(_p(X), X.shape[0], ctypes.byref(cc), _p(obs_point), _p(obs_cam), _p(obs_xy),
                               obs_point.shape[0], float(delta), _p(objective), _stream(stream)), "sfm_ba_objective")


def sfm_ba_apply_step(Rt, X, dc, dp, Rt_out, X_out, stream=None):
    """Rt_out = Exp(dc) Rt per camera, X_out = X + dp (float32 outputs)."""
    lib = _lib.load()
    _need_cuda(Rt, X, dc, dp, Rt_out, X_out)
    check(lib.sfm_ba_apply_step(Rt.shape[0], X.shape[0], _p(Rt), _p(X), _p(dc), _p(dp), _p(Rt_out), _p(X_out),
                                _stream(stream)), "sfm_ba_apply_step")


def sfm_ba_solve_cameras(S, rhs, dc, status=None, stream=None):
    """dc [V,6] of the reduced camera system with camera 0 fixed (S is
    overwritten by its factor)."""
    lib = _lib.load()
    _need_cuda(S, rhs, dc, status)
    check(lib.sfm_ba_solve_cameras(dc.shape[0], _p(S), _p(rhs), _p(dc), _p(status), _stream(stream)),
          "sfm_ba_solve_cameras")


def sfm_ba_back_substitute(Vinv, Vp, gp, Wo, obs_cam, point_obs_offset, point_obs, dc, dp, stream=None):
    """dp [P,3] = V_k^-1 (-gp_k - sum_i W_ik^T dc_i) (written)."""
    lib = _lib.load()
    _need_cuda(Vinv, Vp, gp, Wo, obs_cam, point_obs_offset, point_obs, dc, dp)
    check(lib.sfm_ba_back_substitute(dc.shape[0], Vp.shape[0], obs_cam.shape[0], _p(Vinv), _p(Vp), _p(gp), _p(Wo),
                                     _p(obs_cam), _p(point_obs_offset), _p(point_obs), _p(dc), _p(dp),
                                     _stream(stream)), "sfm_ba_back_substitute")


def gs_mcmc_relocate(g: Gaussians, u: torch.Tensor, src: torch.Tensor, n_dead=None, stream=None):
    """MCMC relocation of the dead Gaussians of g in place (u: float64
    uniforms, one per dead Gaussian in index order; src [N] int32 out)."""
    lib = _lib.load()
    _need_cuda(*g.tensors(), u, src, n_dead)
    ws_bytes = ctypes.c_size_t(0)
    check(lib.gs_mcmc_workspace(g.n, ctypes.byref(ws_bytes)), "gs_mcmc_workspace")
    ws = torch.empty(max(ws_bytes.value, 256), dtype=torch.uint8, device=g.mean.device)
    check(lib.gs_mcmc_relocate(g.n, g.sh_degree, _p(g.mean), _p(g.log_scale), _p(g.quat), _p(g.opacity_logit),
                               _p(g.sh), _p(u), u.numel(), _p(src), _p(n_dead), _p(ws), ws.numel(),
                               _stream(stream)), "gs_mcmc_relocate")


def gs_mcmc_grow(g: Gaussians, n: int, u: torch.Tensor, src: torch.Tensor, stream=None):
    """Growth step: g holds n live rows plus room for len(u) more; rows
    n.. receive the new Gaussians (u: float64 uniforms, one per new
    Gaussian; src [len(u)] int32 out: each new one's source)."""
    lib = _lib.load()
    _need_cuda(*g.tensors(), u, src)
    n_add = u.numel()
    if n + n_add > g.n:
        raise ValueError("gs_mcmc_grow: the parameter arrays hold %d rows, need %d" % (g.n, n + n_add))
    ws_bytes = ctypes.c_size_t(0)
    check(lib.gs_mcmc_workspace(n, ctypes.byref(ws_bytes)), "gs_mcmc_workspace")
    ws = torch.empty(max(ws_bytes.value, 256), dtype=torch.uint8, device=g.mean.device)
    check(lib.gs_mcmc_grow(n, n_add, g.sh_degree, _p(g.mean), _p(g.log_scale), _p(g.quat), _p(g.opacity_logit),
                           _p(g.sh), _p(u), _p(src), _p(ws), ws.numel(), _stream(stream)), "gs_mcmc_grow")


def gs_mcmc_reset_moments(n_rows: int, src: torch.Tensor, row0: int, moments, stream=None):
    """Zero rows row0 + k and src[k] (src[k] >= 0) of every (m, v) pair in
    `moments` (tensors with n_rows rows)."""
    lib = _lib.load()
    arr = (_lib.gs_adam_group * len(moments))()
    for i, (m, v) in enumerate(moments):
        _need_cuda(m, v)
        arr[i] = _lib.gs_adam_group(0, 0, m.data_ptr(), v.data_ptr(), m.numel(), 0.0, 0)
    check(lib.gs_mcmc_reset_moments(n_rows, _p(src), src.numel(), row0, arr, len(moments), _stream(stream)),
          "gs_mcmc_reset_moments")


def gs_mcmc_noise(g: Gaussians, eta: torch.Tensor, noise_lr: float, stream=None):
    """mean += noise_lr * sigmoid(-100 (o - 0.005)) * Sigma eta, in place."""
    lib = _lib.load()
    _need_cuda(*g.tensors(), eta)
    check(lib.gs_mcmc_noise(g.n, _p(g.mean), _p(g.log_scale), _p(g.quat), _p(g.opacity_logit), _p(eta),
                            float(noise_lr), _stream(stream)), "gs_mcmc_noise")


def track_workspace_bytes(batch: Batch) -> int:
    lib = _lib.load()
    ws = ctypes.c_size_t(0)
    bc = batch.c()
    check(lib.track_reproj_workspace(ctypes.byref(bc), ctypes.byref(ws)), "track_reproj_workspace")
    return ws.value


def track_reproj_fwd_bwd(X, obs_point, obs_xy, view_obs_offset, cams: Cameras, batch: Batch, delta: float,
                         weight: float, loss, grad_X, g_pose_tangent, n_masked, ws, Rt=None, stream=None,
                         deterministic: bool = False):
    """The track term of Eq. 6; deterministic: track_reproj_fwd_bwd_det
    (bit-identical results from run to run)."""
    lib = _lib.load()
    _need_cuda(X, obs_point, obs_xy, view_obs_offset, loss, grad_X, g_pose_tangent, n_masked, ws)
    cc, bc = cams.c(Rt), batch.c()
    fn = lib.track_reproj_fwd_bwd_det if deterministic else lib.track_reproj_fwd_bwd
    check(fn(_p(X), X.shape[0], _p(obs_point), _p(obs_xy), _p(view_obs_offset),
             ctypes.byref(cc), ctypes.byref(bc), float(delta), float(weight), _p(loss),
             _p(grad_X), _p(g_pose_tangent), _p(n_masked), _p(ws), ws.numel(),
             _stream(stream)), "track_reproj_fwd_bwd")


def track_reproj_fwd_bwd_static(X, obs_point, obs_xy, view_obs_offset, cams: Cameras, batch: Batch,
                                delta: float, weight: float, loss, grad_X, g_pose_tangent, n_masked, Rt=None,
                                stream=None):
    """The track term with the library's own fixed scratch instead of a
    caller workspace (for callers that cannot allocate device memory)."""
    lib = _lib.load()
    _need_cuda(X, obs_point, obs_xy, view_obs_offset, loss, grad_X, g_pose_tangent, n_masked)
    cc, bc = cams.c(Rt), batch.c()
    check(lib.track_reproj_fwd_bwd_static(_p(X), X.shape[0], _p(obs_point), _p(obs_xy), _p(view_obs_offset),
                                          ctypes.byref(cc), ctypes.byref(bc), float(delta), float(weight),
                                          _p(loss), _p(grad_X), _p(g_pose_tangent), _p(n_masked),
                                          _stream(stream)), "track_reproj_fwd_bwd_static")


def adam_c(lr, beta1, beta2, eps, step: torch.Tensor):
    return _lib.gs_adam(float(lr), float(beta1), float(beta2), float(eps), step.data_ptr())


def pose_se3_update(T0, xi, g_tangent, g_xi, m, v, hp, Rt_out, stream=None):
    """hp: gs_adam struct or None (gradient map and recomposition only).
    float64 T0, xi, ... run the FP64 instantiation."""
    lib = _lib.load()
    _need_cuda(T0, xi, g_tangent, g_xi, m, v, Rt_out)
    f64 = T0.dtype == torch.float64
    check(_fn(lib, "pose_se3_update", f64)(T0.shape[0], _p(T0), _p(xi), _p(g_tangent), _p(g_xi), _p(m), _p(v),
                                           None if hp is None else ctypes.byref(hp), _p(Rt_out), _stream(stream)),
          "pose_se3_update")


def gs_adam_update(p, g, m, v, hp, stream=None):
    lib = _lib.load()
    _need_cuda(p, g, m, v)
    check(lib.gs_adam_update(_p(p), _p(g), _p(m), _p(v), p.numel(), ctypes.byref(hp), _stream(stream)),
          "gs_adam_update")


def gs_adam_update_groups(groups, beta1, beta2, eps, step, stream=None):
    """groups: list of (p, g, m, v, lr), at most 8; one launch."""
    lib = _lib.load()
    arr = (_lib.gs_adam_group * len(groups))()
    for i, (p, g, m, v, lr) in enumerate(groups):
        _need_cuda(p, g, m, v)
        arr[i] = _lib.gs_adam_group(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(), float(lr), 0)
    hp = adam_c(0.0, beta1, beta2, eps, step)
    check(lib.gs_adam_update_groups(arr, len(groups), ctypes.byref(hp), _stream(stream)), "gs_adam_update_groups")


def gs_set_tuning(render_fwd_batch: int = 128, render_bwd_batch: int = 64, sort_blocks_per_sm: int = 1,
                  sort_spin_limit: int = 0):
    lib = _lib.load()
    t = _lib.gs_tuning(int(render_fwd_batch), int(render_bwd_batch), int(sort_blocks_per_sm), int(sort_spin_limit))
    check(lib.gs_set_tuning(ctypes.byref(t)), "gs_set_tuning")


def gs_get_tuning():
    lib = _lib.load()
    t = _lib.gs_tuning()
    check(lib.gs_get_tuning(ctypes.byref(t)), "gs_get_tuning")
    return dict(render_fwd_batch=t.render_fwd_batch, render_bwd_batch=t.render_bwd_batch,
                sort_blocks_per_sm=t.sort_blocks_per_sm, sort_spin_limit=t.sort_spin_limit)


def gs_step_advance(step, stream=None):
    lib = _lib.load()
    _need_cuda(step)
    check(lib.gs_step_advance(_p(step), _stream(stream)), "gs_step_advance")


def gs_gather_view_pixels(src: torch.Tensor, src_px_offset: torch.Tensor, cams: Cameras, batch: Batch,
                          dst: torch.Tensor, stream=None):
    lib = _lib.load()
    _need_cuda(src, src_px_offset, dst)
    cc, bc = cams.c(), batch.c()
    ch = src.shape[1] if src.dim() > 1 else 1
    check(lib.gs_gather_view_pixels(_p(src), _p(src_px_offset), ctypes.byref(cc), ctypes.byref(bc), int(ch), _p(dst),
                                    _stream(stream)), "gs_gather_view_pixels")


def gs_zero(t: torch.Tensor, stream=None):
    lib = _lib.load()
    _need_cuda(t)
    check(lib.gs_zero(_p(t), t.numel() * t.element_size(), _stream(stream)), "gs_zero")
