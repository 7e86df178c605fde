"""Joint pose-appearance training step (Algorithm 1, one iteration) driven
through the C ABI: the batched form (every stage one launch over all views
of the batch, capturable in a CUDA graph) and the plain form (one view per
launch, for comparison)."""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from .core import (Batch, Cameras, Gaussians, Projected, TileLists, adam_c, gs_adam_update, gs_adam_update_groups,
                   gs_gather_view_pixels, gs_photo_loss, gs_project, photo_loss_workspace_bytes,
                   gs_project_bwd, gs_raster_bwd, gs_raster_bwd_det, gs_render_fwd, gs_sort_tiles,
                   gs_step_advance, gs_zero, new_status, pose_se3_update, render_bwd_det_workspace_bytes,
                   render_bwd_workspace_bytes, track_reproj_fwd_bwd,
                   track_workspace_bytes)


def _nomark(name):
    pass


class Renderer:
    """Buffers and launches for rendering one batch of views: projection,
    tile sort, compositing, and the backward.  Launches never read anything
    back; `ensure_capacity` is the only host synchronisation and grows the
    instance buffers when the sort reported an overflow."""

    def __init__(self, n: int, cams: Cameras, batch: Batch, capacity: int = 0, bg=(0.0, 0.0, 0.0),
                 device="cuda", dtype=torch.float32, deterministic: bool = False):
        # dtype float64: the FP64 instantiation of projection and compositing
        # (the Gaussians passed to forward/backward must be float64 too).
        # deterministic: the backward whose gradients and loss do not depend
        # on the order in which tiles run (gs_raster_bwd_det; FP32 only)
        if deterministic and dtype != torch.float32:
            raise ValueError("the deterministic backward is FP32 only")
        self.n, self.cams, self.batch, self.dtype = n, cams, batch, dtype
        self.deterministic = deterministic
        self.proj = Projected(n, batch.B, device, dtype)
        cap = capacity if capacity > 0 else max(1 << 16, 4 * n * batch.B)
        self.tl = TileLists(n, batch, cap, device)
        P = max(batch.n_pixels, 1)
        self.image = torch.zeros((P, 3), dtype=dtype, device=device)
        self.T_final = torch.zeros(P, dtype=dtype, device=device)
        self.n_contrib = torch.zeros(P, dtype=torch.int32, device=device)
        self.bg = torch.tensor(bg, dtype=dtype, device=device)
        self.ws_bwd = torch.empty(max(self._bwd_bytes(), 256), dtype=torch.uint8, device=device)
        self.status = new_status(device)
        self.zero_records()   # so that a first backward may already pass records_zeroed

    def _bwd_bytes(self) -> int:
        if self.deterministic:
            return render_bwd_det_workspace_bytes(self.n, self.batch, self.tl.capacity)
        return render_bwd_workspace_bytes(self.n, self.batch, self.dtype == torch.float64)

    def _layout(self):
        # a batch laid out on the device: its offsets follow the device copy
        # of its view ids, which may have changed since the last launch
        if self.batch.dynamic:
            self.batch.layout(self.cams, self.status)

    def forward(self, g: Gaussians, Rt: torch.Tensor = None, mark=_nomark, after_sort=None, layout=True):
        """Projection, tile sort, compositing; `after_sort()` (if given) is
        called between the sort and the compositing.  layout=False: the
        caller has already laid out a device-laid-out batch on this stream."""
        if layout:
            self._layout()
        gs_project(g, self.cams, self.batch, self.proj, self.status, Rt)
        mark("project")
        gs_sort_tiles(self.n, self.cams, self.batch, self.proj, self.tl, self.status, Rt)
        mark("sort")
        if after_sort is not None:
            after_sort()
        gs_render_fwd(self.batch, self.cams, self.proj, self.tl, self.bg, self.image, self.T_final,
                      self.n_contrib, Rt)
        mark("render_fwd")

    def zero_records(self):
        """Zeroes the screen-space records of the (atomic) backward on the
        current stream, so that a later backward(records_zeroed=True) skips
        it; nothing to do for the deterministic backward, which writes every
        record."""
        if not self.deterministic and self.dtype == torch.float32:
            gs_zero(self.ws_bwd[:self.batch.B * self.n * 48])

    def backward(self, g: Gaussians, dg: Gaussians, g_tangent: torch.Tensor, v_image=None, target=None,
                 l1_weight: float = 1.0, loss=None, Rt: torch.Tensor = None, mark=_nomark,
                 records_zeroed: bool = False, clear_records: bool = False):
        # gs_render_bwd is exactly these two calls; issuing them separately
        # lets a caller time each half.  records_zeroed: the records are
        # zero (zero_records() was issued before, on any stream ordered
        # before this one, or the last backward cleared them).
        # clear_records: the projection backward zeroes each record after
        # reading it, so that the next backward can pass records_zeroed
        if self.deterministic:
            gs_raster_bwd_det(g, self.cams, self.batch, self.proj, self.tl, self.bg, self.image, self.T_final,
                              self.n_contrib, v_image, target, l1_weight, loss, self.ws_bwd, Rt)
        else:
            gs_raster_bwd(g, self.cams, self.batch, self.proj, self.tl, self.bg, self.image, self.T_final,
                          self.n_contrib, v_image, target, l1_weight, loss, self.ws_bwd, Rt,
                          records_zeroed=records_zeroed and self.dtype == torch.float32)
        mark("raster_bwd")
        gs_project_bwd(g, self.cams, self.batch, self.proj, dg, g_tangent, self.ws_bwd, Rt,
                       clear_records=clear_records and self.atomic_records)
        mark("project_bwd")

    @property
    def atomic_records(self) -> bool:
        """The backward accumulates into screen-space records that must be
        zero before it (FP32, not the deterministic form)."""
        return not self.deterministic and self.dtype == torch.float32

    def count_added(self, g: Gaussians, Rt: torch.Tensor = None) -> int:
        """Re-runs the forward with the per-pixel added-splat counter and
        returns the total number of splats composited (a diagnostic)."""
        n_added = torch.zeros_like(self.n_contrib)
        self._layout()
        gs_project(g, self.cams, self.batch, self.proj, self.status, Rt)
        gs_sort_tiles(self.n, self.cams, self.batch, self.proj, self.tl, self.status, Rt)
        gs_render_fwd(self.batch, self.cams, self.proj, self.tl, self.bg, self.image, self.T_final,
                      self.n_contrib, Rt, n_added=n_added)
        return int(n_added.to(torch.int64).sum().item())

    def n_instances(self) -> int:
        return int(self.tl.n_instances.item()) & 0xffffffff

    def ensure_capacity(self, g: Gaussians, Rt: torch.Tensor = None, headroom: float = 1.25) -> bool:
        """Runs projection + sort once, reads the instance count and grows
        the buffers if needed.  Returns True when they were resized."""
        self.status.zero_()
        self._layout()
        gs_project(g, self.cams, self.batch, self.proj, self.status, Rt)
        gs_sort_tiles(self.n, self.cams, self.batch, self.proj, self.tl, self.status, Rt)
        need = self.n_instances()
        if need > self.tl.capacity:
            self.tl = TileLists(self.n, self.batch, int(need * headroom) + 1024, self.image.device)
            if self.deterministic:   # its slots grow with the capacity
                self.ws_bwd = torch.empty(self._bwd_bytes(), dtype=torch.uint8, device=self.image.device)
            self.status.zero_()
            return True
        self.status.zero_()
        return False


@dataclass
class Hyper:
    """Learning rates of Sec. 3.3 ("Implementation"; camera extrinsics: Adam
    with lr 1e-5).  The paper gives no rate for the track points; they use
    the position rate."""
    lr_mean: float = 1.6e-4
    lr_log_scale: float = 5e-3
    lr_quat: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh: float = 2.5e-3
    lr_track: float = 1.6e-4
    lr_pose: float = 1e-5
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    scene_extent: float = 1.0
    lambda_ba: float = 1e-4       # Sec. 3.3 total objective
    huber_delta: float = 1.0      # Eq. 6
    l1_weight: float = 1.0        # weight of the photometric term, Eq. 5
    # lambda_SSIM of Eq. 5 (the paper trains with 0.2).  0 keeps the L1 part
    # alone, fused into the compositing backward; > 0 runs gs_photo_loss
    # (L1 weighted 1 - lambda, SSIM lambda) and feeds its dL/dimage to the
    # backward.  Read when the batch is set.
    lambda_ssim: float = 0.0
    # Variants of the paper's extended ablation study: freeze_poses keeps
    # T = T0 (no pose update); lambda_ba = 0 is the photometric-only variant
    # (the track term is not run at all).
    freeze_poses: bool = False


class JointStep:
    """State and launches of the joint training step.

    Parameters: Gaussians G, track points X, per-camera pose deltas xi with
    T = Exp(xi) T0 (Algorithm 1).  One call of `step()` performs, for the
    current batch: projection, tile sort, compositing, fused L1 + backward
    with pose gradient, the track term, and the Adam updates of G, X and xi
    (which also recomposes the poses used by the next step).  Nothing is
    read back to the host.  `mode="plain"` issues every stage once per view
    (B = 1 launches); `mode="batched"` issues each stage once for the batch.
    """

    def __init__(self, gaussians: Gaussians, cams: Cameras, X: torch.Tensor, obs_point: torch.Tensor,
                 obs_xy: torch.Tensor, view_obs_offset: torch.Tensor, targets: torch.Tensor,
                 target_px_offset: np.ndarray, views, hyper: Hyper = None, mode: str = "batched",
                 capacity: int = 0, device="cuda", tile: int = 16, merged_tracks: bool = False,
                 dynamic_batch: bool = False, deterministic: bool = False):
        # merged_tracks: the "merged tracks" ablation variant, X_k = mu of a
        # Gaussian (obs_point then indexes Gaussians; X is ignored): the track
        # term reads the Gaussian means and adds its gradient into theirs.
        # dynamic_batch: the batch's buffers are sized for any views of the
        # scene and its layout is recomputed on the device at the start of
        # every step, so next_batch() takes views of any sizes without
        # dropping a captured graph (batches of uneven views).
        # deterministic: the step whose results do not depend on the order
        # in which threads run (gs_raster_bwd_det, track_reproj_fwd_bwd_det):
        # two runs from the same state give bit-identical parameters.
        self.dynamic_batch = bool(dynamic_batch)
        self.deterministic = bool(deterministic)
        self.h = hyper or Hyper()
        self.merged_tracks = bool(merged_tracks)
        self.tile = int(tile)
        self.mode = mode
        self.g = gaussians
        self.dg = Gaussians.zeros_like(gaussians)
        self.m = Gaussians.zeros_like(gaussians)
        self.v = Gaussians.zeros_like(gaussians)
        self.cams = cams
        self.T0 = cams.Rt.clone()
        self.Rt = cams.Rt.clone()
        V = cams.V
        self.xi = torch.zeros((V, 6), dtype=torch.float32, device=device)
        self.g_xi = torch.zeros_like(self.xi)
        self.m_xi = torch.zeros_like(self.xi)
        self.v_xi = torch.zeros_like(self.xi)
        self.g_tan = torch.zeros((V, 6), dtype=torch.float64, device=device)
        if self.merged_tracks:
            X = self.g.mean
        self.X = X
        self.gX = self.dg.mean if self.merged_tracks else torch.zeros_like(X)
        self.mX = torch.zeros_like(X)
        self.vX = torch.zeros_like(X)
        self.obs_point, self.obs_xy, self.view_obs_offset = obs_point, obs_xy, view_obs_offset
        self.targets = targets                  # all views, packed by target_px_offset
        self.target_px_offset = np.asarray(target_px_offset, dtype=np.int64)
        self.target_px_offset_dev = torch.as_tensor(self.target_px_offset, device=device)
        self.loss = torch.zeros(2, dtype=torch.float64, device=device)   # [L_photo, sum rho]
        self.n_masked = torch.zeros(1, dtype=torch.int32, device=device)
        self.step_no = torch.zeros(1, dtype=torch.int32, device=device)
        self.device = device
        self._capacity = capacity
        self.graph = None
        self.set_batch(views)

    # -- batch management --------------------------------------------------
    def _new_batch(self, views):
        cap = Batch.capacity_for(self.cams, len(views), self.tile) if self.dynamic_batch else None
        return Batch(self.cams, views, tile=self.tile, device=self.device, capacity=cap)

    def set_batch(self, views):
        views = np.asarray(views, dtype=np.int64)
        self.views = views
        self.batch = self._new_batch(views)
        n = self.g.n
        if self.mode == "batched":
            self.renderers = [Renderer(n, self.cams, self.batch, self._capacity, device=self.device,
                                       deterministic=self.deterministic)]
            self.slot_batches = [self.batch]
        else:
            self.slot_batches = [self._new_batch([v]) for v in views]
            cap = self._capacity // max(len(views), 1)
            self.renderers = [Renderer(n, self.cams, b, cap, device=self.device, deterministic=self.deterministic)
                              for b in self.slot_batches]
        self.track_ws = torch.empty(max(track_workspace_bytes(self.batch), 256), dtype=torch.uint8,
                                    device=self.device)
        self.ssim_on = self.h.lambda_ssim > 0.0
        for r in self.renderers:
            r.v_image = r.ws_photo = None
            if self.ssim_on:
                r.v_image = torch.empty((max(r.batch.n_pixels, 1), 3), dtype=torch.float32, device=self.device)
                r.ws_photo = torch.empty(max(photo_loss_workspace_bytes(r.batch), 256), dtype=torch.uint8,
                                         device=self.device)
        # the batch's target images in its pixel layout; the plain form
        # gathers one view per launch, into one buffer per slot
        for r in self.renderers:
            r.target = torch.empty((max(r.batch.n_pixels, 1), 3), dtype=torch.float32, device=self.device)
        self.target_batch = self.renderers[0].target if self.mode == "batched" else None
        self.load_targets()
        self.graph = None

    def _gather_targets(self):
        for r in self.renderers:
            gs_gather_view_pixels(self.targets, self.target_px_offset_dev, self.cams, r.batch, r.target)

    def load_targets(self):
        """Gathers the batch's target images into slot order on the device
        (the step does this itself; this is for use outside a step)."""
        for r in self.renderers:
            r._layout()
        self._gather_targets()

    def set_tile(self, tile: int):
        """Switches the tile size (16 or 32 pixels): re-allocates the batch's
        buffers (instance capacity kept) and drops the captured graph."""
        if int(tile) == self.tile:
            return
        self.tile = int(tile)
        caps = [r.tl.capacity for r in self.renderers]
        self.set_batch(self.views)
        for r, cap in zip(self.renderers, caps):
            if r.tl.capacity < cap:
                r.tl = TileLists(r.n, r.batch, cap, r.image.device)

    def next_batch(self, views):
        """Switches to another batch of views.  Views of the same per-slot
        sizes are swapped in place on the device, so a captured graph stays
        valid; other sizes re-allocate (and drop the graph)."""
        vs = np.asarray(views, dtype=np.int64).reshape(-1)
        if self.batch.same_layout(self.cams, vs) and (
                self.mode == "batched" or all(b.same_layout(self.cams, [v]) for b, v in zip(self.slot_batches, vs))):
            self.batch.set_views(self.cams, vs)
            if self.mode != "batched":
                for b, v in zip(self.slot_batches, vs):
                    b.set_views(self.cams, [v])
            self.views = vs
        else:
            self.set_batch(views)

    def ensure_capacity(self):
        grew = False
        for r in self.renderers:
            grew |= r.ensure_capacity(self.g, self.Rt)
        if grew:
            self.graph = None
        return grew

    def _side_stream(self) -> torch.cuda.Stream:
        # high priority: its few short kernels get SM slots as soon as the
        # compositing grid frees any, instead of queueing behind all of it
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(device=self.device, priority=-1)
        return self._side

    # -- the step ----------------------------------------------------------
    def _adam(self, p, g, m, v, lr):
        gs_adam_update(p, g, m, v, adam_c(lr, self.h.beta1, self.h.beta2, self.h.eps, self.step_no))

    def step(self, mark=_nomark):
        """One training iteration; `mark(name)` is called after each stage
        (for event timing).  The gradient zeroing, the target gather and the
        track term run on a side stream, forked after the first view's sort
        so that they overlap the compute-bound compositing rather than the
        memory-bound projection, and joined before the first backward."""
        h = self.h
        main = torch.cuda.current_stream()
        side = self._side_stream()

        def fork():
            side.wait_stream(main)
            with torch.cuda.stream(side):
                extra = [] if self.merged_tracks else [self.gX]   # merged: gX is dg.mean
                for t in self.dg.tensors() + extra + [self.g_tan, self.loss, self.n_masked]:
                    gs_zero(t)
                # the backward's screen-space records need no clearing: the
                # last step's projection backward zeroed each after reading
                # it (clear_records), the renderer's construction before that
                self._gather_targets()
                # the track term: done before the join, so its += into the
                # pose tangent (and, merged, into dg.mean) precedes the
                # projection backward's; not run at all when lambda_BA = 0
                if h.lambda_ba != 0.0:
                    track_reproj_fwd_bwd(self.X, self.obs_point, self.obs_xy, self.view_obs_offset, self.cams,
                                         self.batch, h.huber_delta, h.lambda_ba, self.loss[1:2], self.gX,
                                         self.g_tan, self.n_masked, self.track_ws, self.Rt,
                                         deterministic=self.deterministic)

        # every slot's offsets first: the side stream gathers all slots'
        # targets once the first slot is sorted
        for r in self.renderers:
            r._layout()
        joined = False
        for b, r in enumerate(self.renderers):
            r.forward(self.g, self.Rt, mark, after_sort=fork if b == 0 else None, layout=False)
            if not joined:
                main.wait_stream(side)
                joined = True
            tgt = r.target
            if self.ssim_on:
                lam = h.lambda_ssim
                gs_photo_loss(self.cams, r.batch, r.image, tgt, h.l1_weight * (1.0 - lam), h.l1_weight * lam,
                              self.loss[0:1], r.v_image, r.ws_photo, self.Rt)
                mark("photo")
                r.backward(self.g, self.dg, self.g_tan, v_image=r.v_image, loss=self.loss[0:1], Rt=self.Rt,
                           mark=mark, records_zeroed=True, clear_records=True)
            else:
                r.backward(self.g, self.dg, self.g_tan, target=tgt, l1_weight=h.l1_weight, loss=self.loss[0:1],
                           Rt=self.Rt, mark=mark, records_zeroed=True, clear_records=True)
        if not joined:
            fork()
            main.wait_stream(side)
        mark("zero")
        mark("track")
        gs_step_advance(self.step_no)
        # the pose update (one small kernel, independent of the parameter
        # update) runs on the side stream beside Adam
        side.wait_stream(main)
        if not h.freeze_poses:
            with torch.cuda.stream(side):
                hp = adam_c(h.lr_pose, h.beta1, h.beta2, h.eps, self.step_no)
                pose_se3_update(self.T0, self.xi, self.g_tan, self.g_xi, self.m_xi, self.v_xi, hp, self.Rt)
        ext = h.scene_extent
        groups = [
            (self.g.mean, self.dg.mean, self.m.mean, self.v.mean, h.lr_mean * ext),
            (self.g.log_scale, self.dg.log_scale, self.m.log_scale, self.v.log_scale, h.lr_log_scale),
            (self.g.quat, self.dg.quat, self.m.quat, self.v.quat, h.lr_quat),
            (self.g.opacity_logit, self.dg.opacity_logit, self.m.opacity_logit, self.v.opacity_logit,
             h.lr_opacity),
            (self.g.sh, self.dg.sh, self.m.sh, self.v.sh, h.lr_sh)]
        if not self.merged_tracks:   # merged, the means' group updates the track points
            groups.append((self.X, self.gX, self.mX, self.vX, h.lr_track * ext))
        gs_adam_update_groups(groups, h.beta1, h.beta2, h.eps, self.step_no)
        mark("adam")
        main.wait_stream(side)
        mark("pose")

    def kernels_per_step(self) -> int:
        """libgs kernel launches one step issues (memsets not counted)."""
        per_render = 0
        for b in self.slot_batches:
            tbits = int(math.ceil(math.log2(b.n_tiles))) if b.n_tiles > 1 else 0
            tile_passes = min((tbits + 7) // 8, (tbits + 8) // 9)   # 8- or 9-bit digits
            # project 1; sort: zero 1, depth range 1, depth histogram 1,
            # depth passes 4, scan 2, expand 1, one per tile pass, ranges 1;
            # render fwd 1; raster bwd 1; project bwd + finalize 2
            per_render += 1 + (1 + 1 + 1 + 4 + 2 + 1 + tile_passes + 1) + 1 + 1 + 2
            if self.deterministic:
                # slot bases (3-kernel scan), the fixed-order record sums,
                # and the tiles' loss sum with the fused L1
                per_render += 3 + 1 + (0 if self.ssim_on else 1)
            if self.ssim_on:
                per_render += 3  # photometric loss: block list, forward, backward
        # target gather 1 per renderer, layout 1 per renderer (dynamic
        # batches), track + finalize 2 (unless lambda_BA = 0), step advance
        # 1, Adam (all groups) 1, pose 1 (unless frozen)
        nr = len(self.renderers)
        track = (3 * self.batch.B if self.deterministic else 2) if self.h.lambda_ba != 0.0 else 0
        return (per_render + nr + (nr if self.dynamic_batch else 0) + track + 1 +
                1 + (0 if self.h.freeze_poses else 1))

    # -- CUDA graph ----------------------------------------------------------
    def capture(self, warmup: int = 1):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        torch.cuda.synchronize()

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.step()

    def status_flags(self) -> int:
        f = 0
        for r in self.renderers:
            f |= int(r.status.item())
        return f


class TargetStream:
    """Feeds a JointStep its target images from pinned host memory, one
    step ahead, on a copy stream (Algorithm 1, "Sample a batch of views",
    with the dataset kept on the host).

    Two device copies of the dataset layout alternate: while step i runs and
    its gather reads copy i % 2, the views of step i + 1 are uploaded into
    the other copy.  A step waits for its own upload; an upload waits for
    the step that last read its copy.  Attach before capturing the step's
    graph (the gather's source pointers change).

        ts = TargetStream(js, host_targets, px_offset)
        ts.put(views_0)
        for i in range(n):
            ts.begin()            # current stream waits for this step's upload
            js.run()
            ts.end()
            ts.put(views_next)    # overlaps the step just enqueued
    """

    def __init__(self, js: JointStep, host_targets: torch.Tensor, px_offset):
        if not host_targets.is_pinned():
            raise ValueError("TargetStream: host_targets must be in pinned memory")
        dev = js.targets.device
        self.js = js
        self.host = host_targets
        self.off = np.asarray(px_offset, dtype=np.int64)
        self.P = int(self.off[-1])
        self.buf = torch.zeros((2 * max(self.P, 1), 3), dtype=torch.float32, device=dev)
        self.off_host = [torch.as_tensor(self.off + h * self.P).pin_memory() for h in (0, 1)]
        self.off_dev = torch.as_tensor(self.off, device=dev).clone()
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.uploaded = [torch.cuda.Event(), torch.cuda.Event()]
        self.released = [torch.cuda.Event(), torch.cuda.Event()]
        self.next_half = 0   # copy the next put() fills
        self.cur_half = 0    # copy the next begin() uses
        self.last_bytes = 0
        js.targets = self.buf
        js.target_px_offset_dev = self.off_dev
        js.graph = None

    def put(self, views) -> int:
        """Enqueues the upload of these views' targets; returns its bytes."""
        h = self.next_half
        cs = self.copy_stream
        cs.wait_event(self.released[h])
        n = 0
        with torch.cuda.stream(cs):
            base = h * self.P
            for v in np.asarray(views).reshape(-1):
                a, e = int(self.off[v]), int(self.off[v + 1])
                self.buf[base + a:base + e].copy_(self.host[a:e], non_blocking=True)
                n += (e - a) * 12
        self.uploaded[h].record(cs)
        self.next_half = 1 - h
        self.last_bytes = n
        return n

    def begin(self):
        """On the current stream: wait for this step's upload and point the
        gather at its copy (8 (V+1) bytes copied)."""
        h = self.cur_half
        st = torch.cuda.current_stream()
        st.wait_event(self.uploaded[h])
        self.off_dev.copy_(self.off_host[h], non_blocking=True)

    def end(self):
        """On the current stream, after the step: its copy may be refilled."""
        h = self.cur_half
        self.released[h].record(torch.cuda.current_stream())
        self.cur_half = 1 - h
