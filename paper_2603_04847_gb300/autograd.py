"""torch.autograd.Function wrappers of the libgs kernels.

`render(params, cams, T0, xi, views)` returns the batch's packed image as a
differentiable function of the raw Gaussian parameters and of the per-camera
pose deltas xi (T = Exp(xi) T0, Algorithm 1); `track_loss(X, xi, ...)`
returns lambda_BA * L_BA (Eq. 6) as a function of the track points and xi.
Both run every step on the CUDA kernels; the backward of `render`
recomputes compositing from the forward's per-pixel state (T_final and
n_contrib) instead of storing it.

`render` takes float32 or float64 parameters: float32 runs the FP32
kernels; float64 runs their FP64 instantiation end to end (projection,
compositing, their backward and the pose composition in double), so that
torch.autograd.gradcheck compares double-precision finite differences with
double-precision analytic gradients at its default tolerances.  The track
term computes in FP32 and returns its outputs in the inputs' dtype.  A
`RenderState` holds the buffers of one outstanding forward: run its
backward before the next forward on it.
"""
from __future__ import annotations

import torch

from .core import Batch, Cameras, Gaussians, pose_se3_update, track_reproj_fwd_bwd, track_workspace_bytes
from .step import Renderer


class RenderState:
    """Reusable buffers for `render` on a fixed set of cameras and views.
    fixed_capacity=True sizes the tile-instance buffers at the first forward
    only (no host synchronisation afterwards) -- for many evaluations of one
    scene, e.g. finite differences; it is the caller's promise that the
    instance count does not grow (the sort flags it if it does)."""

    def __init__(self, cams: Cameras, views, bg=(0.0, 0.0, 0.0), fixed_capacity: bool = False):
        self.cams = cams
        self.batch = Batch(cams, views, device=cams.K.device)
        self.bg = bg
        self.renderer = None
        self.fixed_capacity = fixed_capacity
        self.sized = False

    def get(self, n: int, dtype=torch.float32) -> Renderer:
        if self.renderer is None or self.renderer.n != n or self.renderer.dtype != dtype:
            self.renderer = Renderer(n, self.cams, self.batch, bg=self.bg, device=self.cams.K.device, dtype=dtype)
            self.sized = False
        return self.renderer


def _f32(t):
    return t.detach().to(torch.float32).contiguous()


def _as(t, dtype):
    return t.detach().to(dtype).contiguous()


def _compose(T0, xi):
    """Rt = Exp(xi) T0 on the device (pose_se3_update without an Adam step),
    in the dtype of T0 and xi."""
    Rt = torch.empty_like(T0)
    zeros = torch.zeros(xi.shape, dtype=torch.float64, device=xi.device)
    pose_se3_update(T0, xi, zeros, None, None, None, None, Rt)
    return Rt


def _map_tangent(T0, xi, g_tan):
    """dL/dxi = Jl(xi)^T g_tangent."""
    g_xi = torch.zeros_like(xi)
    Rt = torch.empty_like(T0)
    pose_se3_update(T0, xi, g_tan, g_xi, None, None, None, Rt)
    return g_xi


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mean, log_scale, quat, opacity_logit, sh, xi, T0, state):
        dt = mean.dtype
        kt = torch.float64 if dt == torch.float64 else torch.float32   # the kernels' precision
        g = Gaussians(_as(mean, kt), _as(log_scale, kt), _as(quat, kt), _as(opacity_logit, kt), _as(sh, kt))
        T0 = _as(T0, kt)
        xik = _as(xi, kt)
        Rt = _compose(T0, xik)
        r = state.get(g.n, kt)
        if not (state.sized and state.fixed_capacity):
            r.ensure_capacity(g, Rt)
            state.sized = True
        r.forward(g, Rt)
        ctx.state = state
        ctx.g, ctx.Rt, ctx.T0, ctx.xik, ctx.dt = g, Rt, T0, xik, dt
        return r.image.to(dt).clone()

    @staticmethod
    def backward(ctx, grad_image):
        r = ctx.state.renderer
        g = ctx.g
        dg = Gaussians.zeros_like(g)
        g_tan = torch.zeros((ctx.xik.shape[0], 6), dtype=torch.float64, device=grad_image.device)
        r.backward(g, dg, g_tan, v_image=_as(grad_image, r.dtype), Rt=ctx.Rt)
        g_xi = _map_tangent(ctx.T0, ctx.xik, g_tan)
        dt = ctx.dt
        return (dg.mean.to(dt), dg.log_scale.to(dt), dg.quat.to(dt), dg.opacity_logit.to(dt), dg.sh.to(dt),
                g_xi.to(dt), None, None)


def render(mean, log_scale, quat, opacity_logit, sh, xi, T0, state: RenderState):
    """Packed image [n_pixels, 3] of the views of `state`, differentiable in
    the raw Gaussian parameters and the pose deltas xi [V,6]."""
    return _Render.apply(mean, log_scale, quat, opacity_logit, sh, xi, T0, state)


class _TrackLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, xi, T0, obs_point, obs_xy, view_obs_offset, cams, batch, delta, weight):
        dt = X.dtype
        X32, xi32, T0 = _f32(X), _f32(xi), _f32(T0)
        Rt = _compose(T0, xi32)
        loss = torch.zeros(1, dtype=torch.float64, device=X.device)
        gX = torch.zeros_like(X32)
        g_tan = torch.zeros((xi32.shape[0], 6), dtype=torch.float64, device=X.device)
        nm = torch.zeros(1, dtype=torch.int32, device=X.device)
        ws = torch.empty(track_workspace_bytes(batch), dtype=torch.uint8, device=X.device)
        track_reproj_fwd_bwd(X32, obs_point, obs_xy, view_obs_offset, cams, batch, delta, weight, loss, gX, g_tan,
                             nm, ws, Rt)
        ctx.saved = (gX, _map_tangent(T0, xi32, g_tan), dt)
        return (loss * weight).to(dt).reshape(())

    @staticmethod
    def backward(ctx, grad):
        gX, g_xi, dt = ctx.saved
        return (gX.to(dt) * grad, g_xi.to(dt) * grad, None, None, None, None, None, None, None, None)


def track_loss(X, xi, T0, obs_point, obs_xy, view_obs_offset, cams: Cameras, batch: Batch, delta=1.0,
               weight=1e-4):
    """weight * sum over the batch's observations of the Huber reprojection
    loss (Eq. 6), differentiable in the track points X and the pose deltas."""
    return _TrackLoss.apply(X, xi, T0, obs_point, obs_xy, view_obs_offset, cams, batch, delta, weight)
