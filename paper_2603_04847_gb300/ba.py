"""Levenberg-Marquardt bundle adjustment of Eq. 4 (Sec. 3.2, "Bundle
Adjustment") on the GPU.

Each iteration runs in libgs kernels: the IRLS normal-equation blocks
(sfm_ba_assemble), the elimination of the points (sfm_ba_schur_pairs, or
sfm_ba_schur with pairs=False), the
reduced camera system with camera 0 fixed (sfm_ba_solve_cameras), the
points' back-substitution, the trial parameters (sfm_ba_apply_step) and
their objective (sfm_ba_objective).  The host reads the two objectives to
accept or reject the step: Marquardt damping, lambda / 10 after an accepted
step and x 10 after a rejected one.  Poses and points are stored as float32
(the residuals then resolve ~1e-5 px at the synthetic workloads' scale);
the blocks and the solve are double precision."""
from __future__ import annotations

import numpy as np
import torch

from .core import (PAIR_CHUNK, Cameras, gs_zero, sfm_ba_apply_step, sfm_ba_assemble, sfm_ba_back_substitute,
                   sfm_ba_lm_accept, sfm_ba_objective, sfm_ba_pair_lists, sfm_ba_schur, sfm_ba_schur_pairs,
                   sfm_ba_schur_pairs_workspace, sfm_ba_solve_cameras)


class BundleAdjuster:
    """State of one bundle adjustment: cams (intrinsics and initial poses),
    X [P,3] float32 device points, and host arrays of the observations
    (obs_point, obs_cam [M] int, obs_xy [M,2] pixels)."""

    def __init__(self, cams: Cameras, X: torch.Tensor, obs_point, obs_cam, obs_xy, delta: float = 1.0,
                 lam: float = 1e-4, pairs: bool = True, pair_chunk: int = PAIR_CHUNK):
        dev = X.device
        self.cams, self.delta, self.lam = cams, float(delta), float(lam)
        self.Rt = cams.Rt.clone()
        self.X = X.clone()
        self.Rt_trial = torch.empty_like(self.Rt)
        self.X_trial = torch.empty_like(self.X)
        op = np.asarray(obs_point, np.int32)
        oc = np.asarray(obs_cam, np.int32)
        xy = np.asarray(obs_xy, np.float32).reshape(-1, 2)
        # observations in camera order (stable; the benchmark's already
        # are): the blocks' warps then share a camera and add its sums once
        # (sfm_ba_assemble); the results do not depend on the order beyond
        # the FP64 summation order
        perm = np.argsort(oc, kind="stable")
        op, oc, xy = op[perm], oc[perm], xy[perm]
        V, P, M = cams.V, self.X.shape[0], op.shape[0]
        # each point's observations as a CSR list (setup, from the host arrays)
        ok = (op >= 0) & (op < P)
        ids = np.nonzero(ok)[0]
        ids = ids[np.argsort(op[ids], kind="stable")]
        off = np.concatenate([[0], np.cumsum(np.bincount(op[ok], minlength=P))])

        def t(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

        self.obs_point, self.obs_cam = t(op, torch.int32), t(oc, torch.int32)
        self.obs_xy = t(xy, torch.float32)
        self.off, self.ids = t(off, torch.int64), t(ids, torch.int32)
        # the elimination by camera pairs: its plan is built once (the
        # observation structure does not change between iterations)
        self.plan = None
        if pairs:
            hplan = sfm_ba_pair_lists(V, P, oc, off, ids, chunk=pair_chunk)
            self.plan = {k: t(a, torch.int64 if a.dtype == np.int64 else torch.int32) for k, a in hplan.items()}
            nb = sfm_ba_schur_pairs_workspace(M, hplan["chunk_start"].shape[0] - 1)
            self.pair_ws = torch.empty(max(nb, 8), dtype=torch.uint8, device=dev)

        def z(*s):
            return torch.zeros(s, dtype=torch.float64, device=dev)

        self.U, self.Vp, self.gc, self.gp = z(V, 36), z(P, 9), z(V, 6), z(P, 3)
        self.Wo = z(max(M, 1), 18)
        self.S, self.rhs, self.Vinv = z(6 * V, 6 * V), z(6 * V), z(P, 9)
        self.dc, self.dp = z(V, 6), z(P, 3)
        self.obj = z(2)   # current, trial
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        sfm_ba_objective(self.X, cams, self.obs_point, self.obs_cam, self.obs_xy, self.delta, self.obj[0:1],
                         Rt=self.Rt)
        self.objective = float(self.obj[0].item())

    def _schur(self, lam):
        if self.plan is not None:
            sfm_ba_schur_pairs(self.U, self.Vp, self.gc, self.gp, self.Wo, self.obs_cam, self.off, self.ids, self.plan,
                               lam, self.S, self.rhs, self.Vinv, self.pair_ws)
        else:
            sfm_ba_schur(self.U, self.Vp, self.gc, self.gp, self.Wo, self.obs_cam, self.off, self.ids, lam, self.S,
                         self.rhs, self.Vinv)

    def step(self, mark=None) -> bool:
        """One LM iteration; returns whether the step was accepted.
        mark(name), if given, is called after each stage's launches."""
        mark = mark or (lambda name: None)
        for a in (self.U, self.Vp, self.gc, self.gp, self.obj[1:2]):
            gs_zero(a)
        sfm_ba_assemble(self.X, self.cams, self.obs_point, self.obs_cam, self.obs_xy, self.delta, self.U, self.Vp,
                        self.gc, self.gp, self.Wo, None, Rt=self.Rt)
        mark("assemble")
        self._schur(self.lam)
        mark("schur")
        sfm_ba_solve_cameras(self.S, self.rhs, self.dc, self.status)
        mark("solve_cameras")
        sfm_ba_back_substitute(self.Vinv, self.Vp, self.gp, self.Wo, self.obs_cam, self.off, self.ids, self.dc,
                               self.dp)
        mark("back_substitute")
        sfm_ba_apply_step(self.Rt, self.X, self.dc, self.dp, self.Rt_trial, self.X_trial)
        sfm_ba_objective(self.X_trial, self.cams, self.obs_point, self.obs_cam, self.obs_xy, self.delta,
                         self.obj[1:2], Rt=self.Rt_trial)
        mark("apply_and_objective")
        new = float(self.obj[1].item())
        if new < self.objective:
            self.Rt, self.Rt_trial = self.Rt_trial, self.Rt
            self.X, self.X_trial = self.X_trial, self.X
            self.objective = new
            self.lam /= 10.0
            return True
        self.lam *= 10.0
        return False

    def run(self, iters: int):
        """iters LM iterations; returns the objective after each."""
        hist = [self.objective]
        for _ in range(iters):
            self.step()
            hist.append(self.objective)
        return hist

    # -- the iteration on the device -----------------------------------------
    def _device_iteration(self):
        """One LM iteration whose accept / reject runs on the device
        (sfm_ba_lm_accept): no host synchronisation, capturable."""
        for a in (self.U, self.Vp, self.gc, self.gp, self.obj[1:2]):
            gs_zero(a)
        sfm_ba_assemble(self.X, self.cams, self.obs_point, self.obs_cam, self.obs_xy, self.delta, self.U, self.Vp,
                        self.gc, self.gp, self.Wo, None, Rt=self.Rt)
        self._schur(self.lam_dev)
        sfm_ba_solve_cameras(self.S, self.rhs, self.dc, self.status)
        sfm_ba_back_substitute(self.Vinv, self.Vp, self.gp, self.Wo, self.obs_cam, self.off, self.ids, self.dc,
                               self.dp)
        sfm_ba_apply_step(self.Rt, self.X, self.dc, self.dp, self.Rt_trial, self.X_trial)
        sfm_ba_objective(self.X_trial, self.cams, self.obs_point, self.obs_cam, self.obs_xy, self.delta,
                         self.obj[1:2], Rt=self.Rt_trial)
        sfm_ba_lm_accept(self.obj, self.lam_dev, self.Rt, self.X, self.Rt_trial, self.X_trial, self.n_acc_dev,
                         self.hist_dev, self.n_iter_dev)

    def run_graph(self, iters: int, max_iters: int = 4096):
        """iters LM iterations as replays of one CUDA graph of the device
        iteration (captured on first use); reads the results back once.
        Returns the objective after each iteration, like run()."""
        dev = self.X.device
        if getattr(self, "graph", None) is None:
            self.lam_dev = torch.tensor([self.lam], dtype=torch.float64, device=dev)
            self.n_acc_dev = torch.zeros(1, dtype=torch.int32, device=dev)
            self.n_iter_dev = torch.zeros(1, dtype=torch.int32, device=dev)
            self.hist_dev = torch.zeros(max_iters, dtype=torch.float64, device=dev)
            # the trial buffers are fixed in the graph: the current
            # parameters stay in self.Rt / self.X from here on
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._device_iteration()
        self.n_iter_dev.zero_()
        for _ in range(iters):
            self.graph.replay()
        hist = [self.objective] + self.hist_dev[:min(iters, self.hist_dev.numel())].cpu().tolist()
        self.objective = hist[-1]
        self.lam = float(self.lam_dev.item())
        return hist

    def accepted(self) -> int:
        """Steps accepted by run_graph so far."""
        return int(self.n_acc_dev.item()) if getattr(self, "n_acc_dev", None) is not None else 0

    def status_flags(self) -> int:
        return int(self.status.item())
