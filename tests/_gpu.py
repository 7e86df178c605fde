"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and the FP64 oracle on the same seeded inputs (the GPU receives the
float32-rounded parameters; the oracle gets the same values in double)."""
import numpy as np
import torch

import oracle


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def scene32(d):
    return {k: f32(v) for k, v in d.items()}


def oracle_scene(d):
    return oracle.Scene(**scene32(d))


def oracle_cam(wh, K, Rt, v, near=0.01, far=1e10):
    return oracle.camera_from_rt(int(wh[v][0]), int(wh[v][1]), f32(K[v]), f32(Rt[v]), near, far)


def gpu_forward(scene, wh, K, Rt, views, capacity=0, bg=(0.0, 0.0, 0.0), tile=16, deterministic=False):
    from paper_2603_04847_gb300 import Batch, Cameras, Gaussians, Renderer
    g = Gaussians.from_numpy(scene)
    cams = Cameras.from_numpy(wh, K, Rt)
    batch = Batch(cams, views, tile=tile)
    r = Renderer(g.n, cams, batch, capacity, bg=bg, deterministic=deterministic)
    r.ensure_capacity(g)
    r.forward(g)
    torch.cuda.synchronize()
    return r, g, cams, batch


def gpu_backward(r, g, v_image=None, target=None, l1_weight=1.0):
    from paper_2603_04847_gb300 import Gaussians
    dg = Gaussians.zeros_like(g)
    g_tan = torch.zeros((r.cams.V, 6), dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    if v_image is not None:
        v_image = torch.as_tensor(np.ascontiguousarray(v_image, dtype=np.float32), device="cuda")
    if target is not None:
        target = torch.as_tensor(np.ascontiguousarray(target, dtype=np.float32), device="cuda")
    r.backward(g, dg, g_tan, v_image=v_image, target=target, l1_weight=l1_weight, loss=loss)
    torch.cuda.synchronize()
    out = {k: t.detach().cpu().numpy().astype(np.float64)
           for k, t in zip(["mean", "log_scale", "quat", "opacity_logit", "sh"], dg.tensors())}
    out["tangent"] = g_tan.cpu().numpy()
    out["loss"] = float(loss.item())
    return out


def rel_linf(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def knife_mask(res):
    return res["knife"] & (oracle.KNIFE_ALPHA_MIN | oracle.KNIFE_T_MIN | oracle.KNIFE_DEPTH) != 0


def pose_rel_err(got, exp, exp_abs):
    """Pose-tangent error (rho and phi parts separately) against
    max(|g*|_inf, 1e-3 * sum |per-term contributions|): the pose gradient is
    a sum of many cancelling terms, each carrying FP32 rounding."""
    errs = []
    for part in (slice(0, 3), slice(3, 6)):
        den = max(np.abs(exp[part]).max(), 1e-3 * np.abs(exp_abs[part]).max(), 1e-30)
        errs.append(np.abs(np.asarray(got[part]) - exp[part]).max() / den)
    return max(errs)
