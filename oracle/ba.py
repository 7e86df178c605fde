"""FP64 oracle of the SfM bundle adjustment of Eq. 4 (Sec. 3.2, "Bundle
Adjustment"): Levenberg-Marquardt over SE(3) camera poses and 3-D points on
the Huber reprojection objective

    L = sum over observations o = (camera i, point k, pixel x) of
        rho(|pi_i(X_k) - x|^2),   pi_i(X) = proj(K_i (R_i X + t_i)).

TEST INFRASTRUCTURE ONLY, like the rest of this package: no product code
imports it.  Plain numpy; every array is float64.

The paper cites its solver (BAE with cuDSS) and states only LM on SE(3).
Where it is silent this oracle takes these readings:
  * rho is the Huber function on the squared residual, as the joint step
    reads Eq. 6: rho(s) = s for s <= delta^2, else 2 delta sqrt(s) - delta^2;
    observations whose camera depth is <= near are left out;
  * a pose moves by a left perturbation T <- Exp(d) T, d = (rho, phi),
    translation first, as in the joint step;
  * the robust loss enters as iteratively reweighted least squares: each
    observation's Gauss-Newton terms carry w = rho'(s);
  * Marquardt damping (H + lambda diag(H)) d = -g; lambda x 10 after a
    rejected step, / 10 after an accepted one;
  * the gauge: camera 0 is held fixed (its unknowns are removed);
  * the points are eliminated with the Schur complement and the reduced
    camera system is solved densely.
"""
from __future__ import annotations

import numpy as np

NEAR = 0.01


def _split(Rt):
    Rt = np.asarray(Rt, np.float64).reshape(-1, 12)
    return Rt[:, :9].reshape(-1, 3, 3), Rt[:, 9:]


def huber_rho(s, delta):
    s = np.asarray(s, np.float64)
    return np.where(s <= delta * delta, s, 2.0 * delta * np.sqrt(s) - delta * delta)


def huber_weight(s, delta):
    """rho'(s)."""
    s = np.asarray(s, np.float64)
    return np.where(s <= delta * delta, 1.0, delta / np.sqrt(np.maximum(s, 1e-300)))


def residuals(X, Rt, K, obs_point, obs_cam, obs_xy):
    """r [M,2] = pi(X_k) - x per observation, the camera points x_c [M,3] and
    a mask of the observations in front of the near plane."""
    R, t = _split(Rt)
    K = np.asarray(K, np.float64).reshape(-1, 4)
    X = np.asarray(X, np.float64).reshape(-1, 3)
    i, k = np.asarray(obs_cam), np.asarray(obs_point)
    xc = np.einsum("mab,mb->ma", R[i], X[k]) + t[i]
    z = xc[:, 2]
    ok = z > NEAR
    zs = np.where(ok, z, 1.0)
    uv = np.stack([K[i, 0] * xc[:, 0] / zs + K[i, 2], K[i, 1] * xc[:, 1] / zs + K[i, 3]], axis=1)
    return uv - np.asarray(obs_xy, np.float64).reshape(-1, 2), xc, ok


def objective(X, Rt, K, obs_point, obs_cam, obs_xy, delta):
    r, _, ok = residuals(X, Rt, K, obs_point, obs_cam, obs_xy)
    s = (r * r).sum(1)
    return float(huber_rho(s[ok], delta).sum())


def jacobians(X, Rt, K, obs_point, obs_cam):
    """Per observation: J_pose [M,2,6] = d r / d(rho, phi) of T <- Exp(d) T
    at d = 0, and J_X [M,2,3] = d r / d X_k.  With x_c = R X + t:
    d x_c / d rho = I, d x_c / d phi = -[x_c]_x, d x_c / d X = R."""
    R, t = _split(Rt)
    K = np.asarray(K, np.float64).reshape(-1, 4)
    X = np.asarray(X, np.float64).reshape(-1, 3)
    i, k = np.asarray(obs_cam), np.asarray(obs_point)
    xc = np.einsum("mab,mb->ma", R[i], X[k]) + t[i]
    x, y, z = xc[:, 0], xc[:, 1], np.where(xc[:, 2] > NEAR, xc[:, 2], 1.0)
    fx, fy = K[i, 0], K[i, 1]
    M = xc.shape[0]
    P = np.zeros((M, 2, 3))          # d pi / d x_c
    P[:, 0, 0] = fx / z
    P[:, 0, 2] = -fx * x / (z * z)
    P[:, 1, 1] = fy / z
    P[:, 1, 2] = -fy * y / (z * z)
    skew = np.zeros((M, 3, 3))
    skew[:, 0, 1], skew[:, 0, 2] = -xc[:, 2], xc[:, 1]
    skew[:, 1, 0], skew[:, 1, 2] = xc[:, 2], -xc[:, 0]
    skew[:, 2, 0], skew[:, 2, 1] = -xc[:, 1], xc[:, 0]
    Jp = np.concatenate([P, -np.einsum("mab,mbc->mac", P, skew)], axis=2)
    JX = np.einsum("mab,mbc->mac", P, R[i])
    return Jp, JX


def normal_equations(X, Rt, K, obs_point, obs_cam, obs_xy, delta):
    """IRLS Gauss-Newton blocks (the factor 2 of d rho(|r|^2) cancels):
    U [V,6,6] = sum w Jp^T Jp, Wb [M,6,3] = w Jp^T JX per observation,
    Vb [P,3,3] = sum w JX^T JX, gc [V,6] = sum w Jp^T r, gp [P,3] = sum w JX^T r.
    Observations behind the near plane contribute nothing."""
    r, _, ok = residuals(X, Rt, K, obs_point, obs_cam, obs_xy)
    Jp, JX = jacobians(X, Rt, K, obs_point, obs_cam)
    w = huber_weight((r * r).sum(1), delta) * ok
    V = np.asarray(Rt).reshape(-1, 12).shape[0]
    Pn = np.asarray(X).reshape(-1, 3).shape[0]
    i, k = np.asarray(obs_cam), np.asarray(obs_point)
    U = np.zeros((V, 6, 6))
    Vb = np.zeros((Pn, 3, 3))
    gc = np.zeros((V, 6))
    gp = np.zeros((Pn, 3))
    np.add.at(U, i, w[:, None, None] * np.einsum("mai,maj->mij", Jp, Jp))
    np.add.at(Vb, k, w[:, None, None] * np.einsum("mai,maj->mij", JX, JX))
    np.add.at(gc, i, w[:, None] * np.einsum("mai,ma->mi", Jp, r))
    np.add.at(gp, k, w[:, None] * np.einsum("mai,ma->mi", JX, r))
    Wb = w[:, None, None] * np.einsum("mai,maj->mij", Jp, JX)
    return U, Wb, Vb, gc, gp


def _regularise(U, Vb, gc, gp):
    """Cameras or points without a valid observation stay put: identity
    blocks and zero right-hand sides for them."""
    U, Vb, gc, gp = U.copy(), Vb.copy(), gc.copy(), gp.copy()
    for A, g in ((U, gc), (Vb, gp)):
        empty = np.all(A == 0.0, axis=(1, 2))
        A[empty] = np.eye(A.shape[1])
        g[empty] = 0.0
    return U, Vb, gc, gp


def _damp(A, lam):
    d = np.einsum("nii->ni", A)
    return A + lam * np.einsum("ni,ij->nij", d, np.eye(A.shape[1]))


def solve_dense(U, Wb, Vb, gc, gp, obs_point, obs_cam, lam):
    """The damped normal equations (H + lam diag(H)) d = -g assembled whole,
    camera 0 removed.  Returns d_cam [V,6] (row 0 zero) and d_pt [P,3]."""
    U, Vb, gc, gp = _regularise(U, Vb, gc, gp)
    V, P = U.shape[0], Vb.shape[0]
    nc = 6 * (V - 1)
    H = np.zeros((nc + 3 * P, nc + 3 * P))
    Ud, Vd = _damp(U, lam), _damp(Vb, lam)
    for i in range(1, V):
        H[6 * (i - 1):6 * i, 6 * (i - 1):6 * i] = Ud[i]
    for k in range(P):
        H[nc + 3 * k:nc + 3 * k + 3, nc + 3 * k:nc + 3 * k + 3] = Vd[k]
    for o, (i, k) in enumerate(zip(obs_cam, obs_point)):
        if i == 0:
            continue
        a, b = 6 * (i - 1), nc + 3 * k
        H[a:a + 6, b:b + 3] += Wb[o]
        H[b:b + 3, a:a + 6] += Wb[o].T
    g = np.concatenate([gc[1:].reshape(-1), gp.reshape(-1)])
    d = np.linalg.solve(H, -g)
    dc = np.zeros((V, 6))
    dc[1:] = d[:nc].reshape(V - 1, 6)
    return dc, d[nc:].reshape(P, 3)


def schur_system(U, Wb, Vb, gc, gp, obs_point, obs_cam, lam):
    """The damped system with the points eliminated, over all cameras:
    S = U - sum_k W_ik V_k^-1 W_jk^T  [6V, 6V],
    rhs = -gc + sum_k W_ik V_k^-1 gp_k  [6V],
    and the damped point blocks' inverses V_k^-1 [P,3,3] (W_ik summed over
    the observations of camera i and point k)."""
    U, Vb, gc, gp = _regularise(U, Vb, gc, gp)
    V, P = U.shape[0], Vb.shape[0]
    Ud, Vd = _damp(U, lam), _damp(Vb, lam)
    Vinv = np.linalg.inv(Vd)
    Wik = {}
    for o, (i, k) in enumerate(zip(obs_cam, obs_point)):
        Wik[(int(i), int(k))] = Wik.get((int(i), int(k)), 0.0) + Wb[o]
    by_point = {}
    for (i, k), W in Wik.items():
        by_point.setdefault(k, []).append((i, W))
    S = np.zeros((6 * V, 6 * V))
    rhs = -gc.reshape(-1).copy()
    for i in range(V):
        S[6 * i:6 * i + 6, 6 * i:6 * i + 6] = Ud[i]
    for k, lst in by_point.items():
        for i, Wi in lst:
            rhs[6 * i:6 * i + 6] += Wi @ Vinv[k] @ gp[k]
            for j, Wj in lst:
                S[6 * i:6 * i + 6, 6 * j:6 * j + 6] -= Wi @ Vinv[k] @ Wj.T
    return S, rhs, Vinv, by_point, gp


def back_substitute(Vinv, gp_reg, by_point, dc):
    """d_pt_k = V_k^-1 (-gp_k - sum_i W_ik^T d_cam_i)."""
    dp = np.zeros((Vinv.shape[0], 3))
    for k in range(Vinv.shape[0]):
        b = -gp_reg[k].copy()
        for i, Wi in by_point.get(k, []):
            b -= Wi.T @ dc[i]
        dp[k] = Vinv[k] @ b
    return dp


def solve_schur(U, Wb, Vb, gc, gp, obs_point, obs_cam, lam):
    """The same system as solve_dense with the points eliminated
    (schur_system), the reduced camera system solved with camera 0 held
    fixed, then the points back-substituted."""
    S, rhs, Vinv, by_point, gp_reg = schur_system(U, Wb, Vb, gc, gp, obs_point, obs_cam, lam)
    V = U.shape[0]
    dc = np.zeros((V, 6))
    dc[1:] = np.linalg.solve(S[6:, 6:], rhs[6:]).reshape(V - 1, 6)
    return dc, back_substitute(Vinv, gp_reg, by_point, dc)


def se3_exp(d):
    """Exp of a tangent (rho, phi) as a [3,4] transform [R | t] with
    R = Rodrigues(phi), t = J_l(phi) rho (the left Jacobian of SO(3))."""
    rho, phi = np.asarray(d[:3], np.float64), np.asarray(d[3:], np.float64)
    th = np.linalg.norm(phi)
    Wx = np.array([[0.0, -phi[2], phi[1]], [phi[2], 0.0, -phi[0]], [-phi[1], phi[0], 0.0]])
    if th < 1e-12:
        R = np.eye(3) + Wx
        J = np.eye(3) + 0.5 * Wx
    else:
        a = np.sin(th) / th
        b = (1.0 - np.cos(th)) / (th * th)
        c = (th - np.sin(th)) / (th ** 3)
        R = np.eye(3) + a * Wx + b * Wx @ Wx
        J = np.eye(3) + b * Wx + c * Wx @ Wx
    return np.concatenate([R, (J @ rho)[:, None]], axis=1)


def apply_update(X, Rt, dc, dp):
    """T_i <- Exp(dc_i) T_i (left perturbation), X_k <- X_k + dp_k."""
    R, t = _split(Rt)
    out = np.zeros((R.shape[0], 12))
    for i in range(R.shape[0]):
        E = se3_exp(dc[i])
        Rn = E[:, :3] @ R[i]
        tn = E[:, :3] @ t[i] + E[:, 3]
        out[i, :9] = Rn.reshape(-1)
        out[i, 9:] = tn
    return np.asarray(X, np.float64).reshape(-1, 3) + dp, out


def lm(X, Rt, K, obs_point, obs_cam, obs_xy, delta=1.0, iters=20, lam=1e-4, schur=True):
    """Levenberg-Marquardt on Eq. 4.  Returns the final X, Rt and the
    objective after each iteration (accepted steps only lower it)."""
    X = np.asarray(X, np.float64).reshape(-1, 3).copy()
    Rt = np.asarray(Rt, np.float64).reshape(-1, 12).copy()
    L = objective(X, Rt, K, obs_point, obs_cam, obs_xy, delta)
    hist = [L]
    solve = solve_schur if schur else solve_dense
    for _ in range(iters):
        U, Wb, Vb, gc, gp = normal_equations(X, Rt, K, obs_point, obs_cam, obs_xy, delta)
        dc, dp = solve(U, Wb, Vb, gc, gp, obs_point, obs_cam, lam)
        X2, Rt2 = apply_update(X, Rt, dc, dp)
        L2 = objective(X2, Rt2, K, obs_point, obs_cam, obs_xy, delta)
        if L2 < L:
            X, Rt, L = X2, Rt2, L2
            lam /= 10.0
        else:
            lam *= 10.0
        hist.append(L)
    return X, Rt, hist
