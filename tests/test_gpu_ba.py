"""Parity of sfm_ba_assemble (the normal-equation blocks of one LM iteration
of Eq. 4) with the FP64 oracle (oracle/ba.py), on the float32-rounded
inputs the GPU receives."""
import numpy as np
import pytest

from oracle import ba
from test_oracle_ba import _problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04847_gb300 import build
    build.build()


def _r32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _assemble(X, Rt, K, op, oc, xy, delta):
    from paper_2603_04847_gb300 import Cameras
    from paper_2603_04847_gb300.core import sfm_ba_assemble
    V, P, M = Rt.shape[0], X.shape[0], len(op)
    cams = Cameras.from_numpy(np.tile([400, 300], (V, 1)), K, Rt)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    U, Vp, gc, gp, Wo, obj = z(V, 36), z(P, 9), z(V, 6), z(P, 3), torch.full((M, 18), np.nan, dtype=torch.float64,
                                                                            device="cuda"), z(1)
    oc_d = dev(oc, torch.int32)
    sfm_ba_assemble(dev(X, torch.float32), cams, dev(op, torch.int32), oc_d, dev(xy, torch.float32), delta,
                    U, Vp, gc, gp, Wo, obj)
    return U, Vp, gc, gp, Wo, obj, oc_d


def _run(X, Rt, K, op, oc, xy, delta):
    out = _assemble(X, Rt, K, op, oc, xy, delta)[:6]
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _close(a, b, tol=1e-9):
    den = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= tol * den


def _check(got, X, Rt, K, op, oc, xy, delta, valid=None):
    U, Vp, gc, gp, Wo, obj = got
    sel = np.ones(len(op), bool) if valid is None else valid
    Ue, We, Ve, gce, gpe = ba.normal_equations(_r32(X), _r32(Rt), _r32(K), op[sel], oc[sel], _r32(xy)[sel], delta)
    assert _close(U.reshape(-1, 6, 6), Ue)
    assert _close(Vp.reshape(-1, 3, 3), Ve)
    assert _close(gc, gce) and _close(gp, gpe)
    assert _close(Wo[sel].reshape(-1, 6, 3), We)
    assert not np.any(Wo[~sel])
    L = ba.objective(_r32(X), _r32(Rt), _r32(K), op[sel], oc[sel], _r32(xy)[sel], delta)
    assert abs(obj[0] - L) <= 1e-9 * L


def test_blocks_match_the_oracle_sorted_by_camera():
    X, Rt, K, op, oc, xy = _problem(3, n_cams=5, n_pts=40, pix_noise=1.0, outliers=6)
    _check(_run(X, Rt, K, op, oc, xy, 1.0), X, Rt, K, op, oc, xy, 1.0)


def test_blocks_match_the_oracle_unsorted_with_invalid_observations():
    """Shuffled observations (warps mix cameras), one point behind camera 0
    and one observation of a point index out of range: both contribute
    nothing."""
    X, Rt, K, op, oc, xy = _problem(8, n_cams=4, n_pts=30, pix_noise=2.0, outliers=4)
    R0, t0 = Rt[0, :9].reshape(3, 3), Rt[0, 9:]
    centre = -R0.T @ t0
    X = np.vstack([X, centre - 1.0 * R0[2]])                      # behind camera 0
    P = X.shape[0]
    op = np.concatenate([op, [P - 1, P + 7]]).astype(np.int32)
    oc = np.concatenate([oc, [0, 1]]).astype(np.int32)
    xy = np.vstack([xy, [[10.0, 10.0], [20.0, 20.0]]])
    perm = np.random.default_rng(9).permutation(len(op))
    op, oc, xy = op[perm], oc[perm], xy[perm]
    valid = op < P
    _, _, front = ba.residuals(_r32(X), _r32(Rt), _r32(K), np.minimum(op, P - 1), oc, _r32(xy))
    valid &= front
    assert (~valid).sum() == 2
    _check(_run(X, Rt, K, op, oc, xy, 1.0), X, Rt, K, op, oc, xy, 1.0, valid=valid)


def _by_point(op, P):
    """CSR lists of each point's observations (in-range points only)."""
    ok = (op >= 0) & (op < P)
    ids = np.nonzero(ok)[0]
    ids = ids[np.argsort(op[ids], kind="stable")]
    off = np.concatenate([[0], np.cumsum(np.bincount(op[ok], minlength=P))]).astype(np.int64)
    return off, ids.astype(np.int32)


def _schur(pairs, U, Vp, gc, gp, Wo, oc, oc_d, off, ids, lam, S, rhs, Vinv):
    """sfm_ba_schur (atomics) or sfm_ba_schur_pairs (camera pairs, plan
    from sfm_ba_pair_lists with small chunks so that pairs span several)."""
    from paper_2603_04847_gb300.core import (sfm_ba_pair_lists, sfm_ba_schur, sfm_ba_schur_pairs,
                                             sfm_ba_schur_pairs_workspace)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    off_d, ids_d = dev(off, torch.int64), dev(ids, torch.int32)
    if not pairs:
        sfm_ba_schur(U, Vp, gc, gp, Wo, oc_d, off_d, ids_d, lam, S, rhs, Vinv)
        return
    V, P = U.shape[0], Vp.shape[0]
    plan = sfm_ba_pair_lists(V, P, oc, off, ids, chunk=7)
    plan_d = {k: dev(a, torch.int64 if a.dtype == np.int64 else torch.int32) for k, a in plan.items()}
    ws = torch.empty(sfm_ba_schur_pairs_workspace(len(oc), plan["chunk_start"].shape[0] - 1), dtype=torch.uint8,
                     device="cuda")
    sfm_ba_schur_pairs(U, Vp, gc, gp, Wo, oc_d, off_d, ids_d, plan_d, lam, S, rhs, Vinv, ws)


@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("lam", [1e-6, 1e-3, 1.0])
def test_schur_elimination_and_back_substitution_match_the_oracle(lam, pairs):
    from paper_2603_04847_gb300.core import sfm_ba_back_substitute
    X, Rt, K, op, oc, xy = _problem(3, n_cams=5, n_pts=40, pix_noise=1.0, outliers=6)
    X = np.vstack([X, [[0.3, 0.2, 0.1]]])          # a point nobody observes
    V, P = Rt.shape[0], X.shape[0]
    U, Vp, gc, gp, Wo, _, oc_d = _assemble(X, Rt, K, op, oc, xy, 1.0)
    off, ids = _by_point(op, P)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    off_d, ids_d = dev(off, torch.int64), dev(ids, torch.int32)
    S = torch.full((6 * V, 6 * V), np.nan, dtype=torch.float64, device="cuda")
    rhs = torch.full((6 * V,), np.nan, dtype=torch.float64, device="cuda")
    Vinv = torch.full((P, 9), np.nan, dtype=torch.float64, device="cuda")
    _schur(pairs, U, Vp, gc, gp, Wo, oc, oc_d, off, ids, lam, S, rhs, Vinv)
    blocks = ba.normal_equations(_r32(X), _r32(Rt), _r32(K), op, oc, _r32(xy), 1.0)
    S_e, rhs_e, Vinv_e, by_point, gp_reg = ba.schur_system(*blocks, op, oc, lam)
    dc = np.zeros((V, 6))
    dc[1:] = np.linalg.solve(S_e[6:, 6:], rhs_e[6:]).reshape(V - 1, 6)
    dp_e = ba.back_substitute(Vinv_e, gp_reg, by_point, dc)
    dp = torch.full((P, 3), np.nan, dtype=torch.float64, device="cuda")
    sfm_ba_back_substitute(Vinv, Vp, gp, Wo, oc_d, off_d, ids_d, dev(dc, torch.float64), dp)
    torch.cuda.synchronize()
    # S is symmetric and only its lower triangle is formed (all the camera
    # solve reads)
    assert _close(np.tril(S.cpu().numpy()), np.tril(S_e)) and _close(rhs.cpu().numpy(), rhs_e)
    assert _close(Vinv.cpu().numpy().reshape(-1, 3, 3), Vinv_e)
    assert _close(dp.cpu().numpy(), dp_e)
    assert not np.any(dp.cpu().numpy()[-1])         # the unobserved point stays put
    # the whole step equals the oracle's dense solve of the undivided system
    dc_d, dp_d = ba.solve_dense(*blocks, op, oc, lam)
    assert _close(dc, dc_d, 1e-7) and _close(dp.cpu().numpy(), dp_d, 1e-7)


def test_schur_by_camera_pairs_equals_the_atomic_form_and_is_reproducible():
    """Shuffled observations, a point seen twice by one camera, an
    observation of an out-of-range point: the pair form equals the atomic
    one to rounding (lower triangle of S, rhs, Vinv), and two runs of it are
    bit-identical."""
    X, Rt, K, op, oc, xy = _problem(5, n_cams=6, n_pts=60, pix_noise=1.0, outliers=5)
    P = X.shape[0]
    op = np.concatenate([op, [3, P + 2]]).astype(np.int32)
    oc = np.concatenate([oc, [oc[np.nonzero(op == 3)[0][0]], 2]]).astype(np.int32)   # point 3 twice in one camera
    xy = np.vstack([xy, xy[np.nonzero(op == 3)[0][0]] + 0.5, [[5.0, 5.0]]])
    perm = np.random.default_rng(2).permutation(len(op))
    op, oc, xy = op[perm], oc[perm], xy[perm]
    V = Rt.shape[0]
    U, Vp, gc, gp, Wo, _, oc_d = _assemble(X, Rt, K, op, oc, xy, 1.0)
    off, ids = _by_point(op, P)
    outs = []
    for pairs in (False, True, True):
        S = torch.full((6 * V, 6 * V), np.nan, dtype=torch.float64, device="cuda")
        rhs = torch.full((6 * V,), np.nan, dtype=torch.float64, device="cuda")
        Vinv = torch.full((P, 9), np.nan, dtype=torch.float64, device="cuda")
        _schur(pairs, U, Vp, gc, gp, Wo, oc, oc_d, off, ids, 1e-3, S, rhs, Vinv)
        torch.cuda.synchronize()
        outs.append((np.tril(S.cpu().numpy()), rhs.cpu().numpy(), Vinv.cpu().numpy()))
    (Sa, ra, va), (Sp, rp, vp), (Sq, rq, vq) = outs
    assert _close(Sp, Sa, 1e-12) and _close(rp, ra, 1e-12)
    np.testing.assert_array_equal(vp, va)
    np.testing.assert_array_equal(Sp, Sq)
    np.testing.assert_array_equal(rp, rq)


@pytest.mark.parametrize("lam", [1e-6, 1e-3, 1.0])
def test_one_lm_step_on_the_gpu_equals_the_oracle_dense_solve(lam):
    """assemble -> eliminate the points -> solve the cameras (camera 0
    fixed) -> back-substitute: the step equals the oracle's dense solve."""
    from paper_2603_04847_gb300.core import sfm_ba_back_substitute, sfm_ba_schur, sfm_ba_solve_cameras
    X, Rt, K, op, oc, xy = _problem(11, n_cams=6, n_pts=50, pix_noise=1.0, outliers=5)
    V, P = Rt.shape[0], X.shape[0]
    U, Vp, gc, gp, Wo, _, oc_d = _assemble(X, Rt, K, op, oc, xy, 1.0)
    off, ids = _by_point(op, P)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    off_d, ids_d = dev(off, torch.int64), dev(ids, torch.int32)
    S = torch.empty((6 * V, 6 * V), dtype=torch.float64, device="cuda")
    rhs = torch.empty(6 * V, dtype=torch.float64, device="cuda")
    Vinv = torch.empty((P, 9), dtype=torch.float64, device="cuda")
    dc = torch.full((V, 6), np.nan, dtype=torch.float64, device="cuda")
    dp = torch.full((P, 3), np.nan, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sfm_ba_schur(U, Vp, gc, gp, Wo, oc_d, off_d, ids_d, lam, S, rhs, Vinv)
    sfm_ba_solve_cameras(S, rhs, dc, status)
    sfm_ba_back_substitute(Vinv, Vp, gp, Wo, oc_d, off_d, ids_d, dc, dp)
    torch.cuda.synchronize()
    blocks = ba.normal_equations(_r32(X), _r32(Rt), _r32(K), op, oc, _r32(xy), 1.0)
    dc_e, dp_e = ba.solve_dense(*blocks, op, oc, lam)
    assert int(status.item()) == 0
    got_c, got_p = dc.cpu().numpy(), dp.cpu().numpy()
    assert not np.any(got_c[0])
    assert _close(got_c, dc_e, 1e-7) and _close(got_p, dp_e, 1e-7)


def _perturbed(seed_problem, seed_noise, n_cams, n_pts, pix_noise=0.0, outliers=0, dpose=0.01, dpt=0.02):
    X, Rt, K, op, oc, xy = _problem(seed_problem, n_cams=n_cams, n_pts=n_pts, pix_noise=pix_noise, outliers=outliers)
    rng = np.random.default_rng(seed_noise)
    dc = rng.normal(0, dpose, (Rt.shape[0], 6))
    dc[0] = 0.0
    X0, Rt0 = ba.apply_update(X, Rt, dc, rng.normal(0, dpt, X.shape))
    return _r32(X0), _r32(Rt0), _r32(K), op, oc, _r32(xy)


def _adjuster(X0, Rt0, K, op, oc, xy):
    from paper_2603_04847_gb300 import Cameras
    from paper_2603_04847_gb300.ba import BundleAdjuster
    cams = Cameras.from_numpy(np.tile([400, 300], (Rt0.shape[0], 1)), K, Rt0)
    X = torch.as_tensor(X0, dtype=torch.float32, device="cuda")
    return BundleAdjuster(cams, X, op, oc, xy, delta=1.0, lam=1e-4)


def test_gpu_lm_first_iteration_matches_the_oracle():
    X0, Rt0, K, op, oc, xy = _perturbed(4, 5, 4, 20, pix_noise=0.5, outliers=3)
    adj = _adjuster(X0, Rt0, K, op, oc, xy)
    L0 = ba.objective(X0, Rt0, K, op, oc, xy, 1.0)
    assert abs(adj.objective - L0) <= 1e-9 * L0
    accepted = adj.step()
    Xo, Rto, hist = ba.lm(X0, Rt0, K, op, oc, xy, delta=1.0, iters=1, lam=1e-4)
    assert accepted == (hist[1] < hist[0])
    assert np.abs(adj.X.cpu().numpy() - Xo).max() <= 1e-5
    assert np.abs(adj.Rt.cpu().numpy() - Rto).max() <= 1e-5
    assert abs(adj.objective - hist[1]) <= 1e-4 * hist[1]


def test_gpu_lm_recovers_a_noiseless_problem():
    X0, Rt0, K, op, oc, xy = _perturbed(4, 5, 4, 20)
    adj = _adjuster(X0, Rt0, K, op, oc, xy)
    hist = adj.run(30)
    assert hist[0] > 1.0
    assert hist[-1] < 1e-6 * hist[0]
    assert all(b <= a for a, b in zip(hist[:-1], hist[1:]))
    np.testing.assert_array_equal(adj.Rt.cpu().numpy()[0], np.float32(Rt0[0]))
    assert adj.status_flags() == 0


def test_gpu_lm_converges_at_the_benchmark_size():
    """The bundle adjustment at the size the benchmark times: 50 cameras
    (1000x750) on a radius-4 sphere, 20k points seen by 2-12 cameras each
    (~140k observations), 0.5 px noise, 2 % outliers uniform over the image,
    poses and points perturbed.  LM never raises the robust objective, and
    within 20 iterations it falls below its value at the true parameters
    (the optimum also fits part of the pixel noise), camera 0 held fixed."""
    import synth
    from paper_2603_04847_gb300 import Cameras
    from paper_2603_04847_gb300.ba import BundleAdjuster
    from paper_2603_04847_gb300.core import sfm_ba_objective
    rng = np.random.default_rng(0)
    V, P, W, H = 50, 20000, 1000, 750
    wh, K, Rt = synth.cameras_sphere(rng, V, (W, W), (H, H))
    X = rng.uniform(-1, 1, (P, 3))
    tr = synth.tracks(rng, X, P, (2, 12), V, 0.5, 0.02)
    op, oc = tr["obs_point"], tr["obs_view"]
    R, t = Rt[oc, :9].reshape(-1, 3, 3), Rt[oc, 9:]
    xc = np.einsum("mab,mb->ma", R, X[op]) + t
    xy = np.stack([K[oc, 0] * xc[:, 0] / xc[:, 2] + K[oc, 2], K[oc, 1] * xc[:, 1] / xc[:, 2] + K[oc, 3]], 1)
    xy = xy + tr["noise"]
    xy[tr["outlier"]] = tr["outlier_uv01"][tr["outlier"]] * [W, H]
    dc = rng.normal(0, 0.002, (V, 6))
    dc[0] = 0.0
    X0, Rt0 = ba.apply_update(X, Rt, dc, rng.normal(0, 0.005, X.shape))
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    truth = torch.zeros(1, dtype=torch.float64, device="cuda")
    cams_t = Cameras.from_numpy(wh, K, Rt)
    sfm_ba_objective(dev(X, torch.float32), cams_t, dev(op, torch.int32), dev(oc, torch.int32),
                     dev(xy, torch.float32), 1.0, truth)
    adj = BundleAdjuster(Cameras.from_numpy(wh, K, Rt0), dev(X0, torch.float32), op, oc, xy, delta=1.0, lam=1e-4)
    hist = adj.run(20)
    assert all(b <= a for a, b in zip(hist[:-1], hist[1:]))
    assert hist[-1] < hist[0]
    assert hist[-1] <= float(truth.item()), (hist[0], hist[-1], float(truth.item()))
    np.testing.assert_array_equal(adj.Rt.cpu().numpy()[0], np.float32(Rt0[0]))
    assert adj.status_flags() == 0
    # the same iterations with the accept / reject on the device, replayed
    # from one CUDA graph: the same kernels, so the same objectives up to
    # the order of the objective's FP64 atomic sums (~1e-16 relative)
    g = BundleAdjuster(Cameras.from_numpy(wh, K, Rt0), dev(X0, torch.float32), op, oc, xy, delta=1.0, lam=1e-4)
    hg = g.run_graph(20)
    np.testing.assert_allclose(hg, hist, rtol=1e-12)
    np.testing.assert_allclose(g.X.cpu().numpy(), adj.X.cpu().numpy(), rtol=0, atol=1e-6)
    np.testing.assert_allclose(g.Rt.cpu().numpy(), adj.Rt.cpu().numpy(), rtol=0, atol=1e-6)
    assert g.status_flags() == 0


def test_gpu_lm_device_loop_matches_the_host_loop_and_recovers_a_noiseless_problem():
    """The graph-replayed device loop follows the host loop (until the
    objective reaches rounding level, where equal-looking objectives may
    order differently) and recovers the noiseless problem."""
    X0, Rt0, K, op, oc, xy = _perturbed(4, 5, 4, 20)
    h = _adjuster(X0, Rt0, K, op, oc, xy).run(30)
    adj = _adjuster(X0, Rt0, K, op, oc, xy)
    g = adj.run_graph(10)
    g += adj.run_graph(20)[1:]      # replays continue from the device state
    # the objective's FP64 atomic sums may round differently run to run
    np.testing.assert_allclose(g[:15], h[:15], rtol=1e-9)
    assert g[-1] < 1e-6 * g[0]
    assert all(b <= a for a, b in zip(g[:-1], g[1:]))
    assert adj.accepted() >= 10


def test_tiled_camera_solve_not_positive_definite_flags_and_zeroes():
    """A reduced camera system that is not positive definite (a negative
    diagonal entry in the third 32 x 32 tile): dc stays zero, the flag is
    raised, and no later tile runs on the failed factor."""
    from paper_2603_04847_gb300.core import sfm_ba_solve_cameras
    V = 20                                   # n = 114 unknowns: 4 tiles, the last ragged
    n = 6 * V
    rng = np.random.default_rng(3)
    B = rng.normal(size=(n, n))
    S = B @ B.T + n * np.eye(n)
    S[6 + 70, 6 + 70] = -1.0
    St = torch.as_tensor(S, dtype=torch.float64, device="cuda").contiguous()
    dc = torch.full((V, 6), np.nan, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sfm_ba_solve_cameras(St, torch.ones(n, dtype=torch.float64, device="cuda"), dc, status)
    torch.cuda.synchronize()
    from paper_2603_04847_gb300 import _lib
    assert int(status.item()) & _lib.GS_FLAG_NOT_SPD
    assert not dc.cpu().numpy().any()


@pytest.mark.parametrize("V", [2, 7, 12, 50, 120])
def test_tiled_camera_solve_equals_a_dense_solve(V):
    """The tiled factorization and the two tiled triangular solves against
    numpy's dense solve of S' x = rhs', for systems of 1 to 22 tiles (ragged
    last tile at 6 (V - 1) = 6, 36, 66, 294, 714 unknowns)."""
    from paper_2603_04847_gb300.core import sfm_ba_solve_cameras
    n = 6 * V
    rng = np.random.default_rng(V)
    B = rng.normal(size=(n, n))
    S = B @ B.T / n + np.diag(rng.uniform(0.5, 2.0, n))
    rhs = rng.normal(size=n)
    St = torch.as_tensor(S, dtype=torch.float64, device="cuda").contiguous()
    dc = torch.full((V, 6), np.nan, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sfm_ba_solve_cameras(St, torch.as_tensor(rhs, device="cuda"), dc, status)
    torch.cuda.synchronize()
    exp = np.linalg.solve(S[6:, 6:], rhs[6:])
    got = dc.cpu().numpy().reshape(-1)
    assert int(status.item()) == 0
    assert not got[:6].any()
    assert np.abs(got[6:] - exp).max() <= 1e-10 * np.abs(exp).max()
    L = np.tril(St.cpu().numpy()[6:, 6:])
    np.testing.assert_allclose(L, np.linalg.cholesky(S[6:, 6:]), rtol=0, atol=1e-12 * np.abs(L).max())
