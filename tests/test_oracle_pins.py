"""Pins of the CPU oracle against things other than itself.

Closed forms (single Gaussian, two-Gaussian ordering, unified-camera
geometry), library routines (numpy matmul for the MLP, scipy rotations for
the quaternion convention, torch casts for bf16/fp8), brute force (tiled vs
per-pixel blending, dense sampling for tile coverage), Monte Carlo for the EWA
linearisation, and the blending invariants.  No GPU needed.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import expit

import gen
import oracle
from conftest import axis_camera, single_gaussian_model


# ---------------------------------------------------------------- single Gaussian
@pytest.mark.parametrize("o,sig_s,z0", [(0.5, 0.5, 10.0), (0.999, 0.7, 4.0), (0.05, 0.3, 25.0)])
def test_single_gaussian_closed_form(o, sig_s, z0):
    """Eq. 1-2 + EWA + blending for one isotropic Gaussian on the optical axis:
    sigma'^2 = (f s / z)^2 + 0.3 and pixel = c min(0.99, o exp(-r^2 / 2 sigma'^2))
    when that alpha is >= 1/255, else 0 (Sec. 3.1)."""
    m = single_gaussian_model(o=o, sig_s=sig_s, z0=z0)
    cam = axis_camera()
    (rgb, T, mg, nc), vr = oracle.render_view(m, cam)
    b2 = [b.astype(np.float64) for b in m.b2]
    o_ = np.tanh(b2[0][0])
    col = expit(b2[1][0:3])
    s = float(m.scale[0]) * expit(b2[2][0])
    sig2 = (cam.fx * s / z0) ** 2 + 0.3
    xs = np.arange(cam.width) + 0.5 - cam.cx
    ys = np.arange(cam.height) + 0.5 - cam.cy
    r2 = xs[None, :] ** 2 + ys[:, None] ** 2
    al = np.minimum(0.99, o_ * np.exp(-r2 / (2 * sig2)))
    al = np.where(al >= 1 / 255, al, 0.0)
    exp = al[..., None] * col[None, None, :]
    assert np.abs(rgb - exp).max() < 1e-12
    assert np.abs(T - (1 - al)).max() < 1e-12
    assert int(vr.rec[:, 0].sum()) == 1


def test_two_gaussian_order():
    """C = c1 a1 + c2 a2 (1 - a1) for the nearer Gaussian first; moving the
    far one in front swaps the roles (front-to-back order by depth)."""
    import gen as g
    k = 10
    W1, b1, W2, b2 = g.glorot_mlps(5, k)
    W2 = [np.zeros_like(w) for w in W2]
    b2 = [np.zeros_like(b) for b in b2]
    b2[0][:] = -1.0
    b2[0][0] = np.arctanh(0.6)
    b2[1][0:3] = [2.0, -2.0, 0.0]
    b2[2][0:3] = 0.0
    b2[2][3:7] = [1, 0, 0, 0]
    b2 = [b.astype(np.float32) for b in b2]

    def model(z_a, z_b):
        # both anchors derive the same attributes (zero layer-2 weights), so
        # only their depths decide which one is blended first
        return g.Model(pos=np.array([[0, 0, z_a], [0, 0, z_b]], np.float32),
                       feat=np.zeros((2, 32), np.float32), offs=np.zeros((2, k, 3), np.float32),
                       scale=np.array([0.2, 0.2], np.float32), level=np.zeros(2, np.uint8), n_levels=1,
                       lod_dmax=0.0, W1=W1, b1=b1, W2=W2, b2=b2, k=k)

    cam = axis_camera()
    px, py = np.array([64]), np.array([48])
    for za, zb in [(5.0, 8.0), (8.0, 5.0)]:
        m = model(za, zb)
        vr = oracle.view_gaussians(m, cam)
        recs = vr.rec[vr.rec[:, 0] > 0]
        assert recs.shape[0] == 2
        rgb, T, _, nc = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, True, px, py)
        # per-Gaussian alpha at the pixel, in depth order
        near = 0 if za < zb else 1
        far = 1 - near
        X, Y = 64.5, 48.5
        def alpha(r):
            dx, dy = X - r[1], Y - r[2]
            q = r[3] * dx * dx + 2 * r[4] * dx * dy + r[5] * dy * dy
            return min(0.99, r[6] * np.exp(-0.5 * q))
        a1, a2 = alpha(recs[near]), alpha(recs[far])
        c = recs[0, 7:10]
        exp = c * a1 + c * a2 * (1 - a1)
        assert np.allclose(rgb[0], exp, atol=1e-14)
        assert abs(T[0] - (1 - a1) * (1 - a2)) < 1e-14
        assert nc[0] == 2
        # the nearer (larger on screen) Gaussian has the larger footprint
        assert recs[near, 12] > recs[far, 12]


# ---------------------------------------------------------------- brute force vs tiled
def test_tiled_equals_brute_force_tiny(tiny):
    """Tiling + opacity-aware exact coverage + sort is lossless (Sec. 6):
    every pixel equals the per-pixel brute force over all Gaussians."""
    m, cam = tiny
    (rgb, T, mg, nc), vr = oracle.render_view(m, cam)
    rs = np.random.default_rng(3)
    px = rs.integers(0, cam.width, 3000)
    py = rs.integers(0, cam.height, 3000)
    b_rgb, b_T, _, b_nc = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, False, px, py)
    assert np.array_equal(b_rgb, rgb[py, px])
    assert np.array_equal(b_T, T[py, px])
    assert np.array_equal(b_nc, nc[py, px])


def test_tiled_equals_brute_force_big_gaussians():
    """Same identity with large, elongated, rotated Gaussians near the camera
    that cover many tiles and cross the image border."""
    m = gen.tiny_scene(seed=7, n=60)
    m.offs *= 10
    m.scale *= 30
    cam = gen.tiny_camera(200, 150)
    (rgb, T, mg, nc), vr = oracle.render_view(m, cam)
    px, py = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    b_rgb, b_T, _, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height, False,
                                     px.ravel(), py.ravel())
    assert np.array_equal(b_rgb.reshape(rgb.shape), rgb)
    assert (nc > 0).mean() > 0.5


# ---------------------------------------------------------------- blending invariants
def test_blend_invariants_trace():
    """T non-increasing, weights summing to 1 - T_final <= 1, alpha <= 0.99,
    nothing below 1/255 contributes, nothing after T (1 - alpha) < 1e-4."""
    rs = np.random.default_rng(0)
    for trial in range(200):
        n = int(rs.integers(1, 200))
        a = np.exp(rs.uniform(np.log(1e-4), np.log(1.5), n))
        c = rs.uniform(0, 1, (n, 3))
        tr, rgb, Tf = oracle.blend_trace(a, c)
        used = tr[:, 0]
        Tb = tr[:, 1]
        w = tr[:, 2]
        assert np.all(np.diff(Tb) <= 0)
        assert abs(w.sum() - (1 - Tf)) < 1e-12 and w.sum() <= 1 + 1e-15
        assert np.all(used[used >= 0] <= 0.99)
        skipped = used < 0
        assert np.all(np.minimum(0.99, a[: len(used)][skipped]) < 1 / 255)
        assert np.all(w[skipped] == 0)
        if len(used) < n or (len(used) == n and Tb[-1] * (1 - max(used[-1], 0)) < 1e-4 and used[-1] >= 0):
            # stopped: the last visited entry was not added and would have crossed 1e-4
            last = len(used) - 1
            if used[last] >= 0 and Tb[last] * (1 - used[last]) < 1e-4:
                assert w[last] == 0
        # everything before the stop keeps T above the bound
        contrib = w > 0
        assert np.all(Tb[contrib] * (1 - used[contrib]) >= 1e-4)
        assert np.all(rgb <= 1 - Tf + 1e-12)


def test_blend_invariants_image(tiny):
    m, cam = tiny
    (rgb, T, mg, nc), vr = oracle.render_view(m, cam)
    assert np.all((T >= 1e-4 - 1e-15) & (T <= 1))
    assert np.all(rgb.max(axis=-1) <= 1 - T + 1e-12)
    assert np.all(rgb >= 0)


# ---------------------------------------------------------------- EWA linearisation (Monte Carlo)
def test_ewa_monte_carlo():
    """For a small Gaussian, the covariance of exactly projected samples
    approaches Sigma' - 0.3 I (the EWA first-order projection)."""
    cam = axis_camera(400, 300, 300.0)
    mu = np.array([0.7, -0.4, 6.0])
    s = np.array([0.03, 0.012, 0.02])
    q = np.array([0.8, 0.3, -0.4, 0.2])
    q = q / np.linalg.norm(q)
    out = oracle.project_gaussian(cam, mu, s, q)
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: scalar last
    Sig = Rq @ np.diag(s ** 2) @ Rq.T
    rs = np.random.default_rng(1)
    X = rs.multivariate_normal(mu, Sig, 400_000)
    u = cam.fx * X[:, 0] / X[:, 2] + cam.cx
    v = cam.fy * X[:, 1] / X[:, 2] + cam.cy
    emp = np.cov(np.stack([u, v]))
    ewa = np.array([[out[2] - 0.3, out[3]], [out[3], out[4] - 0.3]])
    assert np.allclose(emp, ewa, rtol=2e-2, atol=2e-2 * np.abs(ewa).max())
    assert abs(out[0] - (cam.fx * mu[0] / mu[2] + cam.cx)) < 1e-9
    # conic is the inverse of the dilated covariance
    Cm = np.array([[out[5], out[6]], [out[6], out[7]]])
    Sm = np.array([[out[2], out[3]], [out[3], out[4]]])
    assert np.allclose(Cm @ Sm, np.eye(2), atol=1e-12)


def test_quaternion_convention_and_covariance():
    """R(q) matches scipy for (w, x, y, z), is orthonormal; Sigma is symmetric PSD."""
    rs = np.random.default_rng(2)
    for _ in range(100):
        q = rs.normal(size=4)
        q /= np.linalg.norm(q)
        R = oracle.quat_to_rot(q)
        Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.abs(R - Rs).max() < 1e-12
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-12
        assert abs(np.linalg.det(R) - 1) < 1e-12
        s = rs.uniform(0.01, 1, 3)
        Sig = R @ np.diag(s ** 2) @ R.T
        assert np.allclose(Sig, Sig.T, atol=1e-15)
        assert np.linalg.eigvalsh(Sig).min() > 0


# ---------------------------------------------------------------- derivation (Eq. 3)
def test_mlp_matches_numpy(tiny):
    """Raw head outputs equal numpy matmuls of [f, d] through the three
    Linear-ReLU-Linear heads; activations match scipy/numpy functions."""
    m, cam = tiny
    ids = np.arange(0, m.n, 7, dtype=np.uint32)
    p = oracle.camera_center(cam)
    attrs, kept, raw = oracle.derive(m, p, ids, want_raw=True)
    d = m.pos[ids].astype(np.float64) - p[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = np.concatenate([m.feat[ids].astype(np.float64), d], axis=1)
    outs = []
    for h in range(3):
        hid = np.maximum(x @ m.W1[h].astype(np.float64) + m.b1[h], 0.0)
        outs.append(hid @ m.W2[h].astype(np.float64) + m.b2[h])
    ref = np.concatenate(outs, axis=1)
    assert np.abs(raw - ref).max() < 1e-12
    k = m.k
    zo, zc, zv = outs
    assert np.abs(attrs[..., 0] - np.tanh(zo)).max() < 1e-14
    assert np.array_equal(kept, (zo > 0).astype(np.uint8))
    assert np.abs(attrs[..., 1:4] - expit(zc.reshape(-1, k, 3))).max() < 1e-14
    zv = zv.reshape(-1, k, 7)
    s = m.scale[ids].astype(np.float64)[:, None, None] * expit(zv[..., 0:3])
    assert np.abs(attrs[..., 4:7] - s).max() < 1e-14
    qq = zv[..., 3:7] / np.linalg.norm(zv[..., 3:7], axis=-1, keepdims=True)
    assert np.abs(attrs[..., 7:11] - qq).max() < 1e-14


# ---------------------------------------------------------------- culling
def test_cull_matches_fp64_geometry():
    """Frustum (1.3 guard band, near plane) + distance LOD: the pinned float32
    decision equals the float64 predicate except within rounding of a boundary."""
    m = gen.city_scene(n=200_000, seed=3)
    cam = gen.stereo_frames(gen.city_path(n_frames=3, seed=4, start=(-50.0, -80.0), h0=20.0, h1=30.0))[1][0]
    ids = oracle.cull(m, cam)
    assert np.all(np.diff(ids.astype(np.int64)) > 0)
    X = m.pos.astype(np.float64)
    c = X @ cam.R.astype(np.float64).T + cam.t.astype(np.float64)
    tx = (cam.width / 2) / cam.fx
    ty = (cam.height / 2) / cam.fy
    fr = (c[:, 2] > cam.znear) & (np.abs(c[:, 0]) <= 1.3 * tx * c[:, 2]) & (np.abs(c[:, 1]) <= 1.3 * ty * c[:, 2])
    p = oracle.camera_center(cam)
    d = np.linalg.norm(X - p, axis=1)
    lvl = m.level.astype(np.int64)
    thr = m.lod_dmax * 2.0 ** (-lvl)
    lod = (lvl == 0) | (d <= thr)
    ref = fr & lod
    got = np.zeros(m.n, bool)
    got[ids] = True
    diff = np.nonzero(got != ref)[0]
    # each disagreement must sit on a boundary within float32 rounding
    for a in diff:
        marg = min(abs(c[a, 2] - cam.znear), abs(abs(c[a, 0]) - 1.3 * tx * c[a, 2]),
                   abs(abs(c[a, 1]) - 1.3 * ty * c[a, 2]), abs(d[a] - thr[a]))
        assert marg < 1e-3 * max(1.0, d[a])
    assert got.sum() > 1000
    # every LOD level above 0 is cut at its own distance
    for l in range(1, m.n_levels):
        sel = ids[m.level[ids] == l]
        assert np.all(d[sel] <= thr[sel] * (1 + 1e-6))


# ---------------------------------------------------------------- unified camera (Eq. 5-6)
def test_unified_camera_closed_form():
    """Parallel eyes: d_u = d, p_u = midpoint - d b / (2 tan(theta/2)), and each
    eye's centre lies on the unified camera's (unguarded) side plane."""
    poses = gen.city_path(n_frames=5, seed=9)
    for pose in poses:
        L, R = gen.stereo_pair(gen.look_rotation(pose.yaw, pose.pitch), pose.pos, 1920, 1080, 60.0)
        U = oracle.unified_camera(L, R)
        pL, pR = oracle.camera_center(L), oracle.camera_center(R)
        pU = oracle.camera_center(U)
        d = L.R[2].astype(np.float64)
        b = np.linalg.norm(pL - pR)
        tan_half = np.tan(np.deg2rad(30.0))
        exp = (pL + pR) / 2 - d * b / (2 * tan_half)
        assert np.abs(pU - exp).max() < 1e-4 * max(1, np.abs(exp).max())
        assert np.abs(U.R.astype(np.float64) - L.R.astype(np.float64)).max() < 1e-6
        for pe in (pL, pR):
            cpos = U.R.astype(np.float64) @ pe + U.t.astype(np.float64)
            assert abs(abs(cpos[0]) / cpos[2] - tan_half) < 1e-3


def test_unified_camera_contains_both_eyes():
    """With LOD off the unified camera's visible set contains both eyes' sets."""
    m = gen.city_scene(n=300_000, seed=5, n_levels=1)
    poses = gen.city_path(n_frames=40, seed=6, start=(-100.0, 50.0), h0=3.0, h1=120.0)
    for pose in poses[::8]:
        L, R = gen.stereo_pair(gen.look_rotation(pose.yaw, pose.pitch), pose.pos, 1920, 1080, 60.0)
        U = oracle.unified_camera(L, R)
        a = set(oracle.cull(m, L).tolist()) | set(oracle.cull(m, R).tolist())
        u = set(oracle.cull(m, U).tolist())
        assert a <= u
        assert len(u) < 1.2 * len(a)


def test_exact_stereo_sets_are_the_eyes_own():
    """The exact stereo form's filtering: the union of the eyes' sets, each
    eye recovering exactly its own set from the mask (city scene with LOD)."""
    m = gen.city_scene(n=300_000, seed=5)
    poses = gen.city_path(n_frames=40, seed=6, start=(-100.0, 50.0), h0=3.0, h1=120.0)
    for pose in poses[::13]:
        L, R = gen.stereo_pair(gen.look_rotation(pose.yaw, pose.pitch), pose.pos, 1920, 1080, 60.0)
        ids, eyes = oracle.cull_pair(m, L, R)
        a, b = oracle.cull(m, L), oracle.cull(m, R)
        assert np.all(np.diff(ids.astype(np.int64)) > 0)
        assert np.array_equal(ids[(eyes & 1) != 0], a) and np.array_equal(ids[(eyes & 2) != 0], b)
        assert np.all(eyes != 0) and len(ids) == len(np.union1d(a, b))


def test_exact_stereo_form_equals_per_eye_for_a_view_independent_model():
    """If the MLPs ignore the view direction (its W1 rows zero), deriving once
    from the unified camera changes nothing, so the exact stereo form must
    give the plain per-eye image bit for bit.  On the same frames the paper's
    enclosing unified frustum does not (it admits anchors an eye's own filter
    drops), nor does drawing the whole union in each eye."""
    m = gen.city_scene(n=300_000, seed=5)
    for h in range(3):
        m.W1[h][32:35, :] = 0.0
    poses = gen.city_path(n_frames=40, seed=6, start=(-100.0, 50.0), h0=3.0, h1=120.0)
    union_differs = enclosing_differs = 0
    for pose in (poses[15], poses[18]):
        L, R = gen.stereo_pair(gen.look_rotation(pose.yaw, pose.pitch), pose.pos, 480, 270, 60.0)
        U = oracle.unified_camera(L, R)
        ids, _ = oracle.cull_pair(m, L, R)
        attrs, kept = oracle.derive(m, oracle.camera_center(U), ids)
        gid = (ids.astype(np.int64)[:, None] * m.k + np.arange(m.k)[None, :]).reshape(-1)
        for cam in (L, R):
            (plain, T0, _, _), _ = oracle.render_view(m, cam)
            vr = oracle.view_gaussians(m, cam, derive_cam=U, pair=(L, R))
            exact, T1, _, _ = oracle.render(vr.rec, vr.depth32, vr.gid, cam.width, cam.height)
            assert np.array_equal(exact, plain) and np.array_equal(T0, T1)
            rec, d32 = oracle.project_records(m, cam, ids, attrs, kept)  # the whole union in this eye
            union_differs += not np.array_equal(oracle.render(rec, d32, gid, cam.width, cam.height)[0], plain)
            ve = oracle.view_gaussians(m, cam, derive_cam=U)  # Eq. 6's enclosing frustum
            enclosing_differs += not np.array_equal(oracle.render(ve.rec, ve.depth32, ve.gid, cam.width,
                                                                  cam.height)[0], plain)
    assert union_differs >= 2 and enclosing_differs >= 3


# ---------------------------------------------------------------- exact tile coverage
def test_tile_coverage_exact_vs_dense_sampling():
    """A tile is listed iff the hull of its pixel centres meets the ellipse
    q <= tau: listed tiles have a sample point (nearly) inside, unlisted
    tiles have none, and every pixel with alpha >= 1/255 is in a listed tile."""
    rs = np.random.default_rng(4)
    W, H, T = 160, 128, 16
    ntx = W // T
    for trial in range(60):
        mx, my = rs.uniform(-20, W + 20), rs.uniform(-20, H + 20)
        sx, sy = np.exp(rs.uniform(np.log(0.5), np.log(40), 2))
        th = rs.uniform(0, np.pi)
        Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        S = Rm @ np.diag([sx * sx, sy * sy]) @ Rm.T + 0.3 * np.eye(2)
        Ci = np.linalg.inv(S)
        A, B, Cc = Ci[0, 0], Ci[0, 1], Ci[1, 1]
        o = rs.uniform(0.01, 0.99)
        tau = 2 * np.log(255 * o)
        tiles = set(oracle.cover_tiles64(mx, my, A, B, Cc, tau, W, H, T, T).tolist())
        g = np.linspace(0.5, T - 0.5, 61)
        for ty in range(H // T):
            for tx in range(ntx):
                X = tx * T + g[None, :] - mx
                Y = ty * T + g[:, None] - my
                q = A * X * X + 2 * B * X * Y + Cc * Y * Y
                qmin = q.min()
                t = ty * ntx + tx
                if t in tiles:
                    assert qmin <= tau * 1.02 + 0.05, (trial, t, qmin, tau)
                else:
                    assert qmin > tau
        # pixel-level: alpha >= 1/255 implies the tile is listed
        X = np.arange(W) + 0.5 - mx
        Y = np.arange(H) + 0.5 - my
        q = A * X[None, :] ** 2 + 2 * B * X[None, :] * Y[:, None] + Cc * Y[:, None] ** 2
        ys, xs = np.nonzero(o * np.exp(-0.5 * q) >= 1 / 255)
        for x, y in zip(xs, ys):
            assert (y // T) * ntx + x // T in tiles


def test_keygen_f32_agrees_with_fp64_coverage(tiny):
    m, cam = tiny
    vr = oracle.view_gaussians(m, cam)
    r = vr.rec
    valid = r[:, 0] > 0
    tau = r[:, 11] * (1 + 2 ** -10) + 2 ** -10
    counts, keys, vals = oracle.keygen_f32(r[:, 1], r[:, 2], r[:, 3], r[:, 4], r[:, 5], tau,
                                           np.zeros(len(r)), valid, cam.width, cam.height)
    n64 = np.array([len(oracle.cover_tiles64(*r[i, 1:6], tau[i], cam.width, cam.height)) if valid[i] else 0
                    for i in range(len(r))])
    assert np.mean(counts == n64) > 0.995
    assert np.all(np.diff(vals.astype(np.int64)) >= 0)


# ---------------------------------------------------------------- number formats
def test_bf16_rounding_matches_torch():
    import torch
    rs = np.random.default_rng(5)
    x = np.concatenate([rs.normal(0, 3, 20000), rs.normal(0, 1e-30, 200),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8)])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.round_bf16(v) for v in x], np.float32)
    assert np.array_equal(got, ref)


def test_e4m3_rounding_matches_torch():
    import torch
    rs = np.random.default_rng(6)
    x = np.concatenate([rs.normal(0, 50, 20000), rs.normal(0, 0.01, 2000),
                        np.array([0.0, 2 ** -9, 3 * 2 ** -10, 448.0, -448.0, 1.0625, 1.1875])])
    x = np.clip(x, -448, 448).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    got = np.array([oracle.round_e4m3(float(v)) for v in x], np.float32)
    assert np.array_equal(got, ref)
    # reading: values beyond the largest finite e4m3 saturate to +-448
    assert oracle.round_e4m3(1e4) == 448.0 and oracle.round_e4m3(-900.0) == -448.0


def test_fp8_scales_are_tight_powers_of_two_and_bound_the_hidden_layer():
    """FP8 form: every scale a power of two with amax / s in (224, 448]; the
    hidden-activation scale bounds every anchor's hidden layer for any view
    direction (checked on all tiny-scene anchors x random directions)."""
    m = gen.tiny_scene()
    q = oracle.fp8_scales(m)
    assert q.mode == 2

    def tight(s, amax):
        assert np.log2(s) == np.round(np.log2(s))
        assert 224.0 < amax / s <= 448.0

    tight(q.s_x, max(np.abs(m.feat).max(), 1.0))
    rs = np.random.default_rng(0)
    d = rs.standard_normal((m.n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = np.concatenate([m.feat.astype(np.float64), d], axis=1)
    for h in range(3):
        tight(q.s_w1[h], np.abs(m.W1[h]).max())
        tight(q.s_w2[h], np.abs(m.W2[h]).max())
        hid = np.maximum(x @ m.W1[h].astype(np.float64) + m.b1[h], 0.0)
        assert hid.max() <= 448.0 * q.s_h[h]
    assert oracle.pow2_ceil(1.0) == 1.0 and oracle.pow2_ceil(1.5) == 2.0 and oracle.pow2_ceil(0.25) == 0.25
    assert oracle.pow2_ceil(3e-5) == 2.0 ** -15


def test_e4m3_two_term_expansion():
    """The FP8 form's two-term expansion: both terms are E4M3 numbers at the
    scale (torch's float8 cast returns them unchanged), the leading term is
    the one-term rounding, and the sum is within 2^-7 relative of the value
    over the normal range (the second term rounds the first's error, itself
    within 2^-4 relative, to 3 mantissa bits)."""
    import torch
    rs = np.random.default_rng(5)
    s = 2.0 ** -6
    for v in np.concatenate([rs.uniform(-1, 1, 2000) * 10.0 ** rs.uniform(-2, 0.8, 2000), [0.0, 7.0, -0.3]]):
        tot, hi = oracle.e4m3_two_term(v, s)
        lo = tot - hi
        for term in (hi / s, lo / s):
            t = torch.tensor([term], dtype=torch.float64).to(torch.float8_e4m3fn).to(torch.float64).item()
            assert t == term
        assert hi == oracle.round_e4m3(v / s) * s
        if abs(v) / s >= 2.0 ** -6 * 2 ** 4:  # leading term normal, residual not deep subnormal
            assert abs(tot - v) <= 2.0 ** -7 * abs(v)


def test_fp8_form_error_is_the_inputs_rounding(tiny):
    """Two-term weights and hidden activations remove the rounding error
    that one-term E4M3 adds on top of the inputs' own rounding.  Against a
    numpy forward pass with torch's float8 casts: the oracle's mode-2 error
    (RMS over opacity and colour, against float64) is close to the error of
    rounding the inputs alone and well below rounding everything once."""
    import torch
    m, cam = tiny
    ids = oracle.cull(m, cam)[:600]
    pc = oracle.camera_center(cam)
    q = oracle.fp8_scales(m)
    a64, _ = oracle.derive(m, pc, ids)
    a8, _ = oracle.derive(m, pc, ids, q)

    def e4(v, sc):
        t = torch.from_numpy(np.asarray(v / sc, np.float64)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
        return t * sc

    d = m.pos[ids].astype(np.float64) - pc
    x = np.concatenate([m.feat[ids].astype(np.float64), d / np.linalg.norm(d, axis=1, keepdims=True)], axis=1)

    def attrs(round_x, round_rest):
        z = []
        for h in range(3):
            W1, W2 = m.W1[h].astype(np.float64), m.W2[h].astype(np.float64)
            xx = e4(x, q.s_x) if round_x else x
            w1 = e4(W1, q.s_w1[h]) if round_rest else W1
            w2 = e4(W2, q.s_w2[h]) if round_rest else W2
            hid = np.maximum(xx @ w1 + m.b1[h], 0.0)
            hid = e4(hid, q.s_h[h]) if round_rest else hid
            z.append(hid @ w2 + m.b2[h])
        z = np.concatenate(z, axis=1)
        k = m.k
        return np.concatenate([np.tanh(z[:, :k])[..., None], (1 / (1 + np.exp(-z[:, k:4 * k]))).reshape(-1, k, 3)], -1)

    rms = lambda a: float(np.sqrt(np.mean((a - a64[..., :4]) ** 2)))
    e_inputs, e_once, e_form = rms(attrs(True, False)), rms(attrs(True, True)), rms(a8[..., :4])
    assert rms(attrs(False, False)) < 1e-12
    assert e_form <= 1.3 * e_inputs and e_form <= 0.75 * e_once, (e_inputs, e_once, e_form)


def test_e4m3_rounding_closed_forms():
    """E4M3: 3 mantissa bits, bias 7, subnormal spacing 2^-9, largest finite 448, saturating."""
    cases = {1.0: 1.0, 1.0625: 1.0, 1.1875: 1.25, 1.125: 1.125, 448.0: 448.0, 460.0: 448.0, 1e6: 448.0,
             2.0 ** -9: 2.0 ** -9, 1.4 * 2.0 ** -10: 2.0 ** -9, 0.4 * 2.0 ** -9: 0.0, -3.3: -3.25,
             2.0 ** -6 * 1.0625: 2.0 ** -6, 0.01: 0.009765625}
    for x, want in cases.items():
        assert oracle.round_e4m3(x) == want, (x, oracle.round_e4m3(x), want)


# ---------------------------------------------------------------- walk length
def stacked_records(n, opacity, mx, my, sigma=2.0):
    """n identical isotropic Gaussians at (mx, my), depths 1..n (front to back)."""
    rec = np.zeros((n, 16))
    A = 1.0 / sigma ** 2
    tau = 2 * np.log(255 * opacity)
    for i in range(n):
        rec[i, :12] = [1, mx, my, A, 0, A, opacity, 0.5, 0.5, 0.5, 1.0 + i, tau]
    return rec, np.arange(1, n + 1, dtype=np.float32), np.arange(n, dtype=np.int64)


def test_walk_length_closed_form():
    """At the common centre alpha = o exactly: T after k Gaussians is (1-o)^k,
    so with o = 0.95 the 4th Gaussian would bring T to 6.25e-6 < 1e-4 and the
    pixel stops there (walk 4, 3 contributors); with o = 0.5 T = 2^-k stays
    above 1e-4 up to k = 13 and the pixel stops at the 14th; a pixel of a tile
    the Gaussians do not cover walks nothing; far from the centre (alpha <
    1/255 for all) a pixel of a covered tile walks the whole list."""
    W, H = 64, 32
    for o, want_walk, want_nc in [(0.95, 4, 3), (0.5, 14, 13)]:
        rec, d32, gid = stacked_records(20, o, 8.5, 8.5)
        px = np.array([8, 60, 15])
        py = np.array([8, 30, 0])
        rgb, T, mg, nc, wk = oracle.render(rec, d32, gid, W, H, True, px, py, walk=True)
        assert wk[0] == want_walk and nc[0] == want_nc
        assert np.isclose(T[0], (1 - o) ** want_nc)
        assert wk[1] == 0 and nc[1] == 0 and T[1] == 1.0   # tile (3, 1): not covered
        a15 = o * np.exp(-0.5 * (6.5 ** 2 + 8.0 ** 2) / 4.0)  # pixel (15, 0), same tile as the centre
        assert a15 < 1 / 255 and wk[2] == 20 and nc[2] == 0
    # brute-force form (one list for every pixel) walks the same way at the centre
    rec, d32, gid = stacked_records(20, 0.95, 8.5, 8.5)
    _, _, _, _, wk = oracle.render(rec, d32, gid, W, H, False, np.array([8, 60]), np.array([8, 30]), walk=True)
    assert wk[0] == 4 and wk[1] == 20
