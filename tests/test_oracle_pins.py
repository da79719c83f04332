"""Pins of the FP64 oracle against things other than itself.

Every oracle function is checked against one of: a closed form written from
the definitions (Sec. 3 Eq. 1-2, Sec. 3.1), a library routine (scipy's complex
spherical harmonics, numpy's lexsort), a brute-force all-pairs blender, the
paper's printed bound (merged d=2 offsets vs full render above 70 dB, Sec. 3.1),
invariants of alpha blending, or central finite differences of the oracle's
own forward pass (for the analytic backward). A plausible slip anywhere (a
dropped term, a wrong sign or index, a transposed operand) fails one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from brute_force import blend_all_pairs
from paper_2412_13547_b300 import scenes

SQRT_PI = math.sqrt(math.pi)


def ident_cam(w=64, h=48, f=50.0, cx=None, cy=None):
    return orc.Camera(R=np.eye(3), T=np.zeros(3), fx=f, fy=f,
                      cx=(w - 1) / 2 if cx is None else cx, cy=(h - 1) / 2 if cy is None else cy,
                      width=w, height=h, z_near=0.2)


def gauss(means, log_scales, quats=None, logits=None, sh=None, deg=0):
    means = np.atleast_2d(np.asarray(means, np.float64))
    n = means.shape[0]
    return dict(
        means=means,
        log_scales=np.broadcast_to(np.asarray(log_scales, np.float64), (n, 3)).copy(),
        quats=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quats is None else np.atleast_2d(quats).astype(np.float64),
        opacity_logits=np.zeros(n) if logits is None else np.asarray(logits, np.float64).reshape(n),
        sh=np.zeros((n, (deg + 1) ** 2, 3)) if sh is None else np.asarray(sh, np.float64))


def dc_for_colour(c):
    """DC coefficient giving colour c at degree 0 (Y_00 = 1/(2 sqrt(pi)))."""
    return (np.asarray(c, np.float64) - 0.5) * 2.0 * SQRT_PI


# ---------------------------------------------------------------------------
# Spherical harmonics vs scipy (library routine)
# ---------------------------------------------------------------------------

def test_sh_basis_matches_scipy_real_harmonics():
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        got = orc.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                ylm = sph_harm_y(l, abs(m), theta, phi)  # complex, Condon-Shortley phase
                if m == 0:
                    ref = ylm.real
                elif m > 0:
                    ref = math.sqrt(2.0) * ylm.real
                else:
                    ref = math.sqrt(2.0) * ylm.imag
                assert got[l * l + l + m] == pytest.approx(ref, abs=1e-12), (l, m)


def test_sh_degree0_colour_and_sigmoid():
    c = np.array([[0.2, 0.7, 1.0]])
    p = gauss([[0.0, 0.0, 3.0]], -2.0, logits=[0.0], sh=dc_for_colour(c)[:, None, :])
    pr = orc.project(p, ident_cam(), orc.Dilation())
    np.testing.assert_allclose(pr["rgb"], c, atol=1e-14)
    assert pr["opacity"][0] == pytest.approx(0.5, abs=1e-15)
    p["opacity_logits"][:] = math.log(3.0)  # sigmoid = 3/4
    assert orc.project(p, ident_cam(), orc.Dilation())["opacity"][0] == pytest.approx(0.75, abs=1e-15)
    # negative colour is clamped to 0
    p["sh"][0, 0] = dc_for_colour([-0.3, 0.5, 0.5])
    assert orc.project(p, ident_cam(), orc.Dilation())["rgb"][0, 0] == 0.0


# ---------------------------------------------------------------------------
# EWA projection closed forms (Sec. 3.1)
# ---------------------------------------------------------------------------

def closed_radius(a, b, c):
    mid = 0.5 * (a + c)
    return math.ceil(3.0 * math.sqrt(mid + math.sqrt(max(0.1, mid * mid - (a * c - b * b)))))


def test_projection_isotropic_on_axis():
    f, z, s = 50.0, 3.0, 0.1
    cam = ident_cam(f=f)
    pr = orc.project(gauss([[0.0, 0.0, z]], math.log(s)), cam, orc.Dilation())
    var = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0.0, var], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pr["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pr["xy"][0], [cam.cx, cam.cy], atol=1e-12)
    assert pr["depth"][0] == z
    assert pr["radius"][0] == closed_radius(var, 0.0, var)


def test_projection_isotropic_off_axis():
    f, x, z, s = 50.0, 0.6, 2.5, 0.07
    cam = ident_cam(f=f)
    pr = orc.project(gauss([[x, 0.0, z]], math.log(s)), cam, orc.Dilation())
    # J = [[f/z, 0, -f x/z^2], [0, f/z, 0]], Sigma' = s^2 J J^T + 0.3 I
    a = s * s * (f * f / z ** 2 + f * f * x * x / z ** 4) + 0.3
    c = s * s * f * f / z ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [a, 0.0, c], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(pr["xy"][0], [f * x / z + cam.cx, cam.cy], atol=1e-12)


def test_projection_axis_aligned_anisotropic():
    f, z = 40.0, 2.0
    sx, sy, sz = 0.05, 0.2, 0.4
    pr = orc.project(gauss([[0.0, 0.0, z]], np.log([sx, sy, sz])), ident_cam(f=f), orc.Dilation())
    np.testing.assert_allclose(pr["cov2d"][0], [(f * sx / z) ** 2 + 0.3, 0.0, (f * sy / z) ** 2 + 0.3],
                               rtol=1e-13, atol=1e-14)
    # a quarter turn about the view axis swaps the image axes: q = (cos 45, 0, 0, sin 45)
    q = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    pr = orc.project(gauss([[0.0, 0.0, z]], np.log([sx, sy, sz]), quats=[q]), ident_cam(f=f), orc.Dilation())
    np.testing.assert_allclose(pr["cov2d"][0], [(f * sy / z) ** 2 + 0.3, 0.0, (f * sx / z) ** 2 + 0.3],
                               rtol=1e-12, atol=1e-12)


def test_projection_rotation_invariance_of_isotropic():
    rng = np.random.default_rng(1)
    base = orc.project(gauss([[0.1, -0.2, 3.0]], math.log(0.08)), ident_cam(), orc.Dilation())
    for _ in range(5):
        q = rng.standard_normal(4) * rng.uniform(0.3, 3.0)  # unnormalised
        pr = orc.project(gauss([[0.1, -0.2, 3.0]], math.log(0.08), quats=[q]), ident_cam(), orc.Dilation())
        np.testing.assert_allclose(pr["cov2d"], base["cov2d"], rtol=1e-12, atol=1e-13)


def test_projection_rigid_motion_invariance():
    """Rotating/translating scene and camera together leaves the image unchanged.
    Catches a transposed camera rotation or a wrong camera centre."""
    rng = np.random.default_rng(2)
    scene = scenes.small_scene(50, index=7, sh_degree=3, log_scale_mean=-2.0)
    p = {k: np.asarray(v, np.float64) for k, v in scene.as_dict().items()}
    cam = orc.as_camera(scenes.look_at(scenes.orbit_eye(4.0, 10.0, 30.0), width=96, height=64))
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = q * np.sign(np.diag(r))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    tr = rng.standard_normal(3)
    # move the world by x -> Q x + tr; camera R' = R Q^T, T' = T - R Q^T tr
    p2 = dict(p)
    p2["means"] = p["means"] @ Q.T + tr
    # compose the Gaussian orientation with Q via the rotation matrix -> quaternion
    def rot_to_quat(M):
        w = math.sqrt(max(0.0, 1 + M[0, 0] + M[1, 1] + M[2, 2])) / 2
        x = math.copysign(math.sqrt(max(0.0, 1 + M[0, 0] - M[1, 1] - M[2, 2])) / 2, M[2, 1] - M[1, 2])
        y = math.copysign(math.sqrt(max(0.0, 1 - M[0, 0] + M[1, 1] - M[2, 2])) / 2, M[0, 2] - M[2, 0])
        z = math.copysign(math.sqrt(max(0.0, 1 - M[0, 0] - M[1, 1] + M[2, 2])) / 2, M[1, 0] - M[0, 1])
        return np.array([w, x, y, z])
    qQ = rot_to_quat(Q)
    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    p2["quats"] = np.stack([qmul(qQ, qi) for qi in p["quats"]])
    cam2 = orc.Camera(R=cam.R @ Q.T, T=cam.T - cam.R @ Q.T @ tr, fx=cam.fx, fy=cam.fy, cx=cam.cx, cy=cam.cy,
                      width=cam.width, height=cam.height)
    # SH colour is a function of the world direction: rotate the test by using degree-0 only
    p["sh"][:, 1:] = 0.0
    p2["sh"] = p["sh"]
    a = orc.project(p, cam, orc.Dilation())
    b = orc.project(p2, cam2, orc.Dilation())
    for k in ("xy", "conic", "cov2d", "depth", "rgb", "opacity"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-9, atol=1e-9, err_msg=k)


def test_projection_near_plane_cull():
    pr = orc.project(gauss([[0.0, 0.0, 0.1], [0.0, 0.0, -1.0], [0.0, 0.0, 1.0]], -2.0), ident_cam(),
                     orc.Dilation())
    assert list(pr["radius"]) [:2] == [0, 0] and pr["radius"][2] > 0
    assert list(pr["tiles_touched"][:2]) == [0, 0]
    assert pr["flags"][0] & orc.FLAG_CULLED and pr["flags"][1] & orc.FLAG_CULLED


def test_rect_rule_brute_force():
    """Tile tx is touched iff [p_ds - r/d, p_ds + r/d] meets [tile*tx, tile*tx + tile),
    with the lattice-aligned centre (p - o)/d, clipped to the grid."""
    rng = np.random.default_rng(3)
    cam = ident_cam(w=150, h=90, f=60.0)
    n = 300
    p = gauss(np.c_[rng.uniform(-2, 2, n), rng.uniform(-1.5, 1.5, n), rng.uniform(1.0, 4.0, n)],
              rng.normal(-2.5, 0.6, (n, 3)), quats=rng.standard_normal((n, 4)))
    for d, ox, oy, tile in [(1, 0, 0, 16), (2, 1, 0, 16), (3, 2, 1, 8), (4, 3, 3, 16)]:
        dil = orc.Dilation(d, ox, oy, 0, tile)
        pr = orc.project(p, cam, dil)
        w_ds, h_ds, tx_n, ty_n = orc.grid(cam, dil)
        assert w_ds == -(-(150 - ox) // d) and h_ds == -(-(90 - oy) // d)
        for g in range(n):
            if pr["flags"][g] & (orc.FLAG_RECT | orc.FLAG_NEAR):
                continue
            cx = (pr["xy"][g, 0] - ox) / d
            cy = (pr["xy"][g, 1] - oy) / d
            r = pr["radius"][g] / d
            xs = [t for t in range(tx_n) if cx + r >= tile * t and cx - r < tile * (t + 1)]
            ys = [t for t in range(ty_n) if cy + r >= tile * t and cy - r < tile * (t + 1)]
            if not xs or not ys or pr["depth"][g] <= 0.2:
                assert pr["tiles_touched"][g] == 0
                continue
            assert list(pr["rect"][g]) == [xs[0], ys[0], xs[-1], ys[-1]], g
            assert pr["tiles_touched"][g] == len(xs) * len(ys)


# ---------------------------------------------------------------------------
# Binning vs numpy lexsort
# ---------------------------------------------------------------------------

def test_binning_matches_lexsort():
    rng = np.random.default_rng(4)
    n, tx, ty = 200, 7, 5
    x0 = rng.integers(0, tx, n)
    y0 = rng.integers(0, ty, n)
    x1 = np.minimum(tx - 1, x0 + rng.integers(0, 3, n))
    y1 = np.minimum(ty - 1, y0 + rng.integers(0, 3, n))
    rect = np.c_[x0, y0, x1, y1].astype(np.int32)
    culled = rng.uniform(size=n) < 0.1
    rect[culled] = [0, 0, -1, -1]
    tt = np.where(culled, 0, (x1 - x0 + 1) * (y1 - y0 + 1)).astype(np.int64)
    # depths with deliberate exact ties
    depth = rng.choice(rng.uniform(0.5, 5.0, 40), n).astype(np.float32)
    dbits = depth.view(np.uint32)
    keys, vals, ranges = orc.bin_sort(rect, tt, dbits, tx, ty)
    tiles, dks, ids = [], [], []
    for g in range(n):
        if tt[g] == 0:
            continue
        for yy in range(rect[g, 1], rect[g, 3] + 1):
            for xx in range(rect[g, 0], rect[g, 2] + 1):
                tiles.append(yy * tx + xx)
                dks.append(int(dbits[g]))
                ids.append(g)
    tiles, dks, ids = map(np.array, (tiles, dks, ids))
    order = np.lexsort((ids, dks, tiles))
    assert len(keys) == tt.sum()
    np.testing.assert_array_equal(vals, ids[order])
    np.testing.assert_array_equal(keys, (tiles[order].astype(np.uint64) << np.uint64(32)) | dks[order].astype(np.uint64))
    for t in range(tx * ty):
        sel = np.nonzero(tiles[order] == t)[0]
        if len(sel):
            assert tuple(ranges[t]) == (sel[0], sel[-1] + 1)
        else:
            assert ranges[t, 0] == ranges[t, 1]
    # the subset binning gives the same per-tile lists
    sub = np.array([0, 3, 11, 34], np.int32)
    sv, sr = orc.bin_tiles(rect, dbits, tx, sub)
    for k, t in enumerate(sub):
        np.testing.assert_array_equal(sv[sr[k, 0]:sr[k, 1]], vals[ranges[t, 0]:ranges[t, 1]])


# ---------------------------------------------------------------------------
# Alpha blending closed forms, brute force and invariants (Eq. 2)
# ---------------------------------------------------------------------------

def render_full(p, cam, dil, bg=(0.0, 0.0, 0.0)):
    pr = orc.project(p, cam, dil)
    w_ds, h_ds, tx, ty = orc.grid(cam, dil)
    keys, vals, ranges = orc.bin_sort(pr["rect"], pr["tiles_touched"], orc.depth_bits(pr["depth"]), tx, ty)
    return pr, vals, ranges, orc.render_fwd(pr, vals, ranges, cam, dil, bg)


def test_single_gaussian_closed_form():
    f, z, s, o = 50.0, 3.0, 0.15, 0.8
    cam = ident_cam(w=48, h=40, f=f)
    col = np.array([0.9, 0.3, 0.6])
    bg = np.array([0.1, 0.2, 0.3])
    p = gauss([[0.0, 0.0, z]], math.log(s), logits=[math.log(o / (1 - o))], sh=dc_for_colour(col)[None, None, :])
    pr, vals, ranges, out = render_full(p, cam, orc.Dilation(), bg)
    var = (f * s / z) ** 2 + 0.3
    r = closed_radius(var, 0, var)
    ys, xs = np.mgrid[0:40, 0:48]
    dx, dy = xs - cam.cx, ys - cam.cy
    alpha = np.minimum(0.99, o * np.exp(-0.5 * (dx * dx + dy * dy) / var))
    # tile gate: pixel's 16x16 tile must meet [p - r, p + r] in both axes
    tx, ty = xs // 16, ys // 16
    inside = ((tx * 16 <= cam.cx + r) & (tx * 16 + 16 > cam.cx - r) &
              (ty * 16 <= cam.cy + r) & (ty * 16 + 16 > cam.cy - r))
    alpha = np.where(inside & (alpha >= 1 / 255), alpha, 0.0)
    ref = alpha[..., None] * col + (1 - alpha)[..., None] * bg
    np.testing.assert_allclose(out["img"], ref, atol=1e-14)
    np.testing.assert_allclose(out["t_final"], 1 - alpha, atol=1e-14)
    assert set(np.unique(out["last"])) <= {0, 1}


def test_two_gaussian_compositing_order():
    cam = ident_cam(w=32, h=32, f=40.0, cx=16.0, cy=16.0)
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    o1, o2 = 0.6, 0.7
    sh = np.stack([dc_for_colour(c1), dc_for_colour(c2)])[:, None, :]
    # far Gaussian listed first: order must come from depth, not index
    p = gauss([[0.0, 0.0, 4.0], [0.0, 0.0, 2.0]], [[math.log(0.2 * 2)] * 3, [math.log(0.2)] * 3],
              logits=[math.log(o1 / (1 - o1)), math.log(o2 / (1 - o2))], sh=sh[::-1].copy())
    pr, vals, ranges, out = render_full(p, cam, orc.Dilation())
    # at the common centre pixel both have G = 1: near (index 1, colour c1) first
    C = out["img"][16, 16]
    a_near, a_far = o2, o1
    ref = c1 * a_near + c2 * a_far * (1 - a_near)
    np.testing.assert_allclose(C, ref, atol=1e-14)
    assert out["last"][16, 16] == 2


def test_early_stop_and_skip_rules():
    cam = ident_cam(w=32, h=32, f=40.0, cx=16.0, cy=16.0)
    o = 0.95
    n = 5
    p = gauss(np.c_[np.zeros(n), np.zeros(n), 2.0 + 0.5 * np.arange(n)], math.log(0.05),
              logits=np.full(n, math.log(o / (1 - o))), sh=np.tile(dc_for_colour([1.0, 1.0, 1.0]), (n, 1, 1)))
    bg = (0.25, 0.25, 0.25)
    pr, vals, ranges, out = render_full(p, cam, orc.Dilation(), bg)
    # T: 1, .05, .0025, 1.25e-4 -> next would be 6.25e-6 < 1e-4: stop after 3
    assert out["last"][16, 16] == 3
    assert out["t_final"][16, 16] == pytest.approx(0.05 ** 3, rel=1e-12)
    assert out["img"][16, 16, 0] == pytest.approx(o * (1 + 0.05 + 0.0025) + 0.05 ** 3 * 0.25, rel=1e-12)
    # alpha just below 1/255 is skipped, just above is blended
    for a, blended in [(1 / 255 * 0.999, False), (1 / 255 * 1.001, True)]:
        p1 = gauss([[0.0, 0.0, 2.0]], math.log(0.05), logits=[math.log(a / (1 - a))],
                   sh=dc_for_colour([1.0, 1.0, 1.0])[None, None, :])
        _, _, _, o1 = render_full(p1, cam, orc.Dilation())
        assert (o1["last"][16, 16] == 1) == blended
        assert (o1["img"][16, 16, 0] > 0) == blended


def _tiny_scene(seed, n, w, h, deg=0, scale=-2.3):
    rng = np.random.default_rng(seed)
    cam = orc.as_camera(scenes.look_at(scenes.orbit_eye(3.0, 40.0 * seed, 25.0), width=w, height=h))
    p = gauss(rng.uniform(-0.6, 0.6, (n, 3)), rng.normal(scale, 0.4, (n, 3)), quats=rng.standard_normal((n, 4)),
              logits=rng.normal(0.5, 1.5, n), sh=np.concatenate(
                  [rng.uniform(-SQRT_PI, SQRT_PI, (n, 1, 3)), rng.normal(0, 0.2, (n, (deg + 1) ** 2 - 1, 3))], 1))
    return p, cam


@pytest.mark.parametrize("d,ox,oy,mode", [(1, 0, 0, 0), (2, 1, 0, 0), (2, 1, 1, 1), (3, 0, 2, 0)])
def test_tiled_blend_equals_brute_force(d, ox, oy, mode):
    for seed in range(3):
        p, cam = _tiny_scene(seed + 10, 8, 64 - 3 * seed, 48 + 5 * seed, deg=1)
        dil = orc.Dilation(d, ox, oy, mode, 16)
        bg = (0.3, 0.1, 0.7)
        pr, vals, ranges, out = render_full(p, cam, dil, bg)
        w_ds, h_ds, _, _ = orc.grid(cam, dil)
        img, tf = blend_all_pairs(pr, w_ds, h_ds, d, ox, oy, 16, bg)
        np.testing.assert_allclose(out["img"], img, atol=1e-13)
        np.testing.assert_allclose(out["t_final"], tf, atol=1e-13)


def test_blend_invariants_white_scene():
    """With white colours and a black background C = sum_i alpha_i T_i = 1 - T_final."""
    scene = scenes.small_scene(400, index=3)
    p = {k: np.asarray(v, np.float64) for k, v in scene.as_dict().items()}
    p["sh"][:] = dc_for_colour([1.0, 1.0, 1.0])
    p["log_scales"] += 1.0
    cam = orc.as_camera(scenes.look_at(scenes.orbit_eye(4.0, 30.0, 20.0), width=80, height=72))
    for dil in [orc.Dilation(), orc.Dilation(2, 1, 1)]:
        _, _, _, out = render_full(p, cam, dil)
        tf = out["t_final"]
        for ch in range(3):
            np.testing.assert_allclose(out["img"][..., ch], 1.0 - tf, atol=1e-12)
        assert tf.max() <= 1.0 and tf.min() >= 1e-4
        assert (out["last"] > 0).mean() > 0.2


# ---------------------------------------------------------------------------
# Dilated rendering (Sec. 3.1)
# ---------------------------------------------------------------------------

def test_dilated_equals_strided_full_when_rect_inside_one_tile():
    cam = ident_cam(w=128, h=128, f=60.0, cx=40.0, cy=40.0)
    col = np.array([0.2, 0.8, 0.4])
    # centred at hr (40, 40); radius ~6 px: inside hr tile (2,2) and ds tile (1,1)
    p = gauss([[0.0, 0.0, 3.0]], math.log(0.08), logits=[1.0], sh=dc_for_colour(col)[None, None, :])
    _, _, _, full = render_full(p, cam, orc.Dilation())
    for ox in range(2):
        for oy in range(2):
            _, _, _, ds = render_full(p, cam, orc.Dilation(2, ox, oy))
            np.testing.assert_allclose(ds["img"], full["img"][oy::2, ox::2], atol=0)


def merged_psnr(p, cam, mode):
    _, _, _, full = render_full(p, cam, orc.Dilation())
    merged = np.zeros_like(full["img"])
    for ox in range(2):
        for oy in range(2):
            _, _, _, ds = render_full(p, cam, orc.Dilation(2, ox, oy, mode))
            merged[oy::2, ox::2] = ds["img"]
    mse = np.mean((merged - full["img"]) ** 2)
    return (np.inf if mse == 0 else 10 * np.log10(1.0 / mse)), merged, full["img"]


def test_merged_offsets_psnr_above_70db():
    """Sec. 3.1: the four d=2 offsets merged into one hr image agree with the full
    render above 70 dB; the residual sits near tile edges (supplementary Fig.)."""
    scene, cam, _ = scenes.workload_small()
    p = {k: np.asarray(v, np.float64) for k, v in scene.as_dict().items()}
    psnr_lat, merged, full = merged_psnr(p, orc.as_camera(cam), 0)
    psnr_lit, _, _ = merged_psnr(p, orc.as_camera(cam), 1)
    assert psnr_lat > 70.0
    assert psnr_lat >= psnr_lit - 1e-9
    err = np.abs(merged - full).max(-1)
    if err.max() > 0:
        ys, xs = np.nonzero(err > 1e-12)
        # the error lies within 2 px of an hr tile boundary (multiple of 16)
        near = np.minimum(xs % 16, 15 - xs % 16) <= 1
        near |= np.minimum(ys % 16, 15 - ys % 16) <= 1
        assert near.mean() >= 0.5


# ---------------------------------------------------------------------------
# Analytic backward vs central finite differences (FP64)
# ---------------------------------------------------------------------------

def _fd_check(p, cam, dil, bg, seed):
    rng = np.random.default_rng(seed)
    pr, vals, ranges, out = render_full(p, cam, dil, bg)
    assert not out["ambiguous"].any()
    w = rng.standard_normal(out["img"].shape)

    def L(q):
        prq = orc.project(q, cam, dil)
        return float(np.sum(w * orc.render_fwd(prq, vals, ranges, cam, dil, bg)["img"]))

    g2d = orc.render_bwd(pr, vals, ranges, cam, dil, w, bg)
    grads = orc.project_bwd(p, cam, dil, g2d)
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        flat = p[name].reshape(-1)
        num = np.zeros_like(flat)
        for e in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[e]))
            qp = {k: v.copy() for k, v in p.items()}
            qm = {k: v.copy() for k, v in p.items()}
            qp[name].reshape(-1)[e] += h
            qm[name].reshape(-1)[e] -= h
            num[e] = (L(qp) - L(qm)) / (2 * h)
        ana = grads[name].reshape(-1)
        scale = max(np.abs(num).max(), 1e-12)
        assert np.abs(ana - num).max() <= 2e-6 * scale + 1e-9, (name, np.abs(ana - num).max(), scale)
    return grads


@pytest.mark.parametrize("d,ox,oy", [(1, 0, 0), (2, 1, 0)])
def test_backward_matches_finite_differences(d, ox, oy):
    p, cam = _tiny_scene(5, 6, 48, 40, deg=3, scale=-2.0)
    _fd_check(p, cam, orc.Dilation(d, ox, oy), (0.2, 0.5, 0.1), seed=d)


def test_backward_finite_differences_clamped_jacobian():
    """One Gaussian beyond the Jacobian clamp (|t_x/t_z| > 1.3 tan(fov/2)) that
    still reaches into the image, one alpha-clamped (o G > 0.99) Gaussian."""
    cam = ident_cam(w=48, h=40, f=40.0)
    lim = 1.3 * 24 / 40.0
    z = 3.0
    means = [[(lim + 0.08) * z, 0.1, z], [0.05, 0.0, 2.5], [-0.1, 0.05, 2.0]]
    rng = np.random.default_rng(9)
    p = gauss(means, [[-0.9, -1.3, -1.1], [-2.0, -2.2, -1.9], [-2.4, -2.2, -2.6]],
              quats=rng.standard_normal((3, 4)), logits=[1.0, 6.0, 0.3],
              sh=np.concatenate([rng.uniform(-1, 1, (3, 1, 3)), rng.normal(0, 0.2, (3, 15, 3))], 1))
    pr = orc.project(p, cam, orc.Dilation())
    assert pr["tiles_touched"][0] > 0 and pr["xy"][0, 0] > 48
    _fd_check(p, cam, orc.Dilation(), (0.0, 0.0, 0.0), seed=3)


def test_loss_l1_gradient_and_value():
    cam = ident_cam(w=20, h=12)
    dil = orc.Dilation(2, 1, 0)
    w_ds, h_ds, _, _ = orc.grid(cam, dil)
    rng = np.random.default_rng(6)
    img = rng.uniform(0, 1, (h_ds, w_ds, 3))
    target = rng.uniform(0, 1, (12, 20, 3))
    L, g = orc.loss_l1(img, target, cam, dil)
    ref = target[0::2, 1::2]
    assert L == pytest.approx(np.abs(img - ref).mean(), rel=1e-13)
    np.testing.assert_allclose(g, np.sign(img - ref) / img.size, atol=1e-16)


# ---------------------------------------------------------------------------
# Densification statistics (Sec. 3.3) and Adam (Sec. 4.1)
# ---------------------------------------------------------------------------

def test_densify_stats_accumulates_gradient_norms():
    n = 5
    tt = np.array([3, 0, 1, 7, 2])
    g1 = dict(dxy=np.array([[3.0, 4.0]] * n), drgb=np.array([[1.0, 2.0, 2.0]] * n))
    g2 = dict(dxy=np.array([[0.0, 1.0]] * n), drgb=np.array([[0.0, 0.0, 0.5]] * n))
    pos, col, cnt = np.zeros(n), np.zeros(n), np.zeros(n, np.int32)
    orc.densify_stats(tt, g1, pos, col, cnt)
    orc.densify_stats(tt, g2, pos, col, cnt)
    vis = tt > 0
    np.testing.assert_allclose(pos, np.where(vis, 6.0, 0.0))
    np.testing.assert_allclose(col, np.where(vis, 3.5, 0.0))
    np.testing.assert_array_equal(cnt, np.where(vis, 2, 0))


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g both bias-corrected moments are exact (m^ = g,
    v^ = g^2), so every step moves by lr g / (|g| + eps)."""
    g = np.array([[0.3, -2.0, 1e-3], [5.0, -0.01, 0.0]])
    p = np.zeros_like(g)
    m, v = np.zeros_like(g), np.zeros_like(g)
    lr, eps = 0.01, 1e-8
    for t in range(1, 8):
        orc.adam(p, g, m, v, lr, 0.9, 0.999, eps, t)
    np.testing.assert_allclose(p, -7 * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    # masked rows stay put
    p2, m2, v2 = np.zeros_like(g), np.zeros_like(g), np.zeros_like(g)
    orc.adam(p2, g, m2, v2, lr, 0.9, 0.999, eps, 1, row_mask=np.array([0, 1]))
    assert np.all(p2[0] == 0) and np.all(m2[0] == 0) and np.all(p2[1] != 0) | (g[1] == 0).any()


def test_adam_two_steps_by_hand():
    p, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    orc.adam(p, np.array([0.5]), m, v, 0.1, 0.9, 0.99, 0.0, 1)
    assert p[0] == pytest.approx(1.0 - 0.1)  # step 1: -lr sign(g)
    orc.adam(p, np.array([-1.0]), m, v, 0.1, 0.9, 0.99, 0.0, 2)
    m2 = 0.9 * 0.05 + 0.1 * -1.0
    v2 = 0.99 * 0.0025 + 0.01 * 1.0
    step = (m2 / (1 - 0.81)) / math.sqrt(v2 / (1 - 0.9801))
    assert p[0] == pytest.approx(0.9 - 0.1 * step, rel=1e-12)
