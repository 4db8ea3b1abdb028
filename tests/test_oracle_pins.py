"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against a closed form, an invariant, a hand-worked example or a
brute-force search that does not go through the oracle's own code path, chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage, optimize

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- pyramid (Sec. 3.1)
def test_pyr_down_preserves_ramp_in_interior():
    h, w = 29, 37
    y, x = np.mgrid[0:h, 0:w].astype(float)
    a, b, c = 3.0, -2.0, 7.0
    out = oracle.pyr_down(a * x + b * y + c)
    assert out.shape == (15, 19)
    yo, xo = np.mgrid[0:15, 0:19].astype(float)
    ref = a * 2 * xo + b * 2 * yo + c
    inner = (2 * xo - 2 >= 0) & (2 * xo + 2 <= w - 1) & (2 * yo - 2 >= 0) & (2 * yo + 2 <= h - 1)
    assert np.abs(out - ref)[inner].max() < 1e-12


@pytest.mark.parametrize("pos", [(10, 8), (11, 9)])
def test_pyr_down_impulse_gives_binomial_weights(pos):
    # an impulse at (col, row) = pos lands on the even-sampled [1 4 6 4 1]/16 weights
    img = np.zeros((20, 24))
    img[pos[1], pos[0]] = 1.0
    out = oracle.pyr_down(img)
    k = {-2: 1 / 16, -1: 4 / 16, 0: 6 / 16, 1: 4 / 16, 2: 1 / 16}
    ref = np.zeros_like(out)
    for yo in range(out.shape[0]):
        for xo in range(out.shape[1]):
            i, j = pos[0] - 2 * xo, pos[1] - 2 * yo
            if abs(i) <= 2 and abs(j) <= 2:
                ref[yo, xo] = k[i] * k[j]
    assert np.abs(out - ref).max() < 1e-15
    assert abs(out.sum() - (1.0 / 4.0 if pos == (10, 8) else 1.0 / 4.0)) < 1e-15


def test_pyr_down_replicated_border_and_sizes():
    img = np.zeros((7, 9))
    img[0, 0] = 1.0
    out = oracle.pyr_down(img)
    assert out.shape == (4, 5)
    # offsets -2, -1, 0 all clamp onto pixel 0: weight (1 + 4 + 6) / 16 per axis
    assert abs(out[0, 0] - (11 / 16) ** 2) < 1e-15
    const = oracle.pyr_down(np.full((5, 6), 4.25))
    assert np.abs(const - 4.25).max() < 1e-15 and const.shape == (3, 3)


# ---------------------------------------------------------------- gradients
def test_sobel_ramp_interior_border_and_constant():
    h, w = 12, 15
    y, x = np.mgrid[0:h, 0:w].astype(float)
    a, b = 3.0, -2.0
    gx, gy = oracle.sobel(a * x + b * y + 1.0)
    assert np.abs(gx[1:-1, 1:-1] - a).max() < 1e-12
    assert np.abs(gy[1:-1, 1:-1] - b).max() < 1e-12
    # replicated border: one-sided difference over two pixels -> half the slope
    assert np.abs(gx[1:-1, 0] - a / 2).max() < 1e-12 and np.abs(gx[1:-1, -1] - a / 2).max() < 1e-12
    assert np.abs(gy[0, 1:-1] - b / 2).max() < 1e-12
    cx, cy = oracle.sobel(np.full((6, 5), 9.0))
    assert np.abs(cx).max() == 0.0 and np.abs(cy).max() == 0.0


def test_sobel_exact_on_bilinear_function():
    h, w = 10, 11
    y, x = np.mgrid[0:h, 0:w].astype(float)
    gx, gy = oracle.sobel(0.5 + 0.3 * x - 0.7 * y + 0.05 * x * y)
    assert np.abs(gx[1:-1, 1:-1] - (0.3 + 0.05 * y[1:-1, 1:-1])).max() < 1e-12
    assert np.abs(gy[1:-1, 1:-1] - (-0.7 + 0.05 * x[1:-1, 1:-1])).max() < 1e-12


@pytest.mark.parametrize("h,w", [(17, 23), (8, 5), (1, 6)])
def test_pyramid_and_sobel_equal_library_filters_on_noise(h, w):
    """On white noise (no symmetry to hide a transposed or misplaced tap) the pyramid step is
    scipy's separable [1 4 6 4 1]/16 correlation with edge replication sampled at even (x, y),
    and the gradients are scipy's Sobel (difference along the axis, [1 2 1] across it, edge
    replication) divided by 8.  A ramp or a bilinear function cannot tell the Sobel smoothing
    axis apart; noise can."""
    g = np.random.default_rng(h * 31 + w)
    img = g.uniform(0, 255, (h, w))
    k = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0
    ref = ndimage.correlate1d(ndimage.correlate1d(img, k, axis=0, mode="nearest"), k, axis=1, mode="nearest")
    out = oracle.pyr_down(img)
    assert out.shape == ((h + 1) // 2, (w + 1) // 2)
    assert np.abs(out - ref[::2, ::2]).max() < 1e-11
    gx, gy = oracle.sobel(img)
    assert np.abs(gx - ndimage.sobel(img, axis=1, mode="nearest") / 8.0).max() < 1e-11
    assert np.abs(gy - ndimage.sobel(img, axis=0, mode="nearest") / 8.0).max() < 1e-11


# ---------------------------------------------------------------- bilinear sampling
def test_bilinear_exact_and_clamped():
    h, w = 9, 13
    y, x = np.mgrid[0:h, 0:w].astype(float)
    f = lambda X, Y: 1.0 + 0.2 * X - 0.4 * Y + 0.03 * X * Y  # noqa: E731
    img = f(x, y)
    g = np.random.default_rng(1)
    for _ in range(200):
        X, Y = g.uniform(0, w - 1), g.uniform(0, h - 1)
        assert abs(oracle.bilinear(img, X, Y) - f(X, Y)) < 1e-12
    # outside the image the coordinate is clamped first
    assert abs(oracle.bilinear(img, -3.2, 4.5) - f(0, 4.5)) < 1e-12
    assert abs(oracle.bilinear(img, w + 5.0, h + 1.0) - f(w - 1, h - 1)) < 1e-12
    assert abs(oracle.bilinear(img, w - 1.0, 2.25) - f(w - 1, 2.25)) < 1e-12


# ---------------------------------------------------------------- grid and levels
def test_stride_reading_and_counts():
    assert oracle.stride(8, 0.3) == 6 and oracle.stride(8, 0.4) == 5
    assert oracle.stride(12, 0.75) == 3 and oracle.stride(8, 0.5) == 4
    assert oracle.stride(8, 0.3, 4) == 4 and oracle.stride(8, 0.99) == 1
    # 128x96, stride 4: levels 128x96, 64x48, 32x24
    assert [oracle.grid_n(W, 8, 4) * oracle.grid_n(H, 8, 4) for W, H in [(128, 96), (64, 48), (32, 24)]] == [713, 165, 35]
    # 1024x436, theta_ps 8, theta_ov 0.3: levels 4, 3, 2
    assert [oracle.grid_n(W, 8, 6) * oracle.grid_n(H, 8, 6) for W, H in [(64, 28), (128, 55), (256, 109)]] == [55, 189, 774]
    assert oracle.grid_n(1024, 12, 3) * oracle.grid_n(436, 12, 3) == 339 * 143 == 48477
    assert oracle.grid_n(7, 8, 4) == 0 and oracle.grid_n(8, 8, 4) == 1


@pytest.mark.parametrize("L,ps,st", [(37, 8, 6), (64, 8, 4), (8, 8, 3), (436, 12, 3), (29, 12, 5)])
def test_grid_covers_every_pixel_and_stays_inside(L, ps, st):
    n = oracle.grid_n(L, ps, st)
    pos = [oracle.grid_pos(i, L, ps, st) for i in range(n)]
    assert pos[0] == 0 and pos[-1] == L - ps
    assert all(0 <= p <= L - ps for p in pos) and pos == sorted(pos)
    cover = np.zeros(L, int)
    for p in pos:
        cover[p:p + ps] += 1
    assert cover.min() >= 1


def test_paper_values_levels():
    gv = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    for case in gv["theta_ss_examples"]["cases"]:
        rc, ss, sf = oracle.levels(case["width"], case["height"], oracle.params(patch_size=case["ps"]))
        assert rc == 0 and ss == case["theta_ss"]
    p = oracle.params()
    assert (p.delta, p.gamma, p.alpha) == tuple(gv["delta_gamma_alpha"]["value"])
    assert p.var_inner == gv["theta_vi"]["value"]
    # a coarsest level smaller than a patch is lowered (auto) or refused (explicit)
    assert oracle.levels(64, 20, oracle.params(patch_size=8))[1] == 1
    assert oracle.levels(64, 20, oracle.params(patch_size=8, coarsest_scale=3))[0] == 4
    assert oracle.levels(6, 6, oracle.params(patch_size=8))[0] == 4
    # an automatic theta_ss below theta_sf is raised to theta_sf (Alg. 1 runs ss down to sf)
    assert oracle.levels(64, 48, oracle.params(patch_size=8, finest_scale=2)) == (0, 2, 2)
    assert oracle.levels(24, 24, oracle.params(patch_size=8, finest_scale=2))[0] == 4


# ---------------------------------------------------------------- inverse search (Sec. 2.1, supp. A)
def _bilinear_scene(h, w, c, t):
    """I0 = f(x), I1 = f(x - t) for f = c0 + c1 x + c2 y + c3 x y, with exact gradients."""
    y, x = np.mgrid[0:h, 0:w].astype(float)
    f = lambda X, Y: c[0] + c[1] * X + c[2] * Y + c[3] * X * Y  # noqa: E731
    I0, I1 = f(x, y), f(x - t[0], y - t[1])
    return I0, I1, c[1] + c[3] * y, c[2] + c[3] * x


def _patch_index(w, ps, st, px, py):
    nx = oracle.grid_n(w, ps, st)
    return (py // st) * nx + (px // st)


@pytest.mark.parametrize("ps", [8, 12])
def test_search_saddle_centred_on_patch_converges_in_one_step(ps):
    # f = c3 (x - x0)(y - y0) with (x0, y0) the patch centre: mean gradient 0, so the
    # mean-normalised residual is linear in the error and one update is exact.
    h = w = 48
    px = py = 16
    x0 = y0 = px + (ps - 1) / 2
    c3, t = 0.8, (1.37, -0.61)
    c = (c3 * x0 * y0 + 5.0, -c3 * y0, -c3 * x0, c3)
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    u, ui, st = oracle.search_level(I0, gx, gy, I1, ps, 16, 1)
    k = _patch_index(w, ps, 16, px, py)
    uu = u.reshape(-1, 2)[k]
    assert np.abs(uu - np.array(t)).max() < 1e-12 and st.reshape(-1)[k] == 0


def test_search_off_centre_contracts_by_closed_form_matrix():
    # delta_{k+1} = M delta_k with M = n H'^-1 gbar gbar^T (error dynamics of the
    # inverse-compositional step with mean-normalisation on a bilinear image).
    h = w = 64
    ps, st_, px, py = 8, 8, 24, 32
    c = (2.0, 0.4, -0.3, 0.05)
    t = np.array([0.8, 0.45])
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    Y, X = np.mgrid[py:py + ps, px:px + ps].astype(float)
    G = np.stack([(c[1] + c[3] * Y).ravel(), (c[2] + c[3] * X).ravel()], 1)
    Hm = G.T @ G
    gbar = G.mean(0)
    M = ps * ps * np.linalg.solve(Hm, np.outer(gbar, gbar))
    k = _patch_index(w, ps, st_, px, py)
    for iters in range(1, 6):
        u, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, iters)
        err = u.reshape(-1, 2)[k] - t
        ref = np.linalg.matrix_power(M, iters) @ (-t)
        assert np.abs(err - ref).max() < 1e-11, (iters, err, ref)


def test_search_integer_translation_is_fixed_point():
    g = np.random.default_rng(7)
    h, w, t = 40, 44, (3, -2)
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 1.5) * 50 + 100
    I1 = g.uniform(0, 255, (h, w))
    I1[max(0, t[1]):h + min(0, t[1]), max(0, t[0]):w + min(0, t[0])] = \
        I0[max(0, -t[1]):h - max(0, t[1]), max(0, -t[0]):w - max(0, t[0])]
    gx, gy = oracle.sobel(I0)
    Uc = np.zeros((h, w, 2))
    Uc[..., 0], Uc[..., 1] = t
    u, ui, st = oracle.search_level(I0, gx, gy, I1, 8, 4, 12, Uc=Uc, cscale=1.0)
    nx, ny = oracle.grid_n(w, 8, 4), oracle.grid_n(h, 8, 4)
    checked = 0
    for j in range(ny):
        for i in range(nx):
            px, py = oracle.grid_pos(i, w, 8, 4), oracle.grid_pos(j, h, 8, 4)
            if px + t[0] >= 0 and px + 7 + t[0] <= w - 1 and py + t[1] >= 0 and py + 7 + t[1] <= h - 1:
                assert np.abs(u[j, i] - t).max() < 1e-9
                checked += 1
    assert checked > 20


def test_search_matches_brute_force_ssd_minimum():
    # noise-free sub-pixel translation of a smooth texture, one 8x8 patch in a 16x16 image
    h = w = 16
    t = (0.37, -0.61)
    f = lambda X, Y: 100 + 30 * np.sin(0.35 * X + 0.2) * np.cos(0.28 * Y - 0.4) + 12 * np.sin(0.21 * (X + Y))  # noqa
    y, x = np.mgrid[0:h, 0:w].astype(float)
    I0, I1 = f(x, y), f(x - t[0], y - t[1])
    gx, gy = oracle.sobel(I0)
    u, _, st = oracle.search_level(I0, gx, gy, I1, 8, 4, 300)
    u_ic = u[1, 1]
    P = I0[4:12, 4:12]
    T = P - P.mean()
    Yp, Xp = np.mgrid[4:12, 4:12].astype(float)

    def ssd(v):
        wv = ndimage.map_coordinates(I1, [Yp + v[1], Xp + v[0]], order=1, mode="nearest")
        return float(((wv - wv.mean() - T) ** 2).sum())

    grid = np.arange(-2, 2.0001, 1 / 16)
    vals = np.array([[ssd((a, b)) for a in grid] for b in grid])
    jb, ib = np.unravel_index(np.argmin(vals), vals.shape)
    res = optimize.minimize(ssd, [grid[ib], grid[jb]], method="Nelder-Mead",
                            options=dict(xatol=1e-7, fatol=1e-12, maxiter=4000))
    assert np.abs(u_ic - res.x).max() < 5e-3, (u_ic, res.x)
    assert np.abs(u_ic - np.array(t)).max() < 2e-2


@pytest.mark.parametrize("tx,expect_reset", [(7.0, False), (9.0, True)])
def test_search_outlier_reset_threshold(tx, expect_reset):
    # converges to t on a saddle-dominated bilinear image; |t| > theta_ps resets to u_init
    h = w = 72
    ps, px, py = 8, 32, 32
    x0 = y0 = px + 3.5
    c = (0.6 * x0 * y0 + 3.0, -0.6 * y0 + 0.1, -0.6 * x0, 0.6)
    t = (tx, 0.0)
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    u, ui, st = oracle.search_level(I0, gx, gy, I1, ps, 8, 400)
    k = _patch_index(w, ps, 8, px, py)
    if expect_reset:
        assert st.reshape(-1)[k] == 1 and np.abs(u.reshape(-1, 2)[k]).max() == 0.0
    else:
        assert st.reshape(-1)[k] == 0 and np.abs(u.reshape(-1, 2)[k] - t).max() < 1e-9


def test_search_init_from_coarser_level_and_flat_patches():
    # theta_it = 0 exposes u_init = 2 U_{s+1}(c / 2) at the patch centre c = p + (ps - 1)/2
    h, w, ps, st_ = 40, 52, 8, 4
    hc, wc = 20, 26
    yc, xc = np.mgrid[0:hc, 0:wc].astype(float)
    Uc = np.stack([0.1 * xc - 0.05 * yc + 0.3, -0.02 * xc + 0.07 * yc - 0.2], -1)
    g = np.random.default_rng(3)
    I0 = g.uniform(0, 255, (h, w))
    gx, gy = oracle.sobel(I0)
    u, ui, st = oracle.search_level(I0, gx, gy, I0, ps, st_, 0, Uc=Uc, cscale=2.0)
    for j in range(ui.shape[0]):
        for i in range(ui.shape[1]):
            cx = oracle.grid_pos(i, w, ps, st_) + 3.5
            cy = oracle.grid_pos(j, h, ps, st_) + 3.5
            ref = 2 * np.array([0.1 * cx / 2 - 0.05 * cy / 2 + 0.3, -0.02 * cx / 2 + 0.07 * cy / 2 - 0.2])
            assert np.abs(ui[j, i] - ref).max() < 1e-12
    assert np.array_equal(u, ui)
    flat = np.full((h, w), 77.0)
    fx, fy = oracle.sobel(flat)
    u2, ui2, st2 = oracle.search_level(flat, fx, fy, I0, ps, st_, 10, Uc=Uc)
    assert (st2 == 2).all() and np.array_equal(u2, ui2)


# ---------------------------------------------------------------- densification (Eq. 3)
def test_densify_constant_patch_flow_is_reproduced():
    g = np.random.default_rng(5)
    I0, I1 = g.uniform(0, 255, (30, 41)), g.uniform(0, 255, (30, 41))
    ps, st_ = 8, 3
    nx, ny = oracle.grid_n(41, ps, st_), oracle.grid_n(30, ps, st_)
    u = np.tile(np.array([1.25, -0.5]), (ny, nx, 1))
    U = oracle.densify_level(I0, I1, u, ps, st_)
    assert np.abs(U - np.array([1.25, -0.5])).max() < 1e-12


def test_densify_without_overlap_copies_patch_flow():
    g = np.random.default_rng(6)
    I0, I1 = g.uniform(0, 255, (16, 24)), g.uniform(0, 255, (16, 24))
    u = g.uniform(-3, 3, (2, 3, 2))
    U = oracle.densify_level(I0, I1, u, 8, 8)
    ref = np.repeat(np.repeat(u, 8, 0), 8, 1)
    assert np.abs(U - ref).max() < 1e-12


def test_densify_two_patch_hand_example():
    # 12x8 image, theta_ps 8, stride 4: patches at x = 0 and x = 4, both covering x = 4..7.
    # I0 = 0; I1 varies along x.  At x = 5: d_0 = I1(6) = -3 for u_0 = (1, 0) and
    # d_1 = I1(5) = 0.5 for u_1 = (0, 0): weights 1/3 and 1 -> U = (1/3) / (4/3) = 0.25.
    I0 = np.zeros((8, 12))
    row = np.array([0, 0, 0, 0, 0.25, 0.5, -3.0, 2.0, 0.0, 0, 0, 0])
    I1 = np.tile(row, (8, 1))
    u = np.array([[[1.0, 0.0], [0.0, 0.0]]])
    U = oracle.densify_level(I0, I1, u, 8, 4)
    assert abs(U[3, 5, 0] - 0.25) < 1e-15 and U[3, 5, 1] == 0.0
    # x = 4: d_0 = I1(5) = 0.5, d_1 = I1(4) = 0.25 -> both weights 1 -> 0.5
    assert abs(U[3, 4, 0] - 0.5) < 1e-15
    # x = 6: d_0 = I1(7) = 2 -> 1/2, d_1 = I1(6) = -3 -> 1/3 -> (1/2) / (5/6) = 0.6
    assert abs(U[3, 6, 0] - 0.6) < 1e-15
    # x = 2: only patch 0; x = 10: only patch 1
    assert U[0, 2, 0] == 1.0 and U[0, 10, 0] == 0.0


@pytest.mark.parametrize("W,H,ps,st_", [(29, 23, 8, 3), (37, 26, 12, 3), (31, 19, 8, 5), (20, 13, 12, 6)])
def test_densify_ragged_grid_by_brute_force(W, H, ps, st_):
    """Eq. 3 evaluated from its definition: every patch at its corner (min(i*stride, W - ps),
    min(j*stride, H - ps)), i = 0 .. ceil((W - ps) / stride), contributes to the pixels it
    contains with weight 1 / max(1, |I1(x + u_i) - I0(x)|), I1 sampled bilinearly at coordinates
    clamped to the frame (scipy's order-1 interpolation with edge extension).  The ragged sizes
    put the last patch of each row and column off the regular stride, and a few large patch
    flows reach past the frame."""
    g = np.random.default_rng(W * 100 + ps)
    I0, I1 = g.uniform(0, 255, (H, W)), g.uniform(0, 255, (H, W))
    xs = [min(i * st_, W - ps) for i in range(-(-(W - ps) // st_) + 1)]
    ys = [min(j * st_, H - ps) for j in range(-(-(H - ps) // st_) + 1)]
    u = g.normal(0.0, 1.5, (len(ys), len(xs), 2))
    u[::3, ::2] *= 8.0
    U = oracle.densify_level(I0, I1, u, ps, st_)
    assert U.shape == (H, W, 2)
    num = np.zeros((H, W, 2))
    den = np.zeros((H, W))
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    for j, py in enumerate(ys):
        for i, px in enumerate(xs):
            cx = np.clip(xx + u[j, i, 0], 0, W - 1)
            cy = np.clip(yy + u[j, i, 1], 0, H - 1)
            w1 = ndimage.map_coordinates(I1, [cy, cx], order=1, mode="nearest")
            wt = 1.0 / np.maximum(1.0, np.abs(w1 - I0))
            inside = (xx >= px) & (xx < px + ps) & (yy >= py) & (yy < py + ps)
            num += np.where(inside, wt, 0.0)[..., None] * u[j, i]
            den += np.where(inside, wt, 0.0)
    assert den.min() > 0  # the grid covers every pixel
    ref = num / den[..., None]
    assert np.abs(U - ref).max() < 1e-10


# ---------------------------------------------------------------- refinement (Sec. 2.3)
def test_refine_two_pixel_hand_sweep():
    # delta = gamma = 0: pure smoothing.  2x1 image, U = [(1,0), (0,0)], both pixels have
    # |grad u|^2 = 1/4 so equal weights w.  Red pixel 0: d = (0 - 1) -> dU0 = -omega;
    # black pixel 1: d = 1 - omega - 0 -> dU1 = omega (1 - omega).
    I = np.zeros((1, 2))
    U = np.array([[[1.0, 0.0], [0.0, 0.0]]])
    om = 1.6
    out = oracle.refine_level(I, I, U, 1, 1, delta=0.0, gamma=0.0, alpha=10.0, omega=om)
    assert abs(out[0, 0, 0] - (1 - om)) < 1e-14 and abs(out[0, 1, 0] - om * (1 - om)) < 1e-14
    # the same along y (1x2 image) with the v component
    Uy = np.array([[[0.0, 1.0]], [[0.0, 0.0]]])
    outy = oracle.refine_level(I.T.copy(), I.T.copy(), Uy, 1, 1, delta=0.0, gamma=0.0, alpha=3.0, omega=om)
    assert abs(outy[0, 0, 1] - (1 - om)) < 1e-14 and abs(outy[1, 0, 1] - om * (1 - om)) < 1e-14


def test_refine_three_pixel_hand_sweep_unequal_weights():
    # 3x1, U = [(1,0), (0,0), (0,0)]: central differences give |grad u|^2 = 1/4 at pixels 0
    # and 1 and 0 at pixel 2, so psi_S = alpha / (2 sqrt(E_S + eps^2)) is a, a, b.
    # Red (0, 2) first: pixel 0 -> d = -1, pixel 2 -> d = 0.  Black pixel 1 with edge weights
    # w01 = a and w12 = (a + b)/2:  d = w01 (1 - omega) / (w01 + w12).
    alpha, om, eps = 10.0, 1.6, 1e-3
    a = alpha / (2 * math.sqrt(0.25 + eps * eps))
    b = alpha / (2 * eps)
    I = np.zeros((1, 3))
    U = np.array([[[1.0, 0.0], [0.0, 0.0], [0.0, 0.0]]])
    out = oracle.refine_level(I, I, U, 1, 1, delta=0.0, gamma=0.0, alpha=alpha, omega=om)
    d1 = a * (1 - om) / (a + 0.5 * (a + b))
    assert abs(out[0, 0, 0] - (1 - om)) < 1e-14
    assert abs(out[0, 1, 0] - om * d1) < 1e-14 and abs(out[0, 2, 0]) < 1e-14


def test_refine_pure_smoothing_invariants():
    g = np.random.default_rng(11)
    I0, I1 = g.uniform(0, 255, (14, 17)), g.uniform(0, 255, (14, 17))
    U = np.tile(np.array([0.7, -1.1]), (14, 17, 1))
    out = oracle.refine_level(I0, I1, U, 3, 5, delta=0.0, gamma=0.0)
    assert np.abs(out - U).max() < 1e-13
    U2 = g.uniform(-1, 1, (14, 17, 2))
    out2 = oracle.refine_level(I0, I1, U2, 40, 10, delta=0.0, gamma=0.0, omega=1.0)
    assert (out2.max((0, 1)) - out2.min((0, 1))).max() < 1e-3 < (U2.max((0, 1)) - U2.min((0, 1))).min()


def test_refine_zero_residual_is_fixed_point():
    g = np.random.default_rng(12)
    I0 = ndimage.gaussian_filter(g.uniform(0, 255, (20, 23)), 1.0)
    U = np.zeros((20, 23, 2))
    out = oracle.refine_level(I0, I0, U, 2, 5)
    assert np.abs(out).max() < 1e-13


def _ramp_pair(h, w, a, b, t):
    y, x = np.mgrid[0:h, 0:w].astype(float)
    return a * x + b * y, a * (x - t[0]) + b * (y - t[1])


def test_refine_brightness_term_recovers_translation():
    # two channels with independent ramp directions translated by t: the brightness term
    # (one Psi over the channel sum) has full rank and its minimiser is t itself; the
    # gradient term vanishes on ramps.
    h = w = 40
    t = (0.7, -0.4)
    c0 = _ramp_pair(h, w, 3.0, -2.0, t)
    c1 = _ramp_pair(h, w, 1.0, 2.5, t)
    I0, I1 = np.stack([c0[0], c1[0]]), np.stack([c0[1], c1[1]])
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 80, delta=5.0, gamma=10.0, alpha=1e-4)
    assert np.abs(out[15:25, 15:25] - np.array(t)).max() < 1e-8


@pytest.mark.parametrize("axis", [0, 1])
def test_refine_gradient_term_recovers_translation_of_quadratic(axis):
    # I0 = q^2, I1 = (q - t)^2 along one axis q: I_qq = 2, I_qz = -2t, so the gradient
    # constancy term alone gives the displacement t along that axis.
    h = w = 36
    y, x = np.mgrid[0:h, 0:w].astype(float)
    q = x if axis == 0 else y
    t = 0.35
    I0, I1 = 0.2 * q ** 2, 0.2 * (q - t) ** 2
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 80, delta=0.0, gamma=10.0, alpha=1e-4)
    ref = np.zeros(2)
    ref[axis] = t
    assert np.abs(out[12:24, 12:24] - ref).max() < 1e-8


def test_refine_brightness_term_exact_on_quadratics():
    # Ibar = (I0 + I1w) / 2 makes the brightness linearisation exact for quadratics:
    # I0 = a q^2, I1 = a (q - t)^2 gives I_q = a (2q - t), I_z = -a t (2q - t) -> d = t.
    h = w = 36
    y, x = np.mgrid[0:h, 0:w].astype(float)
    t = (0.35, -0.25)
    I0 = np.stack([0.2 * x ** 2, 0.3 * y ** 2])
    I1 = np.stack([0.2 * (x - t[0]) ** 2, 0.3 * (y - t[1]) ** 2])
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 80, delta=5.0, gamma=0.0, alpha=1e-4)
    assert np.abs(out[12:24, 12:24] - np.array(t)).max() < 1e-8


def test_refine_both_terms_on_diagonal_quadratics():
    # channels a (x + y)^2 and b (x - y)^2 moved by t: every second derivative (I_xy too) is
    # non-zero, both data terms fix du + dv and du - dv, so the minimiser is t.
    h = w = 40
    y, x = np.mgrid[0:h, 0:w].astype(float)
    t = (0.3, -0.45)
    I0 = np.stack([0.05 * (x + y) ** 2, 0.08 * (x - y) ** 2])
    I1 = np.stack([0.05 * (x - t[0] + y - t[1]) ** 2, 0.08 * (x - t[0] - y + t[1]) ** 2])
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 100, delta=5.0, gamma=10.0, alpha=1e-4)
    assert np.abs(out[14:26, 14:26] - np.array(t)).max() < 1e-8
    g_only = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 100, delta=0.0, gamma=10.0, alpha=1e-4)
    assert np.abs(g_only[14:26, 14:26] - np.array(t)).max() < 1e-8


def test_refine_beta_normalisation_balances_channels():
    # two channels with opposite-consistent ramps of slopes a1, a2 moving by t1, t2 along x:
    # the brightness term's minimiser is sum_c beta_c a_c^2 t_c / sum_c beta_c a_c^2 with
    # beta_c = 1 / (a_c^2 + 0.01); a third flat channel adds nothing.
    h = w = 30
    y, x = np.mgrid[0:h, 0:w].astype(float)
    a1, a2, t1, t2 = 1.0, 5.0, 0.2, 0.6
    I0 = np.stack([a1 * x, a2 * x, np.full((h, w), 9.0)])
    I1 = np.stack([a1 * (x - t1), a2 * (x - t2), np.full((h, w), 9.0)])
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 80, delta=5.0, gamma=0.0, alpha=1e-4)
    b1, b2 = 1 / (a1 ** 2 + 0.01), 1 / (a2 ** 2 + 0.01)
    ref = (b1 * a1 ** 2 * t1 + b2 * a2 ** 2 * t2) / (b1 * a1 ** 2 + b2 * a2 ** 2)
    assert np.abs(out[10:20, 10:20, 0] - ref).max() < 1e-8
    assert np.abs(out[10:20, 10:20, 1]).max() < 1e-8


def test_refine_gradient_term_beta_normalisation():
    h = w = 30
    y, x = np.mgrid[0:h, 0:w].astype(float)
    a1, a2, t1, t2 = 0.1, 2.0, 0.3, -0.2
    I0 = np.stack([a1 * x ** 2, a2 * x ** 2])
    I1 = np.stack([a1 * (x - t1) ** 2, a2 * (x - t2) ** 2])
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 120, delta=0.0, gamma=10.0, alpha=1e-5)
    # per channel I_xx = 2 a_c, I_xy = 0, I_xz = -2 a_c t_c: beta_x = 1 / (4 a_c^2 + 0.01)
    wts = [(2 * a) ** 2 / ((2 * a) ** 2 + 0.01) for a in (a1, a2)]
    ref = (wts[0] * t1 + wts[1] * t2) / (wts[0] + wts[1])
    assert np.abs(out[10:20, 10:20, 0] - ref).max() < 1e-7


# ---------------------------------------------------------------- up-scaling and pipeline
def test_upsample_linear_field():
    hi, wi = 7, 9
    y, x = np.mgrid[0:hi, 0:wi].astype(float)
    U = np.stack([0.5 * x - 0.25 * y + 1.0, 0.1 * x + 0.2 * y - 0.3], -1)
    out = oracle.upsample_flow(U, 2.0, (13, 17))
    yo, xo = np.mgrid[0:13, 0:17].astype(float)
    ref = np.stack([0.5 * xo - 0.25 * yo + 2.0, 0.1 * xo + 0.2 * yo - 0.6], -1)
    assert np.abs(out - ref).max() < 1e-12
    assert np.array_equal(oracle.upsample_flow(U, 1.0, (hi, wi)), U)


@pytest.mark.parametrize("factor,src,dst", [(2.0, (7, 9), (13, 18)), (4.0, (5, 6), (20, 23)), (8.0, (3, 4), (17, 29))])
def test_upsample_random_field_equals_library_interpolation(factor, src, dst):
    """U_out(x) = factor * U(x / factor), bilinear at coordinates clamped to the coarse field:
    on a random field, against scipy's order-1 interpolation with edge extension (which equals
    clamping the coordinate), per component; the output sizes leave the last coarse sample
    behind the clamp."""
    g = np.random.default_rng(int(factor) * 7 + src[0])
    U = g.normal(0.0, 3.0, src + (2,))
    out = oracle.upsample_flow(U, factor, dst)
    yo, xo = np.mgrid[0:dst[0], 0:dst[1]].astype(float)
    cy = np.clip(yo / factor, 0, src[0] - 1)
    cx = np.clip(xo / factor, 0, src[1] - 1)
    for c in range(2):
        ref = factor * ndimage.map_coordinates(U[..., c], [cy, cx], order=1, mode="nearest")
        assert np.abs(out[..., c] - ref).max() < 1e-11


def test_pipeline_recovers_translation_of_saddle_image():
    # bilinear (saddle) scene: every pyramid level stays bilinear in its interior, interior
    # patches contract exactly onto t / 2^s, so interior pixels of the final flow equal t.
    h = w = 48
    y, x = np.mgrid[0:h, 0:w].astype(float)
    t = (1.3, -0.7)
    f = lambda X, Y: 0.5 * (X - 23.5) * (Y - 23.5) + 100.0  # noqa: E731
    I0, I1 = f(x, y), f(x - t[0], y - t[1])
    p = oracle.params(patch_size=8, stride_override=4, grad_iters=5000, coarsest_scale=1, refine=0,
                      intensity_scale=1.0)
    flow = oracle.dis_flow(I0, I1, p)
    assert np.abs(flow[12:36, 12:36] - np.array(t)).max() < 1e-6


def test_pipeline_translation_sanity_and_frozen_replay():
    from paper_1603_03590_gb300 import synth
    I0, I1, gt = synth.translation_pair(0)
    p = oracle.params(patch_size=8, stride_override=4, grad_iters=16, coarsest_scale=2, var_outer=1)
    flow, rec, hv = oracle.dis_flow(I0, I1, p, record=True, want_hash=True)
    epe = np.linalg.norm(flow - gt, axis=-1)
    assert epe[8:-8, 8:-8].mean() < 0.1
    assert rec.shape == (oracle.total_patches(128, 96, p), 2) == (713 + 165 + 35, 2)
    again, hv2 = oracle.dis_flow(I0, I1, p, frozen=rec, want_hash=True)
    assert np.abs(again - flow).max() < 1e-12
    flow3, hv3 = oracle.dis_flow(I0, I1, p, want_hash=True)
    assert hv3 == hv and np.array_equal(flow3, flow)


def test_charbonnier_loss_closed_forms():
    g = np.random.default_rng(2)
    I0 = g.uniform(0, 1, (9, 10))
    zero = np.zeros((9, 10, 2))
    assert abs(oracle.charbonnier_loss(I0, I0, zero, 1e-3) - 1e-3) < 1e-15
    assert abs(oracle.charbonnier_loss(I0, I0 + 0.25, zero, 1e-3) - math.sqrt(0.0625 + 1e-6)) < 1e-12


# ---- stereo: the vertical degree of freedom removed (supplementary, depth from stereo) ----

def test_stereo_search_contracts_by_scalar_closed_form():
    # Horizontal translation of a bilinear image, v held at 0: the mean-normalised residual is
    # exactly (g_x - mean g_x) du, so one scalar step maps du -> rho du with
    # rho = n mean(g_x)^2 / sum g_x^2 (the 1-D case of the contraction M of the flow search).
    h = w = 64
    ps, st_, px, py = 8, 8, 24, 32
    c = (2.0, -0.3 * 34, -0.3, 0.3)  # g_x = 0.3 (y - 34) changes sign inside the patch
    t = np.array([0.8, 0.0])
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    Y, X = np.mgrid[py:py + ps, px:px + ps].astype(float)
    Gx = (c[1] + c[3] * Y).ravel()
    rho = ps * ps * Gx.mean() ** 2 / (Gx ** 2).sum()
    assert 0.05 < rho < 0.95
    k = _patch_index(w, ps, st_, px, py)
    for iters in range(1, 6):
        u, _, st = oracle.search_level(I0, gx, gy, I1, ps, st_, iters, dof=1)
        err = u.reshape(-1, 2)[k] - t
        assert abs(err[0] - rho ** iters * (-t[0])) < 1e-11 and err[1] == 0.0, (iters, err)


def test_stereo_search_keeps_v_and_needs_horizontal_texture():
    g = np.random.default_rng(21)
    h, w = 40, 48
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 1.5) * 40 + 120
    I1 = np.roll(I0, 1, axis=1)
    gx, gy = oracle.sobel(I0)
    Uc = np.zeros((h, w, 2))
    Uc[..., 1] = 0.75  # the initial vertical displacement survives unchanged
    u, ui, st = oracle.search_level(I0, gx, gy, I1, 8, 4, 8, Uc=Uc, cscale=1.0, dof=1)
    assert (u[..., 1] == 0.75).all() and (st == 0).any()
    # texture along y only: no horizontal gradient, every patch is flat in the scalar search
    Iy = np.tile(ndimage.gaussian_filter(g.standard_normal(h), 1.0)[:, None] * 30 + 100, (1, w))
    gx, gy = oracle.sobel(Iy)
    _, _, st = oracle.search_level(Iy, gx, gy, Iy, 8, 4, 8, dof=1)
    assert (st == 2).all()


def test_stereo_refine_pure_smoothing_matches_flow_u_and_keeps_v():
    # delta = gamma = 0: the 2x2 systems decouple (A = 0), so within one outer pass (fixed
    # smoothness weights) the horizontal component of the flow refinement and the scalar
    # refinement take identical steps; v does not move.  (A second pass differs: the lagged
    # weights see the smoothed v of the flow refinement.)
    g = np.random.default_rng(22)
    I0, I1 = g.uniform(0, 255, (11, 13)), g.uniform(0, 255, (11, 13))
    U = g.uniform(-1, 1, (11, 13, 2))
    a = oracle.refine_level(I0, I1, U, 1, 6, delta=0.0, gamma=0.0)
    b = oracle.refine_level(I0, I1, U, 1, 6, delta=0.0, gamma=0.0, dof=1)
    assert np.abs(a[..., 0] - b[..., 0]).max() < 1e-13
    assert np.array_equal(b[..., 1], U[..., 1])


def test_stereo_refine_brightness_term_recovers_horizontal_translation():
    # one channel suffices in 1-D: a ramp along x translated by t gives I_x du + I_z = 0 at du = t
    h, w = 30, 40
    t = 0.65
    I0, I1 = _ramp_pair(h, w, 2.5, 1.5, (t, 0.0))
    out = oracle.refine_level(I0, I1, np.zeros((h, w, 2)), 1, 80, delta=5.0, gamma=10.0, alpha=1e-4, dof=1)
    assert np.abs(out[10:20, 10:30, 0] - t).max() < 1e-8 and (out[..., 1] == 0.0).all()


def test_stereo_pipeline_recovers_horizontal_translation_of_saddle_image():
    # the scalar form of the saddle-scene pipeline pin: every level stays bilinear in its
    # interior and each interior patch contracts onto t / 2^s by the scalar factor rho < 1
    h = w = 48
    y, x = np.mgrid[0:h, 0:w].astype(float)
    t = 1.3
    f = lambda X, Y: 0.5 * (X - 23.5) * (Y - 23.5) + 100.0  # noqa: E731
    I0, I1 = f(x, y), f(x - t, y)
    q = oracle.params(patch_size=8, stride_override=4, grad_iters=5000, coarsest_scale=1, refine=0,
                      intensity_scale=1.0, dof=1)
    flow = oracle.dis_flow(I0, I1, q)
    assert np.abs(flow[12:36, 12:36, 0] - t).max() < 1e-6 and (flow[..., 1] == 0.0).all()


# ---- robust error norms (supplementary, robust error norms) ----

def test_robust_error_closed_forms():
    for e in (-7.3, -0.2, 0.0, 0.4, 2.0, 31.0):
        assert oracle.robust_error(e, 0) == e
        v = oracle.robust_error(e, 1)
        assert math.copysign(1, v) == math.copysign(1, e) or e == 0.0
        assert abs(v * v - abs(e)) < 1e-12  # squared: the L1 penalty
        b = 2.0
        hv = oracle.robust_error(e, 2, b)
        huber2 = e * e if abs(e) < b else 2 * b * abs(e) - b * b  # twice the Huber penalty
        assert abs(hv * hv - huber2) < 1e-12 and (hv >= 0) == (e >= 0)
    # continuity of the Huber branch at |e| = b
    assert abs(oracle.robust_error(2.0 - 1e-12, 2, 2.0) - oracle.robust_error(2.0, 2, 2.0)) < 1e-9


def test_robust_search_fixed_points_and_large_huber_threshold():
    g = np.random.default_rng(23)
    h, w, t = 40, 44, (2, -1)
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 1.5) * 50 + 100
    I1 = np.roll(np.roll(I0, t[1], axis=0), t[0], axis=1)
    gx, gy = oracle.sobel(I0)
    Uc = np.zeros((h, w, 2))
    Uc[..., 0], Uc[..., 1] = t
    # an exact integer translation: zero error at u = t, a fixed point of every norm
    for norm in (1, 2):
        u, _, _ = oracle.search_level(I0, gx, gy, I1, 8, 4, 10, Uc=Uc, cscale=1.0, norm=norm, huber_b=3.0)
        inner = u[2:-2, 2:-2]
        assert np.abs(inner - t).max() < 1e-9, norm
    # a Huber threshold above every error leaves the L2 iterates unchanged
    I1s = ndimage.shift(I0, (0.3, -0.45), order=1, mode="nearest")
    a, _, _ = oracle.search_level(I0, gx, gy, I1s, 8, 4, 12)
    b, _, _ = oracle.search_level(I0, gx, gy, I1s, 8, 4, 12, norm=2, huber_b=1e9)
    assert np.array_equal(a, b)


def test_robust_norms_downweight_an_outlier_block():
    # a patch whose lower-right quarter is replaced by garbage in I1: the L1 and Huber
    # searches end closer to the true subpixel translation than L2
    g = np.random.default_rng(24)
    h = w = 48
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 2.0) * 60 + 128
    t = (0.6, -0.35)
    I1 = ndimage.shift(I0, (t[1], t[0]), order=3, mode="nearest")
    px = py = 16
    I1[py + 6:py + 12, px + 6:px + 12] = g.uniform(0, 255, (6, 6))
    gx, gy = oracle.sobel(I0)
    k = _patch_index(w, 12, 4, px, py)
    errs = {}
    for norm in (0, 1, 2):
        u, _, st = oracle.search_level(I0, gx, gy, I1, 12, 4, 60, norm=norm, huber_b=4.0)
        errs[norm] = float(np.hypot(*(u.reshape(-1, 2)[k] - t)))
    assert errs[1] < errs[0] and errs[2] < errs[0], errs


@pytest.mark.parametrize("norm,b", [(1, 5.0), (2, 0.6)])
def test_robust_search_one_step_on_centred_saddle(norm, b):
    # saddle centred on the patch: zero mean gradient, so the mean-normalised error at u = 0 is
    # exactly e_q = g_q . t and H' = H; one step gives u = H^-1 sum_q g_q psi(g_q . t) with psi
    # the norm's error transform (for L2 this is the exact one-step pin above).
    h = w = 48
    ps, px, py = 8, 16, 16
    x0 = y0 = px + (ps - 1) / 2
    c3, t = 0.8, np.array([1.37, -0.61])
    c = (c3 * x0 * y0 + 5.0, -c3 * y0, -c3 * x0, c3)
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    Y, X = np.mgrid[py:py + ps, px:px + ps].astype(float)
    G = np.stack([(c[1] + c[3] * Y).ravel(), (c[2] + c[3] * X).ravel()], 1)
    e = G @ t
    if norm == 1:
        psi = np.sign(e) * np.sqrt(np.abs(e))
    else:
        psi = np.where(np.abs(e) < b, e, np.sign(e) * np.sqrt(np.maximum(2 * b * np.abs(e) - b * b, 0.0)))
    assert (np.abs(e) >= b).any() or norm == 1  # both Huber branches are exercised
    ref = np.linalg.solve(G.T @ G, G.T @ psi)
    u, _, _ = oracle.search_level(I0, gx, gy, I1, ps, 16, 1, norm=norm, huber_b=b)
    got = u.reshape(-1, 2)[_patch_index(w, ps, 16, px, py)]
    assert np.abs(got - ref).max() < 1e-12 and np.abs(got - t).max() > 1e-3


# ---- forward-backward consistency (supplementary Sec. B (ii)) ----

def _fb_brute(I0, I1, uf, ub, ps, st_):
    """Merged forward field by the definition, pixel by pixel in Python: the forward patches
    containing x with weight 1/max(1, |I1(x + u) - I0(x)|); every backward patch with weight
    mu(x)/max(1, |I0(x) - I1(x - u')|) and displacement -u', mu(x) the sum over its template
    pixels q of the bilinear weight that q + u' gives x; bilinear samples from scipy (edge
    values replicated, i.e. coordinates clamped)."""
    h, w = I0.shape
    nx, ny = oracle.grid_n(w, ps, st_), oracle.grid_n(h, ps, st_)
    pos = [(oracle.grid_pos(i, w, ps, st_), oracle.grid_pos(j, h, ps, st_), j * nx + i)
           for j in range(ny) for i in range(nx)]

    def sample(img, x, y):
        return float(ndimage.map_coordinates(img, [[y], [x]], order=1, mode="nearest")[0])

    U = np.zeros((h, w, 2))
    for y in range(h):
        for x in range(w):
            num, Z = np.zeros(2), 0.0
            for px, py, k in pos:
                if px <= x < px + ps and py <= y < py + ps:
                    wt = 1.0 / max(1.0, abs(sample(I1, x + uf[k, 0], y + uf[k, 1]) - I0[y, x]))
                    num += wt * uf[k]
                    Z += wt
            for px, py, k in pos:
                mu = 0.0
                for qy in range(py, py + ps):
                    for qx in range(px, px + ps):
                        mu += max(0.0, 1 - abs(x - qx - ub[k, 0])) * max(0.0, 1 - abs(y - qy - ub[k, 1]))
                if mu > 0.0:
                    wt = mu / max(1.0, abs(I0[y, x] - sample(I1, x - ub[k, 0], y - ub[k, 1])))
                    num -= wt * ub[k]
                    Z += wt
            U[y, x] = num / Z
    return U


def test_fb_densify_consistent_translation_is_exact():
    g = np.random.default_rng(41)
    h, w, t = 30, 34, (2, -1)
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 1.5) * 40 + 120
    I1 = np.roll(np.roll(I0, t[1], axis=0), t[0], axis=1)
    ps, st_ = 6, 3
    n = oracle.grid_n(w, ps, st_) * oracle.grid_n(h, ps, st_)
    uf = np.tile(np.array(t, float), (n, 1))
    U = oracle.densify_level_fb(I0, I1, uf, -uf, ps, st_)
    assert np.abs(U - np.array(t)).max() < 1e-12
    Ub = oracle.densify_level_fb(I1, I0, -uf, uf, ps, st_)
    assert np.abs(Ub + np.array(t)).max() < 1e-12


def test_fb_densify_footprints_by_brute_force():
    # equal constant frames: the error weights are 1, so U(x) is the footprint-weighted mean of
    # the forward patch flows containing x and the negated backward flows; integer backward
    # displacements (footprint edges on pixel centres) and fractional ones are mixed
    g = np.random.default_rng(42)
    h, w, ps, st_ = 17, 19, 5, 3
    I0 = np.full((h, w), 80.0)
    n = oracle.grid_n(w, ps, st_) * oracle.grid_n(h, ps, st_)
    uf = g.uniform(-3, 3, (n, 2))
    ub = g.uniform(-3, 3, (n, 2))
    ub[::3] = np.round(ub[::3])
    U = oracle.densify_level_fb(I0, I0, uf, ub, ps, st_)
    ref = _fb_brute(I0, I0, uf, ub, ps, st_)
    assert np.abs(U - ref).max() < 1e-12
    # a backward patch moved by an integer reaches ps x ps pixels, by a fractional amount in both
    # coordinates (ps + 1)^2; its footprint weights sum to ps^2.  With every other patch at 0,
    # U(x) = -d mu(x) / (n(x) + mu(x)), n(x) the number of other contributions, so mu follows.
    for d, cov in [((1.0, -2.0), ps * ps), ((0.5, 1.25), (ps + 1) ** 2)]:
        ubs = np.zeros((n, 2))
        k = n // 2
        ubs[k] = d
        ufz = np.zeros((n, 2))
        Us = oracle.densify_level_fb(I0, I0, ufz, ubs, ps, st_)
        assert int((Us[..., 0] != 0).sum()) == cov
        ones = np.ones((n, 2))
        cnt = oracle.densify_level_fb(I0, I0, ones, np.full((n, 2), -1.0), ps, st_)  # all contributions equal 1
        assert np.abs(cnt - 1.0).max() < 1e-12
        # n(x): forward patches containing x plus the other backward patches (moved by 0)
        nx_, ny_ = oracle.grid_n(w, ps, st_), oracle.grid_n(h, ps, st_)
        N = np.zeros((h, w))
        for j in range(ny_):
            for i in range(nx_):
                px_, py_ = oracle.grid_pos(i, w, ps, st_), oracle.grid_pos(j, h, ps, st_)
                N[py_:py_ + ps, px_:px_ + ps] += 2 if j * nx_ + i != k else 1
        mu = -Us[..., 0] * N / (Us[..., 0] + d[0])
        assert abs(mu.sum() - ps * ps) < 1e-9


def test_fb_densify_weights_by_brute_force():
    g = np.random.default_rng(43)
    h, w, ps, st_ = 15, 18, 4, 2
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 1.0) * 30 + 100
    I1 = ndimage.shift(I0, (0.4, -0.7), order=3, mode="nearest") + g.normal(0, 2.0, (h, w))
    n = oracle.grid_n(w, ps, st_) * oracle.grid_n(h, ps, st_)
    uf = g.uniform(-2, 2, (n, 2))
    ub = g.uniform(-2, 2, (n, 2))
    U = oracle.densify_level_fb(I0, I1, uf, ub, ps, st_)
    ref = _fb_brute(I0, I1, uf, ub, ps, st_)
    assert np.abs(U - ref).max() < 1e-10


def test_fb_pipeline_recovers_translation_both_ways_and_is_symmetric():
    h = w = 48
    y, x = np.mgrid[0:h, 0:w].astype(float)
    t = (1.3, -0.7)
    f = lambda X, Y: 0.5 * (X - 23.5) * (Y - 23.5) + 100.0  # noqa: E731
    I0, I1 = f(x, y), f(x - t[0], y - t[1])
    q = oracle.params(patch_size=8, stride_override=4, grad_iters=5000, coarsest_scale=1, refine=0,
                      intensity_scale=1.0)
    fw, bw = oracle.dis_flow_fb(I0, I1, q)
    assert np.abs(fw[14:34, 14:34] - np.array(t)).max() < 1e-6
    assert np.abs(bw[14:34, 14:34] + np.array(t)).max() < 1e-6
    # the directions are interchangeable: swapping the frames swaps the two results exactly
    g = np.random.default_rng(44)
    A = ndimage.gaussian_filter(g.standard_normal((40, 56)), 1.5) * 0.15 + 0.5
    B = ndimage.shift(A, (0.6, -1.2), order=3, mode="nearest")
    q = oracle.params(patch_size=8, stride_override=4, grad_iters=12, coarsest_scale=2)
    f1, b1 = oracle.dis_flow_fb(A, B, q)
    f2, b2 = oracle.dis_flow_fb(B, A, q)
    assert np.array_equal(f1, b2) and np.array_equal(b1, f2)
    # and the consistency changes the forward flow (the backward patches entered it)
    plain = oracle.dis_flow(A, B, oracle.params(patch_size=8, stride_override=4, grad_iters=12, coarsest_scale=2))
    assert not np.array_equal(plain, f1) and np.abs(plain - f1).max() < 1.0


# ---- early termination on a small step (supplementary Sec. C) ----

def test_early_termination_stops_at_the_closed_form_iteration():
    # bilinear scene, off-centre patch: the error after k steps is M^k (-t) (see the closed-form
    # pin above), so the step of iteration k is M^(k-1) (-t) - M^k (-t); the search must stop at
    # the first k whose step is at most term_eps and return M^k (-t) + t
    h = w = 64
    ps, st_, px, py = 8, 8, 24, 32
    c3 = 0.3
    x0, y0 = px + 3.5 + 2, py + 3.5 + 2  # saddle 2 px off the patch centre: contraction 0.60
    c = (5.0 + c3 * x0 * y0, -c3 * y0, -c3 * x0, c3)
    t = np.array([0.8, 0.45])
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    Y, X = np.mgrid[py:py + ps, px:px + ps].astype(float)
    G = np.stack([(c[1] + c[3] * Y).ravel(), (c[2] + c[3] * X).ravel()], 1)
    M = ps * ps * np.linalg.solve(G.T @ G, np.outer(G.mean(0), G.mean(0)))
    assert 0.5 < max(abs(np.linalg.eigvals(M))) < 0.7
    k_idx = _patch_index(w, ps, st_, px, py)
    errs = [-t]
    for _ in range(60):
        errs.append(M @ errs[-1])
    steps = [np.linalg.norm(errs[k - 1] - errs[k]) for k in range(1, 61)]
    for kwant in (1, 2, 5, 12):
        eps = float(np.sqrt(steps[kwant - 1] * steps[kwant]))  # between the steps of k and k + 1
        kstop = next(k for k in range(1, 61) if steps[k - 1] <= eps)
        assert kstop == kwant + 1
        u, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 60, term_eps=eps)
        assert np.abs(u.reshape(-1, 2)[k_idx] - t - errs[kstop]).max() < 1e-11, (eps, kstop)
    # off: the fixed count; a huge threshold: exactly one step
    a, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 7)
    b, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 7, term_eps=0.0)
    assert np.array_equal(a, b)
    one, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 1)
    big, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 50, term_eps=1e9)
    assert np.array_equal(one, big)


# ---- the converged search of the differentiable form's implicit gradient ----

def test_polished_search_finds_the_exact_translation_of_a_bilinear_scene():
    # g(u) = sum S' (w~ - T) vanishes exactly at u = t on a bilinear image; Newton from any
    # nearby start lands there, wherever the frozen increment left the patch
    h = w = 48
    c3 = 0.3
    c = (5.0 + c3 * 20 * 21, -c3 * 21, -c3 * 20, c3)
    t = np.array([0.7, -0.4])
    I0, I1, gx, gy = _bilinear_scene(h, w, c, t)
    ps, st_ = 8, 8
    n = oracle.grid_n(w, ps, st_) ** 2
    g = np.random.default_rng(61)
    frozen = t + g.uniform(-0.3, 0.3, (n, 2))
    u, _, st = oracle.search_level(I0, gx, gy, I1, ps, st_, 0, frozen=frozen, polish=50)
    inner = [_patch_index(w, ps, st_, px, py) for px in (8, 16, 24, 32) for py in (8, 16, 24, 32)]
    assert np.abs(u.reshape(-1, 2)[inner] - t).max() < 1e-12
    # one degree of freedom: the scalar root in u with v held; a horizontal translation of the
    # same scene is found exactly and v keeps its start
    I1h = _bilinear_scene(h, w, c, (t[0], 0.0))[1]
    fz1 = np.stack([t[0] + g.uniform(-0.3, 0.3, n), np.zeros(n)], -1)
    u1, _, _ = oracle.search_level(I0, gx, gy, I1h, ps, st_, 0, frozen=fz1, polish=50, dof=1)
    assert np.abs(u1.reshape(-1, 2)[inner, 0] - t[0]).max() < 1e-12 and (u1[..., 1] == 0.0).all()
    # a zero increment stands for a patch that did not move: it stays at u_init
    z = frozen.copy()
    z[inner[0]] = 0.0
    u2, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 0, frozen=z, polish=50)
    assert np.array_equal(u2.reshape(-1, 2)[inner[0]], [0.0, 0.0])


def test_polished_search_equals_the_long_fixed_point_iteration():
    # the root of g is the fixed point of the update: where 20000 plain iterations have settled,
    # Newton from a 30-iteration start reaches the same flow
    g = np.random.default_rng(62)
    h, w = 40, 48
    I0 = ndimage.gaussian_filter(g.standard_normal((h, w)), 2.0) * 40 + 120
    I1 = ndimage.shift(I0, (0.35, -0.6), order=3, mode="nearest")
    gx, gy = oracle.sobel(I0)
    ps, st_ = 8, 4
    long_a, _, sa = oracle.search_level(I0, gx, gy, I1, ps, st_, 20000)
    long_b, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 20001)
    short, ui, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 30)
    pol, _, _ = oracle.search_level(I0, gx, gy, I1, ps, st_, 0, frozen=(short - ui).reshape(-1, 2), polish=100)
    settled = (np.abs(long_a - long_b).max(-1) < 1e-12) & (sa == 0)
    assert settled.mean() > 0.8
    assert np.abs(pol - long_a)[settled].max() < 1e-9
