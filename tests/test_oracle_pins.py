"""Pins of the CPU oracle to things other than itself (CPU only).

Each test checks an oracle step against what the paper or the mathematics fixes:
hand-worked examples (tests/golden), closed forms, invariants, special cases that
reduce to a library routine, and brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cfg_for(tile=16, radius=4, **kw):
    from paper_1504_01441_b300 import synth
    return synth.method_params(tile, radius, **kw)


def read_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# --------------------------------------------------------------------- a1
def test_ratio_lut_matches_hand_worked_table(orc):
    for num, den, v, want in read_rows("ratio_lut.txt"):
        num, den, v, want = int(num), int(den), int(v), int(want)
        ref = np.array([v], np.uint8)
        src = np.array([17], np.uint8)
        rn, sn = orc.normalize_ratio(ref, src, num, den)          # reference is darker
        assert rn[0] == want and sn[0] == 17
        rn, sn = orc.normalize_ratio(src, ref, den, num)          # source is darker
        assert sn[0] == want and rn[0] == 17


def test_ratio_one_is_identity(orc):
    rng = np.random.default_rng(0)
    a = rng.integers(0, 256, 1000, dtype=np.uint8)
    b = rng.integers(0, 256, 1000, dtype=np.uint8)
    rn, sn = orc.normalize_ratio(a, b, 1, 1)
    assert np.array_equal(rn, a) and np.array_equal(sn, b)


def test_histeq_uniform_ramp_is_identity(orc):
    img = np.tile(np.arange(256, dtype=np.uint8), 7)
    assert np.array_equal(orc.histeq_lut(img), np.arange(256))


def test_histeq_against_numpy_cdf(orc):
    rng = np.random.default_rng(1)
    for _ in range(5):
        img = np.clip(rng.normal(60, 25, 5000), 0, 255).astype(np.uint8)
        cdf = np.cumsum(np.bincount(img, minlength=256))
        cmin = cdf[img.min()]
        den = img.size - cmin
        want = np.floor((np.maximum(cdf - cmin, 0) * 255 + den // 2) / den).astype(int)
        assert np.array_equal(orc.histeq_lut(img), want)


def test_histeq_constant_frame_maps_to_itself(orc):
    assert np.array_equal(orc.histeq_lut(np.full(100, 77, np.uint8)), np.arange(256))


# --------------------------------------------------------------------- a2
def test_paper_constants_in_defaults():
    c = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    p = cfg_for()
    assert p["levels_max"] == c["levels_max"]
    assert p["min_level_size"] == c["min_level_size_px"]
    assert 2 * p["patch_half"] + 1 == c["patch_side"]
    assert p["sigma_s"] == c["sigma_s"]
    assert max(1, 32 // 16) == 32 * c["candidate_grid_spacing_fraction_of_tile"]


@pytest.mark.parametrize("w,h,L", [(2592, 1944, 5), (640, 480, 3), (199, 400, 1), (200, 200, 2),
                                   (3200, 1600, 5), (4000, 3000, 5), (50, 50, 1), (400, 200, 2)])
def test_level_count(orc, w, h, L):
    # Sec. 2.6: up to 5 levels, stop before a level falls below 100 px in either side
    assert orc.num_levels(w, h, 5, 100) == L


@pytest.mark.parametrize("shape", [(5, 7), (6, 9), (8, 8), (1, 3)])
def test_downsample_brute_force(orc, shape):
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, shape, dtype=np.uint8)
    h, w = shape
    want = np.zeros((h // 2, w // 2), np.int64)
    for y in range(h // 2):
        for x in range(w // 2):
            s = int(img[2 * y, 2 * x]) + int(img[2 * y, 2 * x + 1]) + int(img[2 * y + 1, 2 * x]) + \
                int(img[2 * y + 1, 2 * x + 1])
            want[y, x] = math.floor(s / 4 + 0.5)
    assert np.array_equal(orc.downsample(img), want)


# --------------------------------------------------------------------- a3
def _quadrant_sums_bruteforce(img, x, y, q):
    pad = q + 2
    p = np.pad(img.astype(np.int64), pad, mode="edge")
    X, Y = x + pad, y + pad
    tl = p[Y - q:Y, X - q:X].sum()
    tr = p[Y - q:Y, X:X + q].sum()
    br = p[Y:Y + q, X:X + q].sum()
    bl = p[Y:Y + q, X - q:X].sum()
    return [tl, tr, br, bl]


def test_cornerness_brute_force(orc):
    rng = np.random.default_rng(3)
    img = (rng.random((40, 50)) * 255).astype(np.uint8)
    for _ in range(60):
        x, y = int(rng.integers(-3, 53)), int(rng.integers(-3, 43))
        S = _quadrant_sums_bruteforce(img, x, y, 10)
        d = [abs(S[(j + 1) % 4] - S[j]) for j in range(4)]
        sums, c, m = orc.cornerness(img, x, y, 10)
        assert sums == S and c == sum(d) and m == min(d)


def test_x_junction_cornerness_closed_form(orc):
    # checkerboard X-junction: quadrants 0/255/0/255 -> C = 4 * 255 * q^2, min = 255 q^2
    img = np.zeros((64, 64), np.uint8)
    img[:32, 32:] = 255
    img[32:, :32] = 255
    _, c, m = orc.cornerness(img, 32, 32, 10)
    assert c == 4 * 255 * 100 and m == 255 * 100
    cxy, valid, score = orc.pick_corners(img, cfg_for(tile=64))
    assert valid[0] == 1 and tuple(cxy[0]) == (32, 32) and score[0] == 102000


def test_edge_and_flat_rejected_l_corner_found_off_apex(orc):
    cfg = cfg_for(tile=64)
    edge = np.zeros((64, 64), np.uint8)
    edge[:, 32:] = 200                       # straight edge: two quadrant pairs equal -> min 0
    flat = np.full((64, 64), 90, np.uint8)   # flat tile: no corner (Sec. 2.2)
    for img in (edge, flat):
        _, valid, _ = orc.pick_corners(img, cfg)
        assert valid[0] == 0
    # corner of a bright block: at the apex three quadrants are equal, so the literal
    # Eq. 2 gives min activity 0 there; a grid candidate displaced into the block sees
    # four different quadrant means and is kept.
    lcorner = np.zeros((64, 64), np.uint8)
    lcorner[32:, 32:] = 200
    _, _, m = orc.cornerness(lcorner, 32, 32, 10)
    assert m == 0
    cxy, valid, _ = orc.pick_corners(lcorner, cfg)
    assert valid[0] == 1 and cxy[0, 0] > 32 and cxy[0, 1] > 32


def test_pick_corners_brute_force_with_tie_break(orc):
    rng = np.random.default_rng(4)
    cfg = cfg_for(tile=16)
    img = np.kron(rng.integers(0, 2, (12, 12)) * 200, np.ones((8, 8), np.int64)).astype(np.uint8)
    img = np.clip(img.astype(int) + rng.integers(0, 3, img.shape), 0, 255).astype(np.uint8)
    h, w = img.shape
    cxy, valid, score = orc.pick_corners(img, cfg)
    T, K, s = 16, 4, 1
    t = 0
    for ty in range(h // T):
        for tx in range(w // T):
            cx, cy = tx * T + T // 2, ty * T + T // 2
            best, pos = -1, None
            for j in range(-K, K + 1):          # row-major: offset j outer, i inner
                for i in range(-K, K + 1):
                    S = _quadrant_sums_bruteforce(img, cx + s * i, cy + s * j, 10)
                    d = [abs(S[(k + 1) % 4] - S[k]) for k in range(4)]
                    if min(d) > 200 and sum(d) > best:
                        best, pos = sum(d), (cx + s * i, cy + s * j)
            assert valid[t] == (pos is not None)
            if pos is not None:
                assert tuple(cxy[t]) == pos and score[t] == best
            t += 1


# --------------------------------------------------------------------- a4 + a5
def _ssd_bruteforce(ref, src, p, c, R, hp):
    pad = R + hp + 40
    rp = np.pad(ref.astype(np.int64), pad, mode="edge")
    sp = np.pad(src.astype(np.int64), pad, mode="edge")
    px, py = p[0] + pad, p[1] + pad
    patch = rp[py - hp:py + hp + 1, px - hp:px + hp + 1]
    best = None
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            qx, qy = c[0] + dx + pad, c[1] + dy + pad
            cost = int(((patch - sp[qy - hp:qy + hp + 1, qx - hp:qx + hp + 1]) ** 2).sum())
            key = (cost, (dy + R) * (2 * R + 1) + (dx + R))
            if best is None or key < best[0]:
                best = (key, (c[0] + dx, c[1] + dy))
    return best[1], best[0][0]


def test_identity_pair_zero_displacement(orc, vga_stack):
    cfg = cfg_for()
    ref = vga_stack.ref.y
    cxy, valid, _ = orc.pick_corners(ref, cfg)
    ctr, mxy, cost = orc.search(ref, ref, np.eye(3), cfg, cxy, valid)
    v = valid.astype(bool)
    assert v.sum() > 100
    assert np.array_equal(mxy[v], cxy[v]) and np.all(cost[v] == 0)


@pytest.mark.parametrize("d", [(3, -2), (-4, 4), (0, 1), (-1, -3)])
def test_integer_shift_recovered_exactly(orc, vga_stack, d):
    cfg = cfg_for()
    big = vga_stack.ref.y
    ref = big[20:260, 20:340]
    src = big[20 - d[1]:260 - d[1], 20 - d[0]:340 - d[0]]   # src(q) = ref(q - d)
    cxy, valid, _ = orc.pick_corners(ref, cfg)
    ctr, mxy, cost = orc.search(ref, src, np.eye(3), cfg, cxy, valid)
    h, w = ref.shape
    margin = 10 + 4 + 4
    inner = valid.astype(bool) & (cxy[:, 0] >= margin) & (cxy[:, 0] < w - margin) & \
        (cxy[:, 1] >= margin) & (cxy[:, 1] < h - margin)
    assert inner.sum() > 50
    assert np.array_equal(mxy[inner] - cxy[inner], np.tile(np.array(d), (inner.sum(), 1)))
    assert np.all(cost[inner] == 0)


def test_search_brute_force_tiny(orc):
    rng = np.random.default_rng(5)
    ref = rng.integers(0, 256, (48, 48), dtype=np.uint8)
    src = np.clip(np.roll(ref, (1, -2), (0, 1)).astype(int) + rng.integers(-6, 7, ref.shape),
                  0, 255).astype(np.uint8)
    cfg = cfg_for(tile=16, radius=3)
    H = np.array([[1.001, 0.002, 0.01], [-0.003, 0.999, -0.02], [0.001, -0.002, 1.0]])
    cxy, valid, _ = orc.pick_corners(ref, cfg)
    ctr, mxy, cost = orc.search(ref, src, H, cfg, cxy, valid)
    for t in range(valid.size):
        if not valid[t]:
            continue
        m, c = _ssd_bruteforce(ref, src, cxy[t], ctr[t], 3, 10)
        assert tuple(mxy[t]) == m and cost[t] == c


def test_search_tie_break_lowest_index(orc):
    # constant source: every displacement costs the same -> d = (-R, -R)
    img = np.zeros((64, 64), np.uint8)
    img[:32, 32:] = 255
    img[32:, :32] = 255
    src = np.full((64, 64), 50, np.uint8)
    cfg = cfg_for(tile=64, radius=5)
    cxy, valid, _ = orc.pick_corners(img, cfg)
    ctr, mxy, cost = orc.search(img, src, np.eye(3), cfg, cxy, valid)
    assert tuple(mxy[0] - ctr[0]) == (-5, -5)


def test_search_center_rounding_and_clamp(orc):
    # a pure translation in normalized units: +1.5 px and -2.5 px at level width 100
    w, h = 100, 80
    H = np.array([[1, 0, 2 * 1.5 / w], [0, 1, 2 * -2.5 / w], [0, 0, 1.0]])
    xs, ys, ok = orc.project(H, 10, 20, w, h)
    assert ok and abs(xs - 11.5) < 1e-12 and abs(ys - 17.5) < 1e-12
    assert orc.search_center(H, 10, 20, w, h) == (12, 18)       # floor(x + 0.5)
    assert orc.search_center(H, 99, 0, w, h) == (99, 0)         # clamped into the level
    Hbad = np.array([[1, 0, 0], [0, 1, 0], [0, 0, -1.0]])       # denominator < 0 -> corner
    assert orc.search_center(Hbad, 7, 9, w, h) == (7, 9)


def test_known_similarity_recovered_within_one_pixel(orc):
    from paper_1504_01441_b300 import synth
    spec = synth.StackSpec(480, 360, ratios=((1, 1),), noise_sigma=0.0, field_amp=0.0, movers=0,
                           chroma=False, shift_px=3.0)
    st = synth.make_stack(spec, 77)
    cfg = cfg_for()
    m = orc.match(st.ref.y, st.srcs[0].y, cfg)
    gx, gy = st.gt[0]
    keep = orc.mask_to_bool(m["bits"], m["valid"].size)
    c, q = m["corner_xy"][keep], m["match_xy"][keep]
    err = np.hypot(q[:, 0] - gx[c[:, 1], c[:, 0]], q[:, 1] - gy[c[:, 1], c[:, 0]])
    assert keep.sum() > 100 and np.percentile(err, 95) <= 1.0


# --------------------------------------------------------------------- a6
def test_splitmix64_published_values(orc):
    for k, want in read_rows("splitmix64_seed0.txt"):
        assert orc.splitmix64_at(0, int(k)) == int(want, 16)


def test_weed_sample_distinct_in_range(orc):
    for it in range(200):
        pick = orc.weed_sample(12345, it, 37)
        assert pick is not None and len(set(pick)) == 4 and all(0 <= j < 37 for j in pick)
    assert orc.weed_sample(1, 0, 3) is None     # fewer than 4 candidates


def _two_plane_scene(rng, n_per=60, outlier_frac=0.2, w=640, h=480):
    # two planes seen under different homographies + outliers (toy scene of Sec. 2.3)
    Ha = np.array([[1.01, 0.004, 0.012], [-0.003, 0.995, -0.008], [0.0, 0.0, 1.0]])
    Hb = np.array([[0.98, -0.01, -0.02], [0.012, 1.02, 0.015], [0.0, 0.0, 1.0]])
    pts, mts, lab = [], [], []
    for H, x0 in ((Ha, 20), (Hb, 340)):
        for _ in range(n_per):
            x, y = int(rng.integers(x0, x0 + 280)), int(rng.integers(20, h - 20))
            xn, yn = (2 * x - (w - 1)) / w, (2 * y - (h - 1)) / w
            v = H @ np.array([xn, yn, 1.0])
            u = (v[0] / v[2] * w + (w - 1)) / 2
            vv = (v[1] / v[2] * w + (h - 1)) / 2
            pts.append((x, y))
            mts.append((int(round(u)), int(round(vv))))
            lab.append(0)
    n_out = int(outlier_frac * len(pts) / (1 - outlier_frac))
    for _ in range(n_out):
        x, y = int(rng.integers(20, w - 20)), int(rng.integers(20, h - 20))
        pts.append((x, y))
        mts.append((x + int(rng.integers(8, 20)) * int(rng.choice([-1, 1])),
                    y + int(rng.integers(8, 20)) * int(rng.choice([-1, 1]))))
        lab.append(1)
    return np.array(pts, np.int32), np.array(mts, np.int32), np.array(lab)


def test_weed_toy_scene_two_planes(orc):
    rng = np.random.default_rng(6)
    p, q, lab = _two_plane_scene(rng)
    # delta sized as Sec. 2.3 describes the toy scene: a homography from one plane gathers
    # that plane's support (60 of 150 matches), a mixed sample only a small set
    cfg = cfg_for(weed_delta_div=3)
    valid = np.ones(len(p), np.uint8)
    bits, acc = orc.weed(p, q, valid, 640, 480, cfg, seed=99)
    keep = orc.mask_to_bool(bits, len(p))
    assert acc > 0
    assert keep[lab == 0].all(), "every point on a plane is an inlier of some accepted H"
    assert not keep[lab == 1].any(), "outliers are excluded"


@pytest.mark.parametrize("splits", [[256], [100, 412], [1, 2, 3, 506], list(range(0, 512, 64))[1:]])
def test_weed_split_union_equals_single_run(orc, splits):
    # Sec. 2.3: n instances of 1/n of the iterations, merged by union == one run
    rng = np.random.default_rng(7)
    p, q, lab = _two_plane_scene(rng, outlier_frac=0.35)
    cfg = cfg_for(weed_iters=512)
    valid = (rng.random(len(p)) > 0.1).astype(np.uint8)
    one, _ = orc.weed(p, q, valid, 640, 480, cfg, seed=5)
    bits = orc.mask_words(len(p))
    edges = [0] + list(splits) + [512]
    for a, b in reversed(list(zip(edges[:-1], edges[1:]))):
        orc.weed(p, q, valid, 640, 480, cfg, seed=5, iter_begin=a, iter_end=b, bits=bits)
    assert np.array_equal(bits, one)


# --------------------------------------------------------------------- a7
def test_solve8_against_numpy(orc):
    rng = np.random.default_rng(8)
    for _ in range(20):
        A = rng.normal(size=(8, 8)) + 4 * np.eye(8)
        b = rng.normal(size=8)
        x, st = orc.solve8(A, b)
        assert st == 0 and np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)
    x, st = orc.solve8(np.zeros((8, 8)), np.ones(8))
    assert st == 1


def test_fit_exact_from_four_integer_correspondences(orc):
    # q = p + (5, -3) in pixels maps integers to integers: translation in normalized units
    w, h = 200, 150
    p = np.array([[10, 10], [180, 20], [30, 140], [150, 120]], np.int32)
    q = p + np.array([5, -3], np.int32)
    bits = np.array([0xF], np.uint32)
    H, st = orc.fit_homography(p, q, bits, w, h)
    want = np.array([[1, 0, 2 * 5 / w], [0, 1, 2 * -3 / w], [0, 0, 1]])
    assert st == 0 and np.abs(H - want).max() < 1e-12


def test_fit_integer_affine_many_points(orc):
    # q = 2p - (w-1)/2... i.e. a zoom by 2 about the centre in centred coordinates
    rng = np.random.default_rng(9)
    w, h = 301, 201
    xc = 2 * rng.integers(60, 240, 40) - (w - 1)
    yc = 2 * rng.integers(50, 150, 40) - (h - 1)
    p = np.stack([(xc + (w - 1)) // 2, (yc + (h - 1)) // 2], 1).astype(np.int32)
    # x_c' = 2 x_c -> pixel u = (2 x_c + w - 1) / 2 is an integer since x_c is even here
    q = np.stack([(2 * xc + (w - 1)) // 2, (2 * yc + (h - 1)) // 2], 1).astype(np.int32)
    bits = np.array([(1 << 32) - 1, (1 << 8) - 1], np.uint32)
    H, st = orc.fit_homography(p, q, bits, w, h)
    assert st == 0 and np.abs(H - np.diag([2.0, 2.0, 1.0])).max() < 1e-12


def test_fit_real_recovers_projective_homography(orc):
    rng = np.random.default_rng(10)
    Ht = np.array([[1.02, -0.01, 0.03], [0.015, 0.99, -0.02], [0.05, -0.03, 1.0]])
    P = rng.uniform(-1, 1, (50, 2))
    V = (Ht @ np.c_[P, np.ones(50)].T).T
    Q = V[:, :2] / V[:, 2:]
    H, st = orc.fit_homography_real(P, Q)
    assert st == 0 and np.abs(H - Ht).max() < 1e-10


def test_fit_normalized_coordinates_agree_across_levels(orc):
    # the same physical translation seen at level 0 (2d px) and level 1 (d px) gives one H
    rng = np.random.default_rng(11)
    w0, h0 = 400, 300
    d = np.array([3, -2])
    p1 = rng.integers(20, 180, (30, 2)).astype(np.int32)
    p1[:, 1] = np.minimum(p1[:, 1], 130)
    H1, _ = orc.fit_homography(p1, p1 + d, np.array([(1 << 30) - 1], np.uint32), w0 // 2, h0 // 2)
    p0 = 2 * p1
    H0, _ = orc.fit_homography(p0, p0 + 2 * d, np.array([(1 << 30) - 1], np.uint32), w0, h0)
    assert np.abs(H1 - H0).max() < 1e-12


def test_fit_too_few_keeps_previous(orc):
    Hp = np.array([[1.0, 0.1, 0.0], [0.0, 1.0, 0.2], [0.0, 0.0, 1.0]])
    p = np.array([[1, 1], [5, 5], [9, 2]], np.int32)
    H, st = orc.fit_homography(p, p, np.array([7], np.uint32), 50, 50, Hp)
    assert st == 1 and np.array_equal(H, Hp)


# --------------------------------------------------------------------- a8
def test_dt_sigmas_sum_of_variances(orc):
    # the iteration sigmas of the domain transform add up (in variance) to sigma_s
    for N in (1, 2, 3, 5):
        s = [orc.dt_sigma(400.0, N, i) for i in range(N)]
        assert abs(sum(v[0] ** 2 for v in s) - 400.0 ** 2) < 1e-6
        assert all(abs(a - math.exp(-math.sqrt(2) / sg)) < 1e-15 for sg, a in s)
        assert all(s[i][0] > s[i + 1][0] for i in range(N - 1))


def _impulse_closed_form(a, L, m):
    """One forward + backward pass of J[n] = (1-a) x[n] + a J[n-1] (J[0] = x[0]) on an impulse
    at m, summed as geometric series.

    forward:  f[n] = 0 (n < m), f[m] = 1 if m == 0 else 1-a, f[n] = a^(n-m) f[m] (n > m)
    backward: K[n] = sum_{k=n}^{L-2} (1-a) a^(k-n) f[k] + a^(L-1-n) f[L-1]
    """
    fm = 1.0 if m == 0 else 1.0 - a
    out = np.zeros(L)
    for n in range(m, L):
        k = L - 1 - n
        out[n] = (1 - a) * fm * a ** (n - m) * (1 - a ** (2 * k)) / (1 - a * a) + \
            a ** k * fm * a ** (L - 1 - m)
    for n in range(m):
        out[n] = a ** (m - n) * out[m]
    return out


@pytest.mark.parametrize("m", [0, 7, 40])
def test_dt_one_dimensional_impulse_closed_form(orc, m):
    L = 64
    x = np.zeros((1, L))
    x[0, m] = 1.0
    g = np.zeros((1, L), np.uint8)           # constant guide: the plain exponential smoother
    (y,) = orc.dt_filter([x], g, 40.0, 0.5, 1)
    a = orc.dt_sigma(40.0, 1, 0)[1]
    want = _impulse_closed_form(a, L, m)
    assert np.allclose(y[0], want, rtol=1e-12, atol=1e-15)


def test_dt_three_pixel_worked_example(orc):
    # tests/golden/dt_three_pixel.txt
    ss, sr = 30.0, 0.5
    (y,) = orc.dt_filter([np.array([[0.0, 0.0, 1.0]])], np.array([[0, 0, 255]], np.uint8), ss, sr, 1)
    a = orc.dt_sigma(ss, 1, 0)[1]
    w2 = a ** (1 + ss / sr)
    assert np.allclose(y[0], [a * w2 * (1 - w2), w2 * (1 - w2), 1 - w2], rtol=1e-12, atol=0)


def test_dt_constant_guide_is_separable(orc):
    h, w = 23, 31
    x = np.zeros((h, w))
    x[9, 13] = 1.0
    g = np.full((h, w), 77, np.uint8)
    (y2,) = orc.dt_filter([x], g, 25.0, 0.5, 3)
    # per iteration the 2-D response of an impulse is the outer product of the 1-D ones
    cx = np.zeros((1, w)); cx[0, 13] = 1.0
    cy = np.zeros((1, h)); cy[0, 9] = 1.0
    hx = cx
    vy = cy
    for i in range(3):
        sg, a = orc.dt_sigma(25.0, 3, i)
        # run one iteration with this iteration's a: use a 1-iteration filter whose sigma_s
        # reproduces sigma_i (sigma_s * sqrt(3) / sqrt(3) = sigma_s)
        (hx,) = orc.dt_filter([hx], np.zeros((1, w), np.uint8), sg, 0.5, 1)
        (vy,) = orc.dt_filter([vy], np.zeros((1, h), np.uint8), sg, 0.5, 1)
    assert np.allclose(y2, np.outer(vy[0], hx[0]), rtol=1e-10, atol=1e-18)


def test_flow_constant_residual_is_preserved(orc, vga_stack):
    # all corners carry the same residual rho0 -> F == rho0 wherever N~ > 0 (normalization)
    cfg = cfg_for()
    ref = vga_stack.ref.y
    cxy, valid, _ = orc.pick_corners(ref, cfg)
    n = valid.size
    q = cxy + np.array([2, -1], np.int32)
    bits = orc.mask_words(n)
    for t in np.nonzero(valid)[0]:
        bits[t >> 5] |= np.uint32(1 << (t & 31))
    fu, fv, nt = orc.flow(ref, cxy, q, bits, np.eye(3), cfg)
    ok = nt >= cfg["flow_eps"]
    assert ok.mean() > 0.99
    assert np.abs(fu[ok] - 2.0).max() < 1e-9 and np.abs(fv[ok] + 1.0).max() < 1e-9


def test_flow_identity_pair_is_zero(orc, vga_stack):
    cfg = cfg_for()
    ref = vga_stack.ref.y
    m = orc.match(ref, ref, cfg)
    assert np.abs(m["H0"] - np.eye(3)).max() < 1e-12
    fu, fv, nt = orc.flow(ref, m["corner_xy"], m["match_xy"], m["bits"], m["H0"], cfg)
    assert np.abs(fu).max() < 1e-9 and np.abs(fv).max() < 1e-9


# --------------------------------------------------------------------- a9
def test_warp_identity_is_exact(orc, small_yuv_stack):
    s = small_yuv_stack.srcs[0]
    z = np.zeros(s.y.shape)
    oy, ou, ov = orc.warp(s.y, s.u, s.v, np.eye(3), z, z)
    assert np.array_equal(oy, s.y) and np.array_equal(ou, s.u) and np.array_equal(ov, s.v)


def test_warp_integer_flow_is_exact_shift(orc, small_yuv_stack):
    s = small_yuv_stack.srcs[0]
    h, w = s.y.shape
    oy, _, _ = orc.warp(s.y, None, None, np.eye(3), np.full((h, w), 3.0), np.full((h, w), -2.0))
    assert np.array_equal(oy[2:, :w - 3], s.y[:h - 2, 3:])


def test_warp_reproduces_linear_ramp(orc):
    rng = np.random.default_rng(12)
    w, h = 64, 48
    ys, xs = np.mgrid[0:h, 0:w]
    src = (xs + 2 * ys).astype(np.uint8)          # max 63 + 94 = 157
    from paper_1504_01441_b300 import synth
    H = synth.random_homography(rng, scale=0.01, shift_n=0.01, persp=0.0005)
    fu, fv = synth.random_flow(rng, w, h, 1.5)
    oy, _, _ = orc.warp(src, None, None, H, fu, fv)
    # sample positions
    xn, yn = (2 * xs - (w - 1)) / w, (2 * ys - (h - 1)) / w
    V = np.einsum("ij,jhw->ihw", H, np.stack([xn, yn, np.ones_like(xn)]))
    mx = (V[0] / V[2] * w + (w - 1)) / 2 + fu
    my = (V[1] / V[2] * w + (h - 1)) / 2 + fv
    inside = (mx >= 0) & (mx <= w - 1) & (my >= 0) & (my <= h - 1)
    assert inside.mean() > 0.7
    assert np.abs(oy[inside] - (mx + 2 * my)[inside]).max() < 1e-9


def test_bilinear_equal_taps_exact(orc):
    img = np.full((4, 4), 255, np.uint8)
    for x, y in [(0.3, 1.7), (2.999, 0.001), (1.5, 1.5)]:
        assert orc.bilinear(img, x, y) == 255.0


# --------------------------------------------------------------------- a10
def test_ssim_identical_is_one(orc):
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 255, (30, 40))
    assert np.abs(orc.ssim(x, x) - 1.0).max() < 1e-12


def test_ssim_against_scipy_gaussian_filter(orc):
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(14)
    x = rng.uniform(0, 255, (37, 41))
    y = np.clip(x + rng.normal(0, 20, x.shape), 0, 255)
    f = lambda a: gaussian_filter(a, 1.5, mode="nearest", truncate=10.0 / 3.0)
    mx, my = f(x), f(y)
    vx, vy, cxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    want = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    assert np.abs(orc.ssim(x, y) - want).max() < 1e-9


def test_ghost_mask_ratio_gain_and_clamp(orc):
    rng = np.random.default_rng(15)
    ref_n = rng.integers(0, 200, (30, 30)).astype(np.uint8)
    # a source 4x darker (gain 4 brings it back): identical after normalization -> Q == 1
    q = orc.ghost_mask(ref_n, ref_n / 4.0, mode=0, gain=4.0)
    assert np.abs(q - 1).max() < 1e-12
    q = orc.ghost_mask(ref_n, 255.0 - ref_n, mode=0, gain=1.0)
    assert q.min() >= 0.0


def test_ghost_mask_histeq_identity_lut_equals_ratio_mode(orc):
    # with the identity LUT the equalization branch maps a warped value z in [0, 255] to z,
    # which the ratio branch with gain 1 does as well
    rng = np.random.default_rng(21)
    ref_n = rng.integers(0, 256, (26, 31)).astype(np.uint8)
    wy = rng.uniform(0, 255, (26, 31))
    wy[0, :5] = [0.0, 255.0, 254.75, 0.5, 127.0]
    q1 = orc.ghost_mask(ref_n, wy, mode=1, src_lut=np.arange(256))
    q0 = orc.ghost_mask(ref_n, wy, mode=0, gain=1.0)
    assert np.array_equal(q1, q0)


def test_ghost_mask_histeq_interpolates_the_lut(orc):
    # lut[v] = min(2v, 255); warped values k + 0.25 must enter SSIM as the linear
    # interpolation lut[k] + 0.25 (lut[k+1] - lut[k]), written out by hand:
    # 2k + 0.5 below 127, 254.25 between 127 and 128 (254 -> 255), 255 from 128 on
    rng = np.random.default_rng(22)
    h, w = 24, 28
    k = rng.integers(0, 255, (h, w))
    k[0, :3] = [126, 127, 128]
    wy = k + 0.25
    lut = np.minimum(2 * np.arange(256), 255)
    by_hand = np.where(k < 127, 2 * k + 0.5, np.where(k == 127, 254.25, 255.0))
    ref_n = rng.integers(0, 256, (h, w)).astype(np.uint8)
    q = orc.ghost_mask(ref_n, wy, mode=1, src_lut=lut)
    want = np.maximum(orc.ssim(ref_n.astype(float), by_hand), 0.0)
    assert np.abs(q - want).max() < 1e-12
    # a nearest-level reading (lut at the rounded value) gives another mask
    nearest = np.maximum(orc.ssim(ref_n.astype(float), lut[np.rint(wy).astype(int)].astype(float)),
                         0.0)
    assert np.abs(q - nearest).max() > 1e-3


# --------------------------------------------------------------------- a11
def test_well_exposedness_values(orc):
    assert orc.well_exposedness(127.5) == 1.0
    assert abs(orc.well_exposedness(0.0) - math.exp(-0.25 / 0.08)) < 1e-15
    assert abs(orc.well_exposedness(255.0) - math.exp(-0.25 / 0.08)) < 1e-15


def test_merge_closed_form_exposure_scaled_pair(orc):
    # noiseless, unclipped Z_src = r Z_ref with identity geometry -> E = Z_ref for any weights
    rng = np.random.default_rng(16)
    h, w = 20, 24
    ref_y = rng.integers(1, 63, (h, w)).astype(np.uint8)
    ref_u = rng.integers(100, 156, (h // 2, w // 2)).astype(np.uint8)
    ref_v = rng.integers(100, 156, (h // 2, w // 2)).astype(np.uint8)
    wy = 4.0 * ref_y
    wu = 128 + 4.0 * (ref_u.astype(float) - 128)
    wv = 128 + 4.0 * (ref_v.astype(float) - 128)
    q = rng.uniform(0, 1, (h, w))
    oy, ou, ov = orc.merge(ref_y, ref_u, ref_v, [(wy, wu, wv)], [q], [4.0])
    assert np.abs(oy - ref_y).max() < 1e-12
    assert np.abs(ou - (ref_u - 128.0)).max() < 1e-12 and np.abs(ov - (ref_v - 128.0)).max() < 1e-12


def test_merge_saturated_or_ghosted_source_gives_reference(orc):
    rng = np.random.default_rng(17)
    h, w = 10, 12
    ref_y = rng.integers(0, 256, (h, w)).astype(np.uint8)
    sat = np.full((h, w), 255.0)
    oy, _, _ = orc.merge(ref_y, None, None, [(sat, None, None)], [np.ones((h, w))], [4.0])
    assert np.abs(oy - ref_y).max() < 1e-12
    oy, _, _ = orc.merge(ref_y, None, None, [(np.full((h, w), 99.0), None, None)],
                         [np.zeros((h, w))], [4.0])
    assert np.abs(oy - ref_y).max() < 1e-12


# --------------------------------------------------------------------- whole path
def test_register_merge_identity_stack(orc, small_yuv_stack):
    from paper_1504_01441_b300 import synth
    s = small_yuv_stack
    cfg = cfg_for()
    out = orc.register_merge(s.ref, [s.ref], [(1, 1)], cfg)
    assert np.abs(out["H0"][0] - np.eye(3)).max() < 1e-12
    assert np.abs(out["y"] - s.ref.y).max() < 1e-9
    assert np.abs(out["u"] - (s.ref.u - 128.0)).max() < 1e-9


def test_register_merge_improves_on_homography(orc, vga_stack):
    cfg = cfg_for()
    s = vga_stack
    out = orc.register_merge(s.ref, s.srcs, s.ratios, cfg, want_intermediates=True)
    h, w = s.ref.y.shape
    H = out["H0"][0]
    ys, xs = np.mgrid[0:h, 0:w].astype(float)
    xn, yn = (2 * xs - (w - 1)) / w, (2 * ys - (h - 1)) / w
    V = np.einsum("ij,jhw->ihw", H, np.stack([xn, yn, np.ones_like(xn)]))
    hx, hy = (V[0] / V[2] * w + (w - 1)) / 2, (V[1] / V[2] * w + (h - 1)) / 2
    gx, gy = s.gt[0]
    epe_h = np.hypot(hx - gx, hy - gy).mean()
    epe = np.hypot(hx + out["flow_u"][0] - gx, hy + out["flow_v"][0] - gy).mean()
    assert epe < epe_h and epe < 1.0


def test_inlier_test_matches_reprojection_distance(orc):
    # the division-free predicate equals "projection within eps pixels" (Sec. 2.3)
    rng = np.random.default_rng(18)
    w, h = 320, 240
    from paper_1504_01441_b300 import synth
    n_checked = 0
    for _ in range(3000):
        H = synth.random_homography(rng, scale=0.05, shift_n=0.05, persp=0.01)
        p = (int(rng.integers(0, w)), int(rng.integers(0, h)))
        xs, ys, ok = orc.project(H, p[0], p[1], w, h)
        q = (int(round(xs + rng.uniform(-3, 3))), int(round(ys + rng.uniform(-3, 3))))
        d2 = (xs - q[0]) ** 2 + (ys - q[1]) ** 2
        if abs(d2 - 1.5 ** 2) < 1e-9:
            continue                         # on the boundary: rounding decides either way
        assert orc.is_inlier(orc.to_scaled(H, w), p, q, w, h, 1.5) == (ok and d2 <= 1.5 ** 2)
        n_checked += 1
    assert n_checked > 2900


@pytest.mark.parametrize("z", [254.0, 253.0, 255.0, 1.0, 0.0, 128.0, 254.5, 0.25])
def test_merge_source_weight_closed_form(orc, z):
    # one pixel, Q = 1, no clip flags (a sample is clipped when its value is 0 or 255):
    # E = (w0 Z0 + w1 Z1/r) / (w0 + w1) -> w1 = w0 (Z0 - E) / (E - Z1/r) must be WE(Z1)
    # strictly inside (0, 255) and 0 at either end
    z0, r = 100, 2.0
    oy, _, _ = orc.merge(np.array([[z0]], np.uint8), None, None, [(np.array([[z]]), None, None)],
                         [np.ones((1, 1))], [r])
    e = oy[0, 0]
    w0 = orc.well_exposedness(float(z0))
    want = orc.well_exposedness(z) if 0.0 < z < 255.0 else 0.0
    if want == 0.0:
        assert abs(e - z0) < 1e-12
    else:
        w1 = w0 * (z0 - e) / (e - z / r)
        assert abs(w1 - want) < 1e-9 * max(want, 1e-3)


def test_bilinear_clipped_brute_force(orc):
    # the taps that carry a nonzero bilinear weight, enumerated from the four weights
    # (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy at positions on the grid, on half and
    # quarter steps, off the image (clamped taps) and at random
    rng = np.random.default_rng(19)
    h, w = 9, 11
    img = rng.integers(1, 255, (h, w)).astype(np.uint8)
    img[rng.random((h, w)) < 0.2] = 255
    img[rng.random((h, w)) < 0.1] = 0
    pts = [(x, y) for x in np.arange(-1.0, w + 0.5, 0.25) for y in np.arange(-1.0, h + 0.5, 0.5)]
    pts += [tuple(p) for p in rng.uniform(-1.0, w, (300, 2))]
    n_true = 0
    for x, y in pts:
        x0, y0 = math.floor(x), math.floor(y)
        fx, fy = x - x0, y - y0
        wts = {(0, 0): (1 - fx) * (1 - fy), (1, 0): fx * (1 - fy), (0, 1): (1 - fx) * fy,
               (1, 1): fx * fy}
        want = any(wt > 0 and img[min(max(y0 + j, 0), h - 1), min(max(x0 + i, 0), w - 1)]
                   in (0, 255) for (i, j), wt in wts.items())
        assert orc.bilinear_clipped(img, x, y) == want, (x, y)
        n_true += want
    assert 0.2 * len(pts) < n_true < 0.9 * len(pts)


def test_merge_half_pixel_shifted_clipped_ramp_gives_reference(orc):
    # Noise-free pair on a linear scene: the reference sees Z_ref(x) = 2x, the source (twice
    # the exposure) sees the scene half a pixel further on, src(q) = min(4q + 2, 255), and
    # is warped back by that half pixel. Where both taps are unclipped the bilinear sample
    # is exactly 4x = r Z_ref; from x = 64 on a tap is 255, so the sample is a clipped
    # measurement and must carry no weight. So E = Z_ref at every pixel (x >= 1; x = 0
    # samples the clamped edge). A value rule alone (clipped only at 255 exactly) would
    # let the sample 254.5 at x = 64 through.
    h, w = 6, 100
    xs = np.tile(np.arange(w), (h, 1))
    ref_y = (2 * xs).astype(np.uint8)
    src_y = np.minimum(4 * xs + 2, 255).astype(np.uint8)
    fu, fv = np.full((h, w), -0.5), np.zeros((h, w))
    wy, _, _, clip = orc.warp(src_y, None, None, np.eye(3), fu, fv, want_clip=True)
    assert wy[0, 64] == 254.5 and clip[0, 64] == 1 and clip[0, 63] == 0
    q = np.ones((h, w))
    oy, _, _ = orc.merge(ref_y, None, None, [(wy, None, None)], [q], [2.0], clips=[clip])
    assert np.abs(oy[:, 1:] - ref_y[:, 1:]).max() <= 1e-12 * 255
    by_value, _, _ = orc.merge(ref_y, None, None, [(wy, None, None)], [q], [2.0])
    assert abs(by_value[0, 64] - 128.0) > 0.01


def test_merge_dark_source_zeros_carry_no_weight(orc):
    # A source a quarter of the reference's exposure, noise-free, identity geometry: where
    # the reference is a multiple of 4 the source is exactly Z_ref / 4; where it is 1-3 the
    # source rounds to 0, a clipped sample. E = Z_ref everywhere.
    rng = np.random.default_rng(20)
    h, w = 16, 20
    ref_y = (4 * rng.integers(1, 63, (h, w))).astype(np.uint8)
    small = rng.random((h, w)) < 0.3
    ref_y[small] = rng.integers(1, 4, int(small.sum()))
    src_y = np.where(small, 0, ref_y // 4).astype(np.uint8)
    z = np.zeros((h, w))
    wy, _, _, clip = orc.warp(src_y, None, None, np.eye(3), z, z, want_clip=True)
    assert np.array_equal(clip.astype(bool), small)
    oy, _, _ = orc.merge(ref_y, None, None, [(wy, None, None)], [np.ones((h, w))], [0.25],
                         clips=[clip])
    assert np.abs(oy - ref_y).max() <= 1e-12 * 255


# --------------------------------------------------------------------- a-L (learned path)
def test_predictor_input_identity_and_integer_shift(orc):
    rng = np.random.default_rng(30)
    ref = rng.integers(0, 256, (24, 40), dtype=np.uint8)
    src = rng.integers(0, 256, (24, 40), dtype=np.uint8)
    x = orc.predictor_input(ref, src, np.eye(3))
    assert np.array_equal(x[..., 0], (ref - 127.5) / 127.5)
    assert np.array_equal(x[..., 1], (src - 127.5) / 127.5)
    # a translation of +3 px in x (normalized 2*3/w) samples src[y, x + 3] exactly
    H = np.eye(3)
    H[0, 2] = 2 * 3 / 40
    x = orc.predictor_input(ref, src, H)
    assert np.allclose(x[:, :37, 1], (src[:, 3:] - 127.5) / 127.5, atol=1e-12)


def test_tile_labels_recover_an_integer_shift(orc):
    rng = np.random.default_rng(31)
    c = cfg_for(16, 4)
    img = np.clip(np.kron(rng.integers(0, 256, (34, 42)), np.ones((4, 4))) +
                  rng.normal(0, 3, (136, 168)), 0, 255).astype(np.uint8)[:128, :160]
    src = np.roll(img, (2, -3), axis=(0, 1))  # src(p + (-3, 2)) = ref(p)
    cxy, valid, _ = orc.pick_corners(img, c)
    _, mxy, _ = orc.search(img, src, np.eye(3), c, cxy, valid)
    lab = orc.tile_labels(cxy, mxy, valid, 160, 128, np.eye(3))
    inner = valid.astype(bool) & (cxy[:, 0] > 12) & (cxy[:, 0] < 147) & (cxy[:, 1] > 12) & \
        (cxy[:, 1] < 115)
    assert inner.sum() > 20
    assert np.all(lab[inner] == [-3.0, 2.0])
    assert np.all(lab[~valid.astype(bool)] == 0)


def test_search_predicted_accepts_good_and_rejects_bad_predictions(orc):
    rng = np.random.default_rng(32)
    c = cfg_for(16, 4)
    img = np.clip(np.kron(rng.integers(0, 256, (34, 42)), np.ones((4, 4))) +
                  rng.normal(0, 3, (136, 168)), 0, 255).astype(np.uint8)[:128, :160]
    src = np.roll(img, (1, 2), axis=(0, 1))
    H = np.eye(3)
    cxy, valid, _ = orc.pick_corners(img, c)
    ctr, mxy, cost = orc.search(img, src, H, c, cxy, valid)
    lab = orc.tile_labels(cxy, mxy, valid, 160, 128, H)
    # exact predictions with an unbounded threshold give the plain matches and costs
    m, co, fb = orc.search_predicted(img, src, H, c, cxy, valid, lab + 0.3, 2 ** 32 - 1)
    assert np.array_equal(m, mxy) and np.array_equal(co, cost) and not fb.any()
    # predictions far off with a finite threshold fall back to the full search
    far = lab + np.float32(7.0)
    m, co, fb = orc.search_predicted(img, src, H, c, cxy, valid, far, 1000)
    assert np.array_equal(m, mxy) and np.array_equal(co, cost)
    assert fb.sum() >= (valid.astype(bool) & (cost <= 1000)).sum() * 0.9
    # rounding is floor(d + 0.5): -0.5 rounds to 0, 0.5 rounds to 1
    one = valid.astype(bool).nonzero()[0][:1]
    p0 = np.zeros_like(lab)
    p0[one] = [-0.5, 0.5]
    m, _, _ = orc.search_predicted(img, src, H, c, cxy, valid, p0, 2 ** 32 - 1)
    assert np.array_equal(m[one], ctr[one] + [[0, 1]])


def test_search_predicted_refinement_recovers_one_pixel_errors(orc):
    rng = np.random.default_rng(33)
    c = cfg_for(16, 4)
    img = np.clip(np.kron(rng.integers(0, 256, (34, 42)), np.ones((4, 4))) +
                  rng.normal(0, 3, (136, 168)), 0, 255).astype(np.uint8)[:128, :160]
    src = np.roll(img, (1, 2), axis=(0, 1))
    H = np.eye(3)
    cxy, valid, _ = orc.pick_corners(img, c)
    ctr, mxy, cost = orc.search(img, src, H, c, cxy, valid)
    lab = orc.tile_labels(cxy, mxy, valid, 160, 128, H)
    off = rng.integers(-1, 2, lab.shape).astype(np.float32)  # predictions off by up to 1 px
    # refine = 1 searches the 3 x 3 offsets around the rounded prediction: the plain optimum
    # (inside that window) is found again with its cost, without falling back
    m, co, fb = orc.search_predicted(img, src, H, c, cxy, valid, lab + off, 2 ** 32 - 1, refine=1)
    assert np.array_equal(m, mxy) and np.array_equal(co, cost) and not fb.any()
    # refine = 0 keeps the off-by-one matches where the threshold lets them through
    m0, _, _ = orc.search_predicted(img, src, H, c, cxy, valid, lab + off, 2 ** 32 - 1, refine=0)
    moved = valid.astype(bool) & (np.abs(off).sum(1) > 0)
    assert np.array_equal(m0[moved] - mxy[moved], off[moved].astype(np.int32))
