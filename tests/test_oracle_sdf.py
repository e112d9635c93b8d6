"""Pins of the FP64 oracle's signed-distance functions (Sec. IV-B, IV-C).

Each test checks the oracle against something other than itself: textbook
closed forms, brute force over densely sampled boundaries, an exact-rational
crossing test, a winding-number test, rigid-motion invariance, Lipschitz
continuity, and the geometry printed in the paper.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rect_poly(a, b, cx=0.0, cy=0.0, ccw=True):
    v = [(cx - a, cy - b), (cx + a, cy - b), (cx + a, cy + b), (cx - a, cy + b)]
    return np.array(v if ccw else v[::-1])


def _box_closed_form(p, a, b):
    """Textbook signed distance of an origin-centred a x b half-extent box."""
    qx, qy = np.abs(p[:, 0]) - a, np.abs(p[:, 1]) - b
    outside = np.hypot(np.maximum(qx, 0), np.maximum(qy, 0))
    inside = -np.minimum(a - np.abs(p[:, 0]), b - np.abs(p[:, 1]))
    return np.where((qx > 0) | (qy > 0), outside, inside)


def _brute_unsigned(p, verts, per_edge):
    """min over `per_edge` evenly spaced samples of every edge; also returns h."""
    v = np.asarray(verts, dtype=np.float64)
    w = np.roll(v, -1, axis=0)
    t = np.arange(per_edge) / per_edge
    samples = (v[:, None, :] + t[None, :, None] * (w - v)[:, None, :]).reshape(-1, 2)
    h = np.max(np.hypot(*(w - v).T)) / per_edge
    best = np.full(p.shape[0], np.inf)
    for k in range(0, samples.shape[0], 4096):
        s = samples[k:k + 4096]
        d = np.hypot(p[:, None, 0] - s[None, :, 0], p[:, None, 1] - s[None, :, 1]).min(axis=1)
        best = np.minimum(best, d)
    return best, h


def _winding_number(p, verts):
    """Winding number by summing signed subtended angles (FP64)."""
    v = np.asarray(verts, dtype=np.float64)
    w = np.roll(v, -1, axis=0)
    a = v[None, :, :] - p[:, None, :]
    b = w[None, :, :] - p[:, None, :]
    cross = a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]
    dot = (a * b).sum(-1)
    return np.rint(np.arctan2(cross, dot).sum(axis=1) / (2 * math.pi)).astype(int)


def _exact_crossing_inside(px, py, verts):
    """Ray-casting parity in exact rational arithmetic on the float inputs."""
    X, Y = Fraction(px), Fraction(py)
    inside = False
    n = len(verts)
    for b in range(n):
        vx, vy = (Fraction(c) for c in verts[b])
        wx, wy = (Fraction(c) for c in verts[(b + 1) % n])
        if (vy > Y) != (wy > Y):
            if X < vx + (Y - vy) * (wx - vx) / (wy - vy):
                inside = not inside
    return inside


def _gap_l():
    vals = {}
    with open(os.path.join(GOLDEN, "l_gap_footprint.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    H, W, t = vals["height"], vals["width"], vals["leg"]
    return np.array([(0, 0), (W, 0), (W, t), (t, t), (t, H), (0, H)], dtype=np.float64)


# --------------------------------------------------------------------- boxes
@pytest.mark.parametrize("ccw", [True, False])
def test_polygon_single_rectangle_matches_box_closed_form(ccw):
    g = np.random.default_rng(1)
    a, b = 0.7, 0.3
    p = g.uniform(-2, 2, size=(4000, 2))
    ref = _box_closed_form(p, a, b)
    got = oracle.sdf_points(p, oracle.POLYGON, _rect_poly(a, b, ccw=ccw))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_rect_single_box_matches_closed_form():
    g = np.random.default_rng(2)
    a, b = 0.9, 0.5
    p = g.uniform(-2, 2, size=(4000, 2))
    got = oracle.sdf_points(p, oracle.RECTS, [[0.0, 0.0, a, b]])
    np.testing.assert_allclose(got, _box_closed_form(p, a, b), rtol=0, atol=1e-14)


def test_rect_box_offset_centre():
    g = np.random.default_rng(3)
    p = g.uniform(-3, 3, size=(2000, 2))
    got = oracle.sdf_points(p, oracle.RECTS, [[1.5, -0.35, 0.6, 0.075]])
    ref = _box_closed_form(p - np.array([1.5, -0.35]), 0.6, 0.075)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


# --------------------------------------------------------------------- convex
def test_convex_polygon_interior_is_max_of_halfplanes():
    g = np.random.default_rng(4)
    n = 9
    ang = np.sort(g.uniform(0, 2 * math.pi, n))
    verts = np.stack([np.cos(ang), np.sin(ang)], 1) * 1.3  # inscribed in a circle: convex
    w = np.roll(verts, -1, 0)
    e = w - verts
    normal = np.stack([e[:, 1], -e[:, 0]], 1) / np.hypot(e[:, 0], e[:, 1])[:, None]  # outward (CCW)
    p = g.uniform(-1.3, 1.3, size=(6000, 2))
    halfplane = ((p[:, None, :] - verts[None]) * normal[None]).sum(-1).max(axis=1)
    inside = halfplane < -1e-9
    got = oracle.sdf_points(p[inside], oracle.POLYGON, verts)
    np.testing.assert_allclose(got, halfplane[inside], rtol=0, atol=1e-13)
    assert inside.sum() > 1000


def test_regular_ngon_approaches_circle():
    n, R = 256, 1.0
    a = 2 * math.pi * np.arange(n) / n
    verts = np.stack([np.cos(a), np.sin(a)], 1) * R
    g = np.random.default_rng(5)
    r = g.uniform(0.0, 3.0, 3000)
    t = g.uniform(0, 2 * math.pi, 3000)
    p = np.stack([r * np.cos(t), r * np.sin(t)], 1)
    got = oracle.sdf_points(p, oracle.POLYGON, verts)
    circle = r - R
    # the polygon lies between the circles of radius R cos(pi/n) and R
    assert np.all(got >= circle - 1e-12)
    assert np.all(got <= circle + R * (1 - math.cos(math.pi / n)) + 1e-12)


# --------------------------------------------------------------------- concave
@pytest.mark.parametrize("name", ["l_c1", "l_gap", "star"])
def test_concave_unsigned_matches_brute_force(name):
    g = np.random.default_rng(6)
    verts = {"l_c1": synth.l_footprint().astype(np.float64), "l_gap": _gap_l(),
             "star": synth.star_polygon(np.random.default_rng(7), 7, 0.3, 1.2).astype(np.float64)}[name]
    lo, hi = verts.min(0) - 0.8, verts.max(0) + 0.8
    p = g.uniform(lo, hi, size=(150, 2))
    got = oracle.sdf_points(p, oracle.POLYGON, verts)
    brute, h = _brute_unsigned(p, verts, 100_000)
    diff = brute - np.abs(got)
    assert np.all(diff >= -1e-12), diff.min()
    assert np.all(diff <= h / 2 + 1e-12), (diff.max(), h)


def test_sign_matches_exact_rational_crossing_and_winding():
    g = np.random.default_rng(8)
    for verts in (synth.l_footprint().astype(np.float64), _gap_l(),
                  synth.star_polygon(g, 11, 0.3, 1.2).astype(np.float64)):
        lo, hi = verts.min(0) - 0.5, verts.max(0) + 0.5
        p = g.uniform(lo, hi, size=(400, 2))
        d = oracle.sdf_points(p, oracle.POLYGON, verts)
        keep = np.abs(d) > 1e-9
        exact = np.array([_exact_crossing_inside(x, y, verts) for x, y in p[keep]])
        wn = _winding_number(p[keep], verts) != 0
        np.testing.assert_array_equal(d[keep] < 0, exact)
        np.testing.assert_array_equal(d[keep] < 0, wn)
        np.testing.assert_array_equal(oracle.inside_points(p[keep], verts), exact)


def test_points_on_vertex_heights_and_lattice():
    # rays through vertices: points sharing a vertex's y coordinate
    verts = _gap_l()
    ys = np.unique(verts[:, 1])
    xs = np.linspace(-0.5, 2.5, 61)
    p = np.array([(x, y) for y in ys for x in xs])
    d = oracle.sdf_points(p, oracle.POLYGON, verts)
    keep = np.abs(d) > 1e-12
    exact = np.array([_exact_crossing_inside(x, y, verts) for x, y in p[keep]])
    wn = _winding_number(p[keep], verts) != 0
    np.testing.assert_array_equal(d[keep] < 0, exact)
    np.testing.assert_array_equal(exact, wn)


def test_zero_on_vertices_and_edge_midpoints():
    for verts in (synth.l_footprint().astype(np.float64), _gap_l()):
        mid = 0.5 * (verts + np.roll(verts, -1, 0))
        assert np.all(oracle.sdf_points(verts, oracle.POLYGON, verts) == 0.0)
        assert np.all(np.abs(oracle.sdf_points(mid, oracle.POLYGON, verts)) <= 1e-15)


def test_gap_l_hand_derived_points():
    verts = _gap_l()  # 2.0 x 2.0 m L with 0.4 m legs
    cases = [((1.0, 0.2), -0.2), ((0.2, 1.0), -0.2), ((1.0, 1.0), 0.6), ((3.0, 0.2), 1.0),
             ((3.0, 3.0), math.hypot(1.0, 2.6)), ((-1.0, -1.0), math.sqrt(2.0)),
             ((0.2, 0.2), -0.2), ((0.3, 0.35), -math.hypot(0.1, 0.05)), ((1.2, 0.5), 0.1),
             ((0.5, 0.45), 0.05)]
    p = np.array([c[0] for c in cases])
    got = oracle.sdf_points(p, oracle.POLYGON, verts)
    np.testing.assert_allclose(got, [c[1] for c in cases], rtol=0, atol=1e-12)


def test_zero_length_edge_is_vertex_distance():
    verts = np.array([(0, 0), (1, 0), (1, 0), (1, 1), (0, 1)], dtype=np.float64)
    g = np.random.default_rng(9)
    p = g.uniform(-1, 2, size=(1000, 2))
    ref = oracle.sdf_points(p, oracle.POLYGON, np.array([(0, 0), (1, 0), (1, 1), (0, 1)], float))
    np.testing.assert_allclose(oracle.sdf_points(p, oracle.POLYGON, verts), ref, atol=1e-15, rtol=0)


# --------------------------------------------------------------------- invariances
def test_lipschitz():
    g = np.random.default_rng(10)
    verts = synth.star_polygon(g, 13, 0.3, 1.2).astype(np.float64)
    p = g.uniform(-2, 2, size=(3000, 2))
    q = p + g.normal(0, 0.05, size=p.shape)
    dp = oracle.sdf_points(p, oracle.POLYGON, verts)
    dq = oracle.sdf_points(q, oracle.POLYGON, verts)
    assert np.all(np.abs(dp - dq) <= np.hypot(*(p - q).T) * (1 + 1e-12) + 1e-15)
    dr = oracle.sdf_points(p, oracle.RECTS, synth.forklift_rects())
    dr2 = oracle.sdf_points(q, oracle.RECTS, synth.forklift_rects())
    assert np.all(np.abs(dr - dr2) <= np.hypot(*(p - q).T) * (1 + 1e-12) + 1e-15)


@pytest.mark.parametrize("kind", [oracle.POLYGON, oracle.RECTS])
def test_rigid_motion_invariance_of_batch(kind):
    """d(R^T(o - t), B) equals the distance of o to the footprint placed at (t, theta)."""
    g = np.random.default_rng(11)
    pts = g.uniform(-4, 4, size=(300, 2))
    poses = np.column_stack([g.uniform(-2, 2, (5, 2)), g.uniform(-math.pi, math.pi, 5)])
    if kind == oracle.POLYGON:
        fp = synth.l_footprint().astype(np.float64)
    else:
        fp = synth.forklift_rects().astype(np.float64)
        # only a polygon can be placed in the world frame exactly; use a single rectangle
        fp = fp[:1]
    dist, dmin, arg = oracle.sdf_batch(pts, poses, kind, fp)
    for k, (x, y, th) in enumerate(poses):
        c, s = math.cos(th), math.sin(th)
        if kind == oracle.POLYGON:
            world = fp @ np.array([[c, s], [-s, c]]) + np.array([x, y])
        else:
            cx, cy, a, b = fp[0]
            world = _rect_poly(a, b, cx, cy) @ np.array([[c, s], [-s, c]]) + np.array([x, y])
        ref = oracle.sdf_points(pts, oracle.POLYGON, world)
        np.testing.assert_allclose(dist[k], ref, rtol=0, atol=1e-12)
        assert dmin[k] == dist[k].min() and arg[k] == int(np.argmin(dist[k]))


def test_body_frame_special_angles():
    pts = np.array([[1.0, 2.0], [-3.0, 0.5]])
    d0, _, _ = oracle.sdf_batch(pts, [[0.0, 0.0, 0.0]], oracle.RECTS, [[0, 0, 0.1, 0.1]])
    np.testing.assert_allclose(d0[0], oracle.sdf_points(pts, oracle.RECTS, [[0, 0, 0.1, 0.1]]))
    # theta = pi/2: body x axis points along world +y, so p_body = (o_y, -o_x)
    d1, _, _ = oracle.sdf_batch(pts, [[0.0, 0.0, math.pi / 2]], oracle.RECTS, [[0.5, 0, 0.1, 0.2]])
    ref = oracle.sdf_points(np.column_stack([pts[:, 1], -pts[:, 0]]), oracle.RECTS, [[0.5, 0, 0.1, 0.2]])
    np.testing.assert_allclose(d1[0], ref, atol=1e-15)


def test_mask_excludes_points_and_empty_is_inf():
    pts = np.array([[0.0, 0.0], [5.0, 0.0]])
    mask = np.array([0, 1], dtype=np.uint8)
    dist, dmin, arg = oracle.sdf_batch(pts, [[0, 0, 0]], oracle.RECTS, [[0, 0, 1, 1]], mask=mask)
    assert dist[0, 0] == np.inf and dmin[0] == 4.0 and arg[0] == 1
    dist, dmin, arg = oracle.sdf_batch(pts, [[0, 0, 0]], oracle.RECTS, [[0, 0, 1, 1]],
                                       mask=np.zeros(2, np.uint8))
    assert np.all(np.isinf(dist)) and dmin[0] == np.inf and arg[0] == -1


# --------------------------------------------------------------------- rect vs polygon
FORKLIFT_OUTLINE = np.array([(-0.9, -0.5), (0.9, -0.5), (0.9, -0.425), (2.1, -0.425), (2.1, -0.275),
                             (0.9, -0.275), (0.9, 0.275), (2.1, 0.275), (2.1, 0.425), (0.9, 0.425),
                             (0.9, 0.5), (-0.9, 0.5)])
T_RECTS = np.array([[0.0, 0.5, 1.0, 0.2], [0.0, -0.2, 0.25, 0.6]])  # bar + stem (overlapping)
T_OUTLINE = np.array([(-0.25, -0.8), (0.25, -0.8), (0.25, 0.3), (1.0, 0.3), (1.0, 0.7),
                      (-1.0, 0.7), (-1.0, 0.3), (-0.25, 0.3)])


FORKLIFT_RECTS = np.array([(0.0, 0.0, 0.9, 0.5), (1.5, 0.35, 0.6, 0.075), (1.5, -0.35, 0.6, 0.075)])


@pytest.mark.parametrize("rects,outline", [(FORKLIFT_RECTS, FORKLIFT_OUTLINE),
                                           (T_RECTS, T_OUTLINE)]
                         + [(r, o)
                            for o, r in synth.rectilinear_shapes().values()])
def test_rect_cover_vs_polygon_outline(rects, outline):
    """Sec. IV-C exactness statement: equal outside, same sign, interior rect >= poly."""
    g = np.random.default_rng(12)
    p = g.uniform(-2.5, 2.5, size=(20000, 2))
    dr = oracle.sdf_points(p, oracle.RECTS, rects)
    dp = oracle.sdf_points(p, oracle.POLYGON, outline)
    off = np.abs(dp) > 1e-9
    np.testing.assert_array_equal((dr < 0)[off], (dp < 0)[off])
    out = dp > 1e-9
    np.testing.assert_allclose(dr[out], dp[out], rtol=0, atol=1e-12)
    ins = dp < -1e-9
    assert np.all(dr[ins] >= dp[ins] - 1e-12)
    assert out.sum() > 1000 and ins.sum() > 100
