"""Pins of the oracle's integrand: the PSS path contribution F(x) (CPU only)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_07148_gb300 import scenes


# ------------------------------------------------------------ white furnace
@pytest.mark.parametrize("depth,rho,le", [(0, 0.5, 1.0), (3, 0.5, 1.0), (8, 0.3, 2.0), (40, 0.5, 1.0)])
def test_white_furnace_closed_form(depth, rho, le):
    """Closed cube, Lambertian rho and emission L_e on every face, camera
    inside: every path has F = L_e (1 - rho^(depth+1)) / (1 - rho) exactly
    (cosine sampling makes every bounce weight rho; every ray hits)."""
    sc = scenes.furnace(depth=depth, albedo=rho, emission=le)
    S = O.Scene(sc)
    x = np.random.default_rng(depth).random((2000, sc.D))
    F, p, u, k = O.eval_states(S, x)
    rho, le = float(np.float32(rho)), float(np.float32(le))   # the scene stores float32
    expect = le * (1 - rho ** (depth + 1)) / (1 - rho)
    assert np.abs(F - expect).max() <= 1e-12 * expect
    assert np.allclose(u, 1.0)
    assert np.allclose(k, 1.0 / p)


def test_white_furnace_image_is_flat():
    """Jump Restore on the furnace: p constant, so the image is flat at the
    closed form; only J vs sum(dt) fluctuates."""
    sc = scenes.furnace(width=4, height=4, depth=5, albedo=0.5, emission=1.0)
    S = O.Scene(sc)
    vals = []
    for b in range(8):
        ch = O.Chains(S, sc.D, 4, 4, n_chains=128, chain_begin=128 * b, seed=3)
        ch.advance(400)
        vals.append(ch.image().mean())
    expect = (1 - 0.5 ** 6) / 0.5
    vals = np.array(vals)
    se = vals.std(ddof=1) / np.sqrt(len(vals))
    assert abs(vals.mean() - expect) < 4 * se + 1e-12


def test_empty_scene_has_zero_integrand():
    sc = scenes.empty()
    S = O.Scene(sc)
    x = np.random.default_rng(0).random((100, sc.D))
    F, p, u, k = O.eval_states(S, x)
    assert np.all(F == 0) and np.all(p == 0) and np.all(np.isinf(k))


# ------------------------------------------------------------ intersection
def test_ray_triangle_hand_cases():
    v0, v1, v2 = [0, 0, 0], [1, 0, 0], [0, 1, 0]
    assert O.intersect_triangle([0.25, 0.25, 1], [0, 0, -1], v0, v1, v2) == 1.0
    assert O.intersect_triangle([0.25, 0.25, 2], [0, 0, -2], v0, v1, v2) == 1.0   # t in units of |d|
    assert O.intersect_triangle([0.25, 0.25, -1], [0, 0, -1], v0, v1, v2) == math.inf  # behind
    assert O.intersect_triangle([0.75, 0.75, 1], [0, 0, -1], v0, v1, v2) == math.inf  # outside u+v>1
    assert O.intersect_triangle([-0.1, 0.2, 1], [0, 0, -1], v0, v1, v2) == math.inf   # u<0
    assert O.intersect_triangle([0.2, 0.2, 0], [1, 0, 0], v0, v1, v2) == math.inf     # in the plane
    t = O.intersect_triangle([0.1, 0.1, 3.0], [0.1, 0.1, -1.0], v0, v1, v2)
    assert abs(t - 3.0) < 1e-15
    # both windings hit (two-sided test)
    assert O.intersect_triangle([0.25, 0.25, 1], [0, 0, -1], v0, v2, v1) == 1.0


def test_bvh_closest_hit_equals_brute_force():
    sc = scenes.cornell_spheres(n_lon=24, n_lat=13)
    Sb = O.Scene(sc, bvh=True)
    S = O.Scene(sc)
    rng = np.random.default_rng(1)
    for _ in range(3000):
        o = rng.random(3)
        d = rng.normal(size=3)
        i1, t1 = S.closest_hit(o, d, use_bvh=False)
        i2, t2 = Sb.closest_hit(o, d, use_bvh=True)
        assert i1 == i2 and (t1 == t2 or (math.isinf(t1) and math.isinf(t2)))
    x = rng.random((500, sc.D))
    a = O.eval_states(S, x, hit_ids=True)
    b = O.eval_states(Sb, x, hit_ids=True)
    assert np.array_equal(a[4], b[4]) and np.array_equal(a[0], b[0])


def test_camera_center_ray_and_pixel_rows():
    """The film centre looks along f; x1 = 0 is the top row (rays tilt +up)."""
    sc = scenes.cornell()
    S = O.Scene(sc)
    # the centre ray of the Cornell camera hits the back wall at (0.5, 0.5, 0)
    i, t = S.closest_hit(sc.camera[:3], sc.camera[3:6])
    assert abs(t - 2.3) < 1e-6
    # the top-row ray (x1 ~ 0) hits the ceiling, the bottom row the floor
    x = np.array([[0.5, 0.01] + [0.5] * (sc.D - 2), [0.5, 0.99] + [0.5] * (sc.D - 2)])
    ids = O.eval_states(S, x, hit_ids=True)[4]
    assert ids[0, 0] in (2, 3) and ids[1, 0] in (0, 1)   # ceiling quad = tris 2,3; floor = 0,1


# ------------------------------------------------------------ BSDF sampling
def _ring(u1s, u2s):
    return [(a, b) for a in u1s for b in u2s]


def test_lambert_sampling_is_cosine_weighted():
    m = scenes.material(scenes.LAMBERT, (0.3, 0.5, 0.7))
    ng = np.array([0.3, -0.4, 0.866])
    ng /= np.linalg.norm(ng)
    d = -ng + np.array([0.1, 0.0, 0.0])
    d /= np.linalg.norm(d)
    n = 128
    cs, c2 = [], []
    for u1, u2 in _ring((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n):
        ok, wi, w = O.scatter(m, d, ng, u1, u2)
        assert ok and np.allclose(w, [0.3, 0.5, 0.7])
        assert abs(np.linalg.norm(wi) - 1) < 1e-12
        c = wi @ ng
        assert c >= 0
        cs.append(c)
        c2.append(c * c)
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2 (stratified grid)
    assert abs(np.mean(cs) - 2 / 3) < 2e-3 and abs(np.mean(c2) - 0.5) < 2e-3
    # hitting the back side flips the hemisphere
    ok, wi, w = O.scatter(m, -d, ng, 0.3, 0.6)
    assert wi @ ng <= 0


def test_phong_normal_incidence_albedo_is_rho():
    """At normal incidence the modified Phong lobe never dips below the
    surface and E[weight] = rho exactly (the lobe integrates to rho)."""
    for nexp in (1.0, 10.0, 50.0):
        m = scenes.material(scenes.PHONG, (0.7, 0.7, 0.7), phong_n=nexp)
        ng = np.array([0.0, 0.0, 1.0])
        d = np.array([0.0, 0.0, -1.0])
        n = 256
        ws = []
        for u1, u2 in _ring((np.arange(n) + 0.5) / n, (np.arange(8) + 0.5) / 8):
            ok, wi, w = O.scatter(m, d, ng, u1, u2)
            ws.append(w[0])
        assert abs(np.mean(ws) - 0.7) < 2e-3 * (1 + nexp / 50)


def test_fresnel_matches_angle_form():
    """The Fresnel equations in their angle form (Hecht): R_s = sin^2(i-t) /
    sin^2(i+t), R_p = tan^2(i-t) / tan^2(i+t), against the oracle's cosine
    form; normal incidence gives ((n-1)/(n+1))^2, and total internal
    reflection gives 1."""
    eta = 1.5
    assert abs(O.fresnel(1.0, 1.0, eta) - ((eta - 1) / (eta + 1)) ** 2) < 1e-15
    for deg in (10, 30, 45, 60, 80, 89):
        i = math.radians(deg)
        t = math.asin(math.sin(i) / eta)
        rs = math.sin(i - t) ** 2 / math.sin(i + t) ** 2
        rp = math.tan(i - t) ** 2 / math.tan(i + t) ** 2
        assert abs(O.fresnel(math.cos(i), 1.0, eta) - 0.5 * (rs + rp)) < 1e-13
    crit = math.asin(1 / eta)
    assert O.fresnel(math.cos(crit + 0.01), eta, 1.0) == 1.0


def test_dielectric_snell_and_mirror():
    m = scenes.material(scenes.DIELECTRIC, (1, 1, 1), ior=1.5)
    ng = np.array([0.0, 0.0, 1.0])
    th = math.radians(40)
    d = np.array([math.sin(th), 0.0, -math.cos(th)])
    R = O.fresnel(math.cos(th), 1.0, 1.5)
    ok, wi, w = O.scatter(m, d, ng, R - 1e-9, 0.5)      # reflect
    assert np.allclose(wi, [math.sin(th), 0, math.cos(th)]) and np.allclose(w, 1)
    ok, wi, w = O.scatter(m, d, ng, R + 1e-9, 0.5)      # refract
    assert abs(np.linalg.norm(wi) - 1) < 1e-12
    sin_t = math.hypot(wi[0], wi[1])
    assert abs(1.0 * math.sin(th) - 1.5 * sin_t) < 1e-12 and wi[2] < 0
    # from inside, beyond the critical angle: always reflected
    th2 = math.radians(60)
    d2 = np.array([math.sin(th2), 0.0, math.cos(th2)])
    ok, wi, w = O.scatter(m, d2, ng, 0.999999, 0.5)
    assert np.allclose(wi, [math.sin(th2), 0, -math.cos(th2)])


# ------------------------------------------------------------ Cornell box
def test_cornell_jump_restore_matches_plain_path_tracing():
    """Two different estimators of the same pixels -- Jump Restore (Alg. 2 +
    Section 6.3) and plain Monte Carlo -- agree pixel by pixel within 4.5
    standard errors on a 16x16 Cornell box."""
    sc = scenes.cornell(width=16, height=16, depth=3)
    S = O.Scene(sc)
    jr = []
    for b in range(16):
        ch = O.Chains(S, sc.D, 16, 16, n_chains=256, chain_begin=256 * b, seed=21)
        ch.advance(1500)
        jr.append(ch.image())
    jr = np.array(jr)
    pt = []
    for b in range(16):
        img, _ = O.render_pt(S, sc.D, 16, 16, 1 << 19, seed=22, sample_begin=b << 19)
        pt.append(img)
    pt = np.array(pt)
    d = jr.mean(0) - pt.mean(0)
    se = np.sqrt(jr.var(0, ddof=1) / len(jr) + pt.var(0, ddof=1) / len(pt))
    ok = se > 0
    assert np.all(d[~ok] == 0)                      # pixels/channels that are exactly zero on both sides
    z = d[ok] / se[ok]
    assert np.mean(np.abs(z) > 4.5) <= 0.002
    assert 0.6 < np.mean(z ** 2) < 1.5              # differences are the size the noise predicts
    rel = np.mean(d ** 2 / (pt.mean(0) ** 2 + 1e-2))
    noise = np.mean(se ** 2 / (pt.mean(0) ** 2 + 1e-2))
    assert rel < 2.0 * noise
