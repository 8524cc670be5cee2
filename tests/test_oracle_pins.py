"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test checks an oracle function against something other than itself: published
known-answer values, the paper's closed kernel values and worked example (Fig. 7),
identities between kernel families, library routines (scipy), quadrature identities of
the microfacet model, and Monte-Carlo / enumeration properties of the estimators.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, ndimage

import oracle
import stf_synth as synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------------ Philox
def test_philox_known_answers():
    for v in _gold("philox_kat.json")["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert list(oracle.philox(ctr, key)) == out


# ------------------------------------------------------------------------ kernels
FILTERS = ["linear", "bspline", "catmull_rom", "mitchell"]


def _taps(f):
    return (0, 1) if f == "linear" else (-1, 0, 1, 2)


@pytest.mark.parametrize("f", FILTERS)
def test_partition_of_unity(f):
    # Eq. filtered-texture: the weights of a filter footprint sum to 1
    for t in np.linspace(0, 1, 10001)[:-1]:
        s = sum(oracle.kernel(f, t - k) for k in _taps(f))
        assert abs(s - 1.0) < 1e-13


def test_closed_values():
    for c in _gold("filter_closed_values.json")["cases"]:
        t = c["t"]
        want = [float(Fraction(x)) for x in c["w"]]
        got = [oracle.kernel(c["filter"], t - k) for k in _taps(c["filter"])]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
        # the FP32 decision weights agree with the FP64 definition to FP32 rounding
        np.testing.assert_allclose(oracle.weights32(c["filter"], t), want, rtol=0, atol=2e-7)


def test_bc_family_identities():
    # Mitchell & Netravali BC(0, 1/2) is Keys' cubic with a = -1/2, and BC(1, 0) is the
    # cubic B-spline (supplement Eq. cubic-bspline).  A dropped or mis-signed term in the
    # BC formula breaks one of these.
    for d in np.linspace(-2.5, 2.5, 2001):
        assert abs(oracle.kernel_bc(0.0, 0.5, d) - oracle.kernel_keys(-0.5, d)) < 1e-14
        assert abs(oracle.kernel_bc(1.0, 0.0, d) - oracle.kernel("bspline", d)) < 1e-14
        # the lookups' kernels are the factored forms of the same polynomials; the expanded
        # forms' own cancellation near the double root at |d| = 2 is ~1e-15 (the factored
        # forms are checked against exact arithmetic below)
        assert abs(oracle.kernel("catmull_rom", d) - oracle.kernel_keys(-0.5, d)) < 4e-15
        assert abs(oracle.kernel("mitchell", d) - oracle.kernel_bc(1 / 3, 1 / 3, d)) < 4e-15


def test_bspline_is_fourfold_box_convolution():
    # Sec. 4.2: degree-n B-splines are repeated convolutions of the unit box (Cox-de Boor)
    h = 1e-3
    x = np.arange(-0.5, 0.5, h) + h / 2
    box = np.ones_like(x)
    k = box.copy()
    for _ in range(3):
        k = np.convolve(k, box) * h
    xs = (np.arange(k.size) - (k.size - 1) / 2) * h
    ref = np.array([oracle.kernel("bspline", d) for d in xs[::50]])
    np.testing.assert_allclose(k[::50], ref, atol=3e-6)


def test_polynomial_reproduction():
    # Keys' a = -1/2 cubic reproduces quadratics; BC filters with B + 2C = 1 and the
    # B-spline reproduce linear functions; the tent reproduces linear functions.
    for t in np.linspace(0, 1, 257):
        for f, deg in (("catmull_rom", 2), ("mitchell", 1), ("bspline", 1), ("linear", 1)):
            for p in range(deg + 1):
                s = sum(oracle.kernel(f, t - k) * k ** p for k in _taps(f))
                assert abs(s - t ** p) < 1e-12, (f, p, t)
    # and the B-spline does NOT reproduce t^2 (it is approximating, not interpolating)
    s = sum(oracle.kernel("bspline", 0.5 - k) * k ** 2 for k in _taps("bspline"))
    assert abs(s - 0.25 - 1 / 3) < 1e-12


@pytest.mark.parametrize("f", FILTERS)
def test_fp32_weights_match_fp64(f):
    rng = np.random.default_rng(5)
    for t in np.concatenate([rng.random(2000), [0.0, 0.5, 1.0 - 2 ** -24]]).astype(np.float32):
        w64 = [oracle.kernel(f, float(t) - k) for k in _taps(f)]
        np.testing.assert_allclose(oracle.weights32(f, t), w64, rtol=0, atol=1e-6)


def _exact_cubic(f, d):
    """Keys' a = -1/2 cubic and Mitchell-Netravali BC(1/3, 1/3) at d in exact rational
    arithmetic, from the published piecewise polynomials (expanded form)."""
    d = abs(Fraction(d))
    if f == "catmull_rom":
        a = Fraction(-1, 2)
        if d < 1:
            return (a + 2) * d ** 3 - (a + 3) * d ** 2 + 1
        return a * d ** 3 - 5 * a * d ** 2 + 8 * a * d - 4 * a if d < 2 else Fraction(0)
    B = C = Fraction(1, 3)
    if d < 1:
        return ((12 - 9 * B - 6 * C) * d ** 3 + (-18 + 12 * B + 6 * C) * d ** 2 + (6 - 2 * B)) / 6
    if d < 2:
        return ((-B - 6 * C) * d ** 3 + (6 * B + 30 * C) * d ** 2 + (-12 * B - 48 * C) * d + (8 * B + 24 * C)) / 6
    return Fraction(0)


def _near_root_ts():
    """FP32 positions t near the signed cubics' roots: t -> 0 and t -> 1 (the double root of
    the outer piece at |d| = 2 and Keys' root at |d| = 1) and Mitchell's zero crossings of the
    outer piece at t = 1/7 and 6/7, plus random positions."""
    ts = [2.0 ** -k for k in range(1, 25)] + [1.0 - 2.0 ** -k for k in range(1, 25)]
    for c in (1 / 7, 6 / 7):
        x = np.float32(c)
        for k in range(-8, 9):
            ts.append(float(np.nextafter(x, np.float32(2 if k > 0 else -1)) if k else x))
            x = np.nextafter(x, np.float32(2 if k > 0 else -1)) if k else x
    ts += list(np.random.default_rng(9).random(500))
    return np.unique(np.array(ts, dtype=np.float32))


@pytest.mark.parametrize("f", ["catmull_rom", "mitchell"])
def test_signed_weights_keep_relative_precision_near_roots(f):
    # A positivized sample picks its sign class from the ratio of the small negative-lobe
    # weights, so both the FP64 definition and the FP32 decision weights must be accurate
    # RELATIVE to the weight, with the exact sign, also where the weight tends to zero.
    for t in _near_root_ts():
        tf = Fraction(float(t))
        exact = [_exact_cubic(f, tf - k) for k in _taps(f)]
        w64 = [oracle.kernel(f, float(t) - k) for k in _taps(f)]
        w32 = oracle.weights32(f, t)
        for e, a, b in zip(exact, w64, w32):
            if e == 0:
                assert a == 0 and b == 0, (t, e, a, b)
                continue
            assert abs(Fraction(a) - e) <= abs(e) * Fraction(1, 2 ** 48), (f, float(t), float(e), a)
            assert abs(Fraction(float(b)) - e) <= abs(e) * Fraction(1, 2 ** 18), (f, float(t), float(e), float(b))


# ------------------------------------------------------------------------ picks
def test_fig7_frs_probabilities():
    # Fig. 7: the u-measure of each cell of the CDF equals the printed probability
    p = np.array(_gold("frs_fig7.json")["probabilities"])
    m = 1 << 14
    xi = (np.arange(m) + 0.5) / m
    hist = np.bincount([oracle.pick_array(p, x) for x in xi], minlength=9) / m
    np.testing.assert_allclose(hist, p, atol=1.0 / m)
    assert hist[6] == 0.0          # the 0% cell is never selected


@pytest.mark.parametrize("f", FILTERS)
@pytest.mark.parametrize("cls", [0, 1, -1])
def test_pick32_enumeration(f, cls):
    # Sec. 2.2 "Sampling arrays": the FP32 inversion selects tap k on a u-interval of
    # length |w_k| / sum|w| (restricted to a sign class for positivization).
    rng = np.random.default_rng(11)
    m = 1 << 13
    xi = ((np.arange(m) + 0.5) / m).astype(np.float32)
    for t in rng.random(6).astype(np.float32):
        w = oracle.weights32(f, t)
        sel = np.array([(cls == 0) or (cls > 0 and x > 0) or (cls < 0 and x < 0) for x in w])
        if not sel.any():
            continue
        a = np.abs(w.astype(np.float64)) * sel
        hist = np.bincount([oracle.pick32(w, x, cls) for x in xi], minlength=len(w)) / m
        np.testing.assert_allclose(hist, a / a.sum(), atol=2.0 / m)


# ------------------------------------------------------------------------ shading
L_DIR = np.array([0.48, 0.36, 0.80], dtype=np.float32).astype(np.float64)
V_DIR = np.array([-0.28, 0.0, 0.96], dtype=np.float32).astype(np.float64)


def test_ggx_alpha_one_is_uniform():
    for nh in np.linspace(0.01, 1, 50):
        assert abs(oracle.ggx_D(1.0, nh) - 1 / math.pi) < 1e-14


@pytest.mark.parametrize("alpha", [0.05, 0.1, 0.3, 0.7, 1.0])
def test_ggx_D_normalized(alpha):
    # integral over the hemisphere of D(h) (n.h) d omega_h = 1
    f = lambda th: oracle.ggx_D(alpha, math.cos(th)) * math.cos(th) * math.sin(th) * 2 * math.pi
    val, _ = integrate.quad(f, 0, math.pi / 2, points=[alpha, 2 * alpha, 4 * alpha], limit=400)
    assert abs(val - 1.0) < 1e-7


@pytest.mark.parametrize("alpha", [0.2, 0.5])
@pytest.mark.parametrize("theta_o", [0.2, 0.7, 1.2])
def test_smith_masking_projected_area(alpha, theta_o):
    # Smith masking consistency (Heitz 2014): G1(o) * int <o,m>+ D(m) dm = cos(theta_o),
    # with G1 = 1 / (1 + Lambda(o)) -- pins Lambda against D.
    o = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])

    def inner(phi, th):
        m = np.array([math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)])
        return max(0.0, float(o @ m)) * oracle.ggx_D(alpha, math.cos(th)) * math.sin(th)

    val, _ = integrate.dblquad(inner, 0, math.pi / 2, 0, 2 * math.pi, epsabs=1e-9, epsrel=1e-9)
    g1 = 1.0 / (1.0 + oracle.smith_lambda(alpha, math.tan(theta_o) ** 2))
    assert abs(g1 * val - math.cos(theta_o)) < 1e-6


def test_ggx_reciprocity_and_closed_forms():
    rng = np.random.default_rng(3)
    rho = np.array([0.3, 0.5, 0.7])
    for _ in range(200):
        n = rng.normal(size=3); n[2] = abs(n[2]) + 1.0; n /= np.linalg.norm(n)
        l = rng.normal(size=3); l[2] = abs(l[2]) + 0.5; l /= np.linalg.norm(l)
        v = rng.normal(size=3); v[2] = abs(v[2]) + 0.5; v /= np.linalg.norm(v)
        a = rng.uniform(0.05, 1.0)
        f1 = oracle.ggx_eval(n, l, v, a, rho, 0.04)
        f2 = oracle.ggx_eval(n, v, l, a, rho, 0.04)
        nl, nv = n @ l, n @ v
        if nl > 0 and nv > 0:
            np.testing.assert_allclose(f1 / nl, f2 / nv, rtol=1e-12)   # BRDF reciprocity
            # Lambert part is linear in rho: f(rho) - f(0) = rho nl / pi
            np.testing.assert_allclose(oracle.ggx_eval(n, l, v, a, rho, 0.04)
                                       - oracle.ggx_eval(n, l, v, a, np.zeros(3), 0.04),
                                       rho * nl / math.pi, rtol=1e-12, atol=1e-15)
        else:
            assert np.all(f1 == 0)
    # normal incidence, l = v = n: D = 1/(pi a^2), G2 = 1, F = F0 -> spec = F0 / (4 pi a^2)
    z = np.array([0.0, 0.0, 1.0])
    for a in (float(np.float32(0.05)), 0.2, 1.0):     # alpha is clamped at the FP32 0.05f
        got = oracle.ggx_eval(z, z, z, a, np.zeros(3), 0.04)
        np.testing.assert_allclose(got, 0.04 / (4 * math.pi * a * a), rtol=1e-13)


def test_ggx_directional_albedo_bounded():
    # energy conservation of the specular lobe: int f_spec cos d omega_l <= 1
    z = np.array([0.0, 0.0, 1.0])
    for a in (0.1, 0.5, 1.0):
        for tv in (0.0, 0.6, 1.2):
            v = np.array([math.sin(tv), 0.0, math.cos(tv)])

            def integrand(phi, th):
                l = np.array([math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)])
                return oracle.ggx_eval(z, l, v, a, np.zeros(3), 1.0)[0] * math.sin(th)
            val, _ = integrate.dblquad(integrand, 0, math.pi / 2, 0, 2 * math.pi, epsabs=1e-6)
            assert 0 < val <= 1.0 + 1e-6


# ------------------------------------------------------------------------ estimators
def _tiny_tex(n=8, seed=7, fmt="f32", mips=False):
    if fmt == "f32":
        return oracle.Texture([synth.texture_rgba32f(n, seed)])
    m = synth.material_rgba8(n, seed, octaves=3, base=2, mips=mips)
    return oracle.Texture(m.albedo_rough, m.normal)


@pytest.mark.parametrize("f,order", [("linear", 1), ("bspline", 3)])
def test_ntap_matches_scipy_spline(f, order):
    # With the identity shade, filter-before reconstructs the texture with the filter:
    # scipy's map_coordinates (order 1, and order 3 without prefiltering = direct cubic
    # B-spline convolution of the samples) with periodic addressing is an independent
    # implementation.  Texel centres sit at integer coordinates p = uv * res - 1/2.
    tex = _tiny_tex(8)
    q = synth.queries_uniform(500, 21)
    r = oracle.filter_shade(tex, q, f, "ntap_before", "linear", spp=1)
    img = tex.levels[0].astype(np.float64)
    py = q.v.astype(np.float64) * 8 - 0.5
    px = q.u.astype(np.float64) * 8 - 0.5
    for c in range(3):
        ref = ndimage.map_coordinates(img[..., c], [py, px], order=order, mode="grid-wrap",
                                      prefilter=False)
        np.testing.assert_allclose(r.rgb[:, c], ref, atol=1e-12)


@pytest.mark.parametrize("f", FILTERS)
def test_linear_shade_before_equals_after(f):
    # Sec. 3: for a shade that is affine in the texture, filtering before and after
    # shading agree (with MIP levels, jitter and the stochastic LOD's linear blend)
    m = synth.material_rgba8(32, 5, octaves=4, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_uniform(400, 9, res=32, lod_range=4.0)
    a = oracle.filter_shade(tex, q, f, "ntap_before", "linear", spp=3, seed=4)
    b = oracle.filter_shade(tex, q, f, "ntap_after", "linear", spp=3, seed=4)
    np.testing.assert_allclose(a.rgb, b.rgb, atol=1e-12)


def test_constant_texture_reproduced():
    # a constant texture is reproduced exactly by every sample of the single-tap
    # estimator for positive filters, and by positivization up to rounding of W+ - W-
    c = np.zeros((16, 16, 4), dtype=np.float32)
    c[...] = [0.2, 0.4, 0.6, 0.3]
    tex = oracle.Texture([c])
    q = synth.queries_uniform(300, 2, const_derivs=(1 / 64, 0.0, 0.0, 1 / 64))
    want = oracle.shade_batch(c[0, 0, :3].astype(np.float64)[None], [c[0, 0, 3]], [[0, 0, 1]])[0]
    for f in ("linear", "bspline"):
        r = oracle.filter_shade(tex, q, f, "stochastic", spp=4)
        assert np.all(r.rgb == want)
    for f in ("catmull_rom", "mitchell"):
        r = oracle.filter_shade(tex, q, f, "positivized", spp=4)
        np.testing.assert_allclose(r.rgb, np.broadcast_to(want, r.rgb.shape), rtol=1e-13)
        r = oracle.filter_shade(tex, q, f, "ntap_after", spp=1)
        np.testing.assert_allclose(r.rgb, np.broadcast_to(want, r.rgb.shape), rtol=1e-13)


@pytest.mark.parametrize("f,mode", [("linear", "stochastic"), ("bspline", "stochastic"),
                                    ("mitchell", "stochastic"), ("mitchell", "positivized"),
                                    ("catmull_rom", "positivized")])
def test_stochastic_mean_converges_to_filter_after(f, mode):
    # Eq. stochastic-sum: the single-tap estimator is unbiased for the filter-after sum.
    # Same seed => same jitter and LOD per sample; the paired difference isolates the
    # texel-selection noise, whose mean must be within 3 sigma of zero.
    m = synth.material_rgba8(8, 3, octaves=3, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_uniform(6, 13, res=8, lod_range=2.5)
    spp = 1 << 15
    for seed in (1, 2):
        s = oracle.filter_shade(tex, q, f, mode, spp=spp, seed=seed)
        a = oracle.filter_shade(tex, q, f, "ntap_after", spp=spp, seed=seed)
        # per-query variance estimate from a second independent run of spp/64 samples
        small = [oracle.filter_shade(tex, q, f, mode, spp=1, seed=1000 + k).rgb for k in range(64)]
        small_a = [oracle.filter_shade(tex, q, f, "ntap_after", spp=1, seed=1000 + k).rgb for k in range(64)]
        sd = np.std(np.array(small) - np.array(small_a), axis=0) + 1e-6
        z = np.abs(s.rgb - a.rgb) / (sd / math.sqrt(spp))
        assert z.max() < 4.5, z.max()


def test_stochastic_expectation_by_enumeration():
    # exact expectation: sum over all (kx, ky) of P(kx) P(ky) * estimate equals the
    # filter-after sum (one query, no jitter, no MIP levels), for every filter
    tex = _tiny_tex(8, seed=17)
    img = tex.levels[0].astype(np.float64)
    q = synth.queries_uniform(5, 31)
    for f in FILTERS:
        a = oracle.filter_shade(tex, q, f, "ntap_after")
        for i in range(q.n):
            px, py = float(np.float32(q.u[i]) * np.float32(8)) - 0.5, float(np.float32(q.v[i]) * np.float32(8)) - 0.5
            ix0, iy0 = math.floor(px), math.floor(py)
            tx, ty = px - ix0, py - iy0
            wx = np.array([oracle.kernel(f, tx - k) for k in _taps(f)])
            wy = np.array([oracle.kernel(f, ty - k) for k in _taps(f)])
            W = np.abs(wx).sum() * np.abs(wy).sum()
            e = np.zeros(3)
            for jx, kx in enumerate(_taps(f)):
                for jy, ky in enumerate(_taps(f)):
                    p = abs(wx[jx]) * abs(wy[jy]) / W
                    t = img[(iy0 + ky) % 8, (ix0 + kx) % 8]
                    sh = oracle.shade_batch([t[:3]], [t[3]], [[0, 0, 1]])[0]
                    e += p * np.sign(wx[jx] * wy[jy]) * W * sh
            np.testing.assert_allclose(e, a.rgb[i], rtol=1e-12)


@pytest.mark.parametrize("f,mode", [("linear", "stochastic"), ("bspline", "stochastic"),
                                    ("mitchell", "stochastic"), ("mitchell", "positivized"),
                                    ("catmull_rom", "positivized")])
def test_fp32_decisions_agree_with_fp64_off_boundary(f, mode):
    m = synth.material_rgba8(64, 8, octaves=4, base=4)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_uniform(20000, 77, res=64, lod_range=6.0)
    r = oracle.filter_shade(tex, q, f, mode, spp=8, seed=9, want_picks=True)
    diff = np.any(r.picks != r.picks64, axis=(1, 2))
    # every FP32/FP64 disagreement lies within 1e-6 of an FP64 boundary, and they are as rare
    # as the parity criterion for the kernel's FP32 decisions demands
    assert np.all(r.bdist[diff] < 1e-6)
    assert diff.sum() <= max(1, math.ceil(1e-5 * q.n))


# ------------------------------------------------------------------------ volume
def _box_segment(cam, W, H, px, py, jx, jy):
    e, f, rr, u = cam[:3], cam[3:6], cam[6:9], cam[9:12]
    sx = (px + jx) * 2.0 / W - 1.0
    sy = 1.0 - (py + jy) * 2.0 / H
    d = f + sx * rr + sy * u
    d /= np.linalg.norm(d)
    with np.errstate(divide="ignore"):
        t1, t2 = (0 - e) / d, (1 - e) / d
    tmin = max(0.0, np.max(np.minimum(t1, t2)))
    tmax = np.min(np.maximum(t1, t2))
    return max(0.0, tmax - tmin)


@pytest.mark.parametrize("f", ["linear", "bspline"])
@pytest.mark.parametrize("mode", ["ntap_before", "ntap_after", "stochastic"])
def test_volume_constant_density(f, mode):
    # constant sigma: T = exp(-sigma L) for the segment length L, in every mode;
    # zero density: T = 1
    W, H = 24, 16
    cam = synth.camera_pinhole(W, H).as_array().astype(np.float64)
    vol = np.full((8, 8, 8), 0.5, dtype=np.float16)
    r = oracle.march(vol, 3.0, cam, W, H, 32, f, mode, spp=4, seed=2, flags=oracle.FLAG_STRATIFIED)
    want = []
    for pix in range(W * H):
        px, py = pix % W, pix // W
        t = 0.0
        for s in range(4):
            L = _box_segment(cam, W, H, px, py, (s % 2 + 0.5) / 2, (s // 2 + 0.5) / 2)
            t += math.exp(-1.5 * L)
        want.append(t / 4)
    np.testing.assert_allclose(r.T, want, rtol=2e-6)
    z = oracle.march(np.zeros((8, 8, 8), np.float16), 3.0, cam, W, H, 32, f, mode, spp=2, seed=2)
    np.testing.assert_allclose(z.T, 1.0, rtol=0, atol=1e-13)   # sum of weights = 1 to FP64 rounding


def test_volume_linear_density_trilinear_exact():
    # trilinear reconstruction of a density linear in z (clamped to the voxel range)
    # integrated by the midpoint rule along the central ray
    n, W, H, steps = 16, 1, 1, 64
    z = np.clip(np.arange(n, dtype=np.float64), 0, n - 1) / (n - 1)
    vol = np.broadcast_to(z[:, None, None], (n, n, n)).astype(np.float16)
    cam = synth.camera_pinhole(W, H).as_array().astype(np.float64)
    cam[6:12] = 0.0    # every sample goes straight down +z through (0.5, 0.5)
    r = oracle.march(vol, 2.0, cam, W, H, steps, "linear", "ntap_before", spp=1, seed=1)
    dt = 1.0 / steps
    zk = (np.arange(steps) + 0.5) * dt * n - 0.5
    zk = np.clip(zk, 0, n - 1)
    dens = np.interp(zk, np.arange(n), vol[:, 0, 0].astype(np.float64))
    want = math.exp(-2.0 * dens.sum() * dt)
    assert abs(r.T[0] - want) < 1e-12


def test_volume_stochastic_unbiased():
    # E[prod_k exp(-sigma_pick dt)] = prod_k sum_i w_i exp(-sigma_i dt) (independent
    # picks per step); paired with identical jitter per seed, mean diff within 3 sigma
    vol = synth.volume_cloud(16, 5, zero_frac=0.5, octaves=3, base=2)
    W, H = 4, 3
    cam = synth.camera_pinhole(W, H).as_array()
    for f in ("linear", "bspline"):
        d = []
        for seed in range(1, 1501):
            s = oracle.march(vol, 20.0, cam, W, H, 48, f, "stochastic", spp=1, seed=seed, pix_begin=5, pix_count=1)
            a = oracle.march(vol, 20.0, cam, W, H, 48, f, "ntap_after", spp=1, seed=seed, pix_begin=5, pix_count=1)
            d.append(s.T[0] - a.T[0])
        d = np.array(d)
        assert abs(d.mean()) < 3.5 * d.std() / math.sqrt(len(d)) + 1e-12


# ------------------------------------------------------------------------ decode, LOD, jitter
def test_decode_roundtrip_against_encoder():
    # the generator encodes unit normals to RG8 and roughness to a byte; the oracle's
    # decode must invert that encoding to within the 8-bit quantisation
    m = synth.material_rgba8(32, 4, octaves=3, base=2, mips=False)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    h = m.height
    gx = 0.5 * (np.roll(h, -1, axis=1) - np.roll(h, 1, axis=1))
    gy = 0.5 * (np.roll(h, -1, axis=0) - np.roll(h, 1, axis=0))
    k = 0.35 / np.sqrt(0.5 * (gx.var() + gy.var()))
    nrm = np.stack([-k * gx, -k * gy, np.ones_like(gx)], -1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    for iy in range(0, 32, 5):
        for ix in range(0, 32, 3):
            d = oracle.fetch(tex, 0, ix, iy)
            np.testing.assert_allclose(d[:3], m.albedo_rough[0][iy, ix, :3] / 255.0, atol=1e-15)
            assert 0.05 <= d[3] <= 1.0
            assert abs(d[3] - (0.05 + 0.95 * m.albedo_rough[0][iy, ix, 3] / 255.0)) < 1e-15
            assert abs(np.linalg.norm(d[4:]) - 1) < 1e-14
            np.testing.assert_allclose(d[4:], nrm[iy, ix], atol=1.5 * 2 / 255)


def _level_hist(tex, q, spp):
    r = oracle.filter_shade(tex, q, "linear", "stochastic", spp=spp, want_picks=True)
    return (r.picks64[..., 0] >> 28).astype(np.int64)


def test_lod_stochastic_level_frequency_and_aniso_cap():
    # Sec. 4.2.1: LOD = log2 of the minor footprint axis (in level-0 texels), one MIP
    # level chosen stochastically: level floor(lam)+1 with probability frac(lam); the
    # anisotropy ratio is capped at 64 by growing the minor axis.
    m = synth.material_rgba8(256, 6, octaves=3, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    res = 256.0
    lam = 2.3
    ln = 2 ** lam / res
    q = synth.queries_uniform(64, 5, const_derivs=(ln * 0.6, ln * 0.8, -ln * 0.8, ln * 0.6))
    lv = _level_hist(tex, q, 256)
    assert set(np.unique(lv)) <= {2, 3}
    assert abs((lv == 3).mean() - 0.3) < 4 * math.sqrt(0.21 / lv.size)
    # anisotropy 2^7 with major axis 2^9 texels: minor grows to 2^9 / 64 = 2^3 -> level 3
    q = synth.queries_uniform(64, 6, const_derivs=(2 ** 9 / res, 0.0, 0.0, 2 ** 2 / res))
    assert np.all(_level_hist(tex, q, 4) == 3)
    # magnification clamps to level 0; beyond the pyramid clamps to the last level
    q = synth.queries_uniform(32, 7, const_derivs=(0.25 / res, 0.0, 0.0, 0.25 / res))
    assert np.all(_level_hist(tex, q, 4) == 0)
    q = synth.queries_uniform(32, 8, const_derivs=(2 ** 12 / res, 0.0, 0.0, 2 ** 12 / res))
    assert np.all(_level_hist(tex, q, 4) == len(m.albedo_rough) - 1)


def test_jitter_footprint_matches_scipy():
    # stratified screen-space jitter (Sec. 4.2.1, Fig. 6): with the identity shade the
    # filter-before estimate is the average of the bilinear reconstruction over the
    # jittered positions x = uv + (j_x - 1/2) ddx + (j_y - 1/2) ddy
    tex = _tiny_tex(16, seed=23)
    img = tex.levels[0].astype(np.float64)
    d = (0.7 / 16, 0.2 / 16, -0.3 / 16, 0.9 / 16)
    q = synth.queries_uniform(50, 41, const_derivs=d)
    k = 8
    r = oracle.filter_shade(tex, q, "linear", "ntap_before", "linear", spp=k * k, flags=oracle.FLAG_STRATIFIED)
    acc = np.zeros((q.n, 3))
    for s in range(k * k):
        jx, jy = (s % k + 0.5) / k - 0.5, (s // k + 0.5) / k - 0.5
        x = q.u.astype(np.float64) + jx * d[0] + jy * d[2]
        y = q.v.astype(np.float64) + jx * d[1] + jy * d[3]
        for c in range(3):
            acc[:, c] += ndimage.map_coordinates(img[..., c], [y * 16 - 0.5, x * 16 - 0.5], order=1,
                                                 mode="grid-wrap", prefilter=False)
    np.testing.assert_allclose(r.rgb, acc / (k * k), atol=1e-6)


# ------------------------------------------------------------------------ lattice sampler
def test_lattice_picks_are_stratified():
    # FLAG_LATTICE: the pick uniform of sample s is frac(s/spp + phi), so over the spp
    # samples of one query (no jitter, one level) each tap is chosen floor or ceil of
    # spp * p_k times -- the lattice's stratification, with the exact per-tap probability
    tex = _tiny_tex(16, seed=3)
    q = synth.queries_uniform(200, 81)
    spp = 16
    r = oracle.filter_shade(tex, q, "bspline", "stochastic", spp=spp, seed=5, flags=oracle.FLAG_LATTICE,
                            want_picks=True)
    for i in range(q.n):
        px = float(np.float32(q.u[i]) * np.float32(16)) - 0.5
        tx = px - math.floor(px)
        p = np.array([oracle.kernel("bspline", tx - k) for k in _taps("bspline")])
        ix0 = math.floor(px)
        xs = (r.picks64[i, :, 0] & 0x3FFF).astype(int)
        counts = np.array([np.sum(xs == (ix0 + k) % 16) for k in _taps("bspline")])
        assert np.all(np.abs(counts - spp * p) <= 1.0 + 1e-9), (counts, spp * p)


@pytest.mark.parametrize("f,mode", [("bspline", "stochastic"), ("mitchell", "positivized")])
def test_lattice_estimator_unbiased(f, mode):
    m = synth.material_rgba8(8, 3, octaves=3, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_uniform(4, 19, res=8, lod_range=2.5)
    d = []
    for seed in range(1, 2001):
        s = oracle.filter_shade(tex, q, f, mode, spp=4, seed=seed, flags=oracle.FLAG_LATTICE).rgb
        a = oracle.filter_shade(tex, q, f, "ntap_after", spp=4, seed=seed).rgb
        d.append(s - a)
    d = np.array(d)
    z = np.abs(d.mean(0)) / (d.std(0) / math.sqrt(len(d)) + 1e-12)
    assert z.max() < 4.5, z.max()


def test_volume_lattice_unbiased_and_lower_variance():
    vol = synth.volume_cloud(16, 5, zero_frac=0.5, octaves=3, base=2)
    W, H = 4, 3
    cam = synth.camera_pinhole(W, H).as_array()
    ind, lat = [], []
    for seed in range(1, 801):
        a = oracle.march(vol, 20.0, cam, W, H, 48, "bspline", "ntap_after", spp=8, seed=seed, pix_begin=5, pix_count=1).T[0]
        ind.append(oracle.march(vol, 20.0, cam, W, H, 48, "bspline", "stochastic", spp=8, seed=seed,
                                pix_begin=5, pix_count=1).T[0] - a)
        lat.append(oracle.march(vol, 20.0, cam, W, H, 48, "bspline", "stochastic", spp=8, seed=seed,
                                flags=oracle.FLAG_LATTICE, pix_begin=5, pix_count=1).T[0] - a)
    ind, lat = np.array(ind), np.array(lat)
    assert abs(lat.mean()) < 4 * lat.std() / math.sqrt(len(lat)) + 1e-12
    assert lat.std() < ind.std()


# ------------------------------------------------------------------------ sample reuse
@pytest.mark.parametrize("f", FILTERS)
def test_reuse_joint_distribution_by_enumeration(f):
    # one uniform drives both axes, remapped after the first decision: the u-measure of
    # every (kx, ky) cell equals p_x(kx) p_y(ky) (Eq. uniform-sample-reuse)
    rng = np.random.default_rng(17)
    m = 1 << 14
    for tx, ty in rng.random((3, 2)).astype(np.float32):
        wx, wy = oracle.weights32(f, tx), oracle.weights32(f, ty)
        px = np.abs(wx.astype(np.float64)); px /= px.sum()
        py = np.abs(wy.astype(np.float64)); py /= py.sum()
        hist = np.zeros((len(wx), len(wy)))
        for u in (np.arange(m) + 0.5) / m:
            kx, r = oracle.pick32_reuse(wx, u)
            ky, _ = oracle.pick32_reuse(wy, r)
            hist[kx, ky] += 1.0 / m
        np.testing.assert_allclose(hist, np.outer(px, py), atol=3.0 / m)


@pytest.mark.parametrize("f", ["bspline", "mitchell"])
def test_reuse_estimator_unbiased(f):
    m = synth.material_rgba8(8, 3, octaves=3, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_uniform(4, 23, res=8, lod_range=2.5)
    d = []
    for seed in range(1, 2001):
        s = oracle.filter_shade(tex, q, f, "stochastic", spp=4, seed=seed, flags=oracle.FLAG_REUSE).rgb
        a = oracle.filter_shade(tex, q, f, "ntap_after", spp=4, seed=seed).rgb
        d.append(s - a)
    d = np.array(d)
    z = np.abs(d.mean(0)) / (d.std(0) / math.sqrt(len(d)) + 1e-12)
    assert z.max() < 4.5, z.max()


def test_volume_reuse_unbiased():
    vol = synth.volume_cloud(16, 6, zero_frac=0.5, octaves=3, base=2)
    W, H = 4, 3
    cam = synth.camera_pinhole(W, H).as_array()
    d = []
    for seed in range(1, 1201):
        a = oracle.march(vol, 20.0, cam, W, H, 48, "bspline", "ntap_after", spp=1, seed=seed, pix_begin=5, pix_count=1).T[0]
        s = oracle.march(vol, 20.0, cam, W, H, 48, "bspline", "stochastic", spp=1, seed=seed, flags=oracle.FLAG_REUSE,
                         pix_begin=5, pix_count=1).T[0]
        d.append(s - a)
    d = np.array(d)
    assert abs(d.mean()) < 4 * d.std() / math.sqrt(len(d)) + 1e-12


# ------------------------------------------------------------------------ EWA (supplement "Stochastic EWA")
def test_ewa_table_closed_form():
    # 128 Gaussian weights exp(-2 r^2) - exp(-2) at r^2 = i/127: 1 - e^-2 at the centre, 0 at
    # the rim, strictly decreasing
    t = oracle.ewa_table().astype(np.float64)
    r2 = np.arange(128) / 127.0
    np.testing.assert_allclose(t, np.exp(-2 * r2) - math.exp(-2), rtol=1e-7, atol=1e-8)
    assert t[0] == np.float32(1 - math.exp(-2)) and t[127] == 0.0
    assert np.all(np.diff(t) < 0)


@pytest.mark.parametrize("case", [
    (0.31, 0.47, 0.0, 0.0, 0.0, 0.0, 64),                      # magnification: unit circle
    (0.5, 0.5, 8 / 64, 0.0, 0.0, 1 / 64, 64),                  # axis-aligned, 8 x 1 texels
    (0.2, 0.7, 0.09, 0.05, -0.012, 0.02, 64),                  # rotated, anisotropic
    (0.6, 0.3, 0.5 / 64, 1.2 / 64, 0.011 / 64, -0.005 / 64, 64),  # eccentricity above 64: capped
])
def test_ewa_weights_match_fp64_quadratic_form(case):
    # r^2 = x^T (J J^T + I)^-1 x: the covariance of the pixel footprint (columns of J = the
    # derivative vectors in texels, the minor one stretched to major/64 if the ratio is
    # larger) plus a one-texel reconstruction term.  Brute force in FP64 with numpy's
    # inverse; the FP32 weights must equal table[floor(128 r^2)] except at bin edges.
    x, y, a, b, c, d, R = case
    box, w = oracle.ewa_box(x, y, a, b, c, d, R, R)
    f32 = lambda z: float(np.float32(z))
    J = np.array([[f32(a) * R, f32(c) * R], [f32(b) * R, f32(d) * R]], dtype=np.float64)
    l0, l1 = np.linalg.norm(J[:, 0]), np.linalg.norm(J[:, 1])
    if min(l0, l1) > 0 and min(l0, l1) * 64 < max(l0, l1):
        k = 0 if l0 < l1 else 1
        J[:, k] *= max(l0, l1) / (min(l0, l1) * 64)
    Minv = np.linalg.inv(J @ J.T + np.eye(2))
    cx, cy = f32(x) * R - 0.5, f32(y) * R - 0.5
    table = oracle.ewa_table()
    s0, s1, t0, t1 = box
    checked = 0
    for t in range(t0, t1 + 1):
        for s in range(s0, s1 + 1):
            p = np.array([s - cx, t - cy])
            r2 = float(p @ Minv @ p)
            got = w[t - t0, s - s0]
            if abs(r2 - 1.0) < 1e-4 or abs(r2 * 128 - round(r2 * 128)) < 1e-3:
                continue      # FP32 and FP64 may fall on either side of an edge
            want = table[int(r2 * 128)] if r2 < 1.0 else 0.0
            assert got == want, (s, t, r2, got, want)
            checked += 1
    assert checked > 0
    # the box covers the ellipse: no texel just outside it is inside the ellipse
    for t in range(t0 - 1, t1 + 2):
        for s in (s0 - 1, s1 + 1):
            p = np.array([s - cx, t - cy])
            assert float(p @ Minv @ p) > 1.0 - 1e-4


def _ewa_query(du0, dv0, du1, dv1, n=1, u=0.37, v=0.61):
    f = lambda z: np.full(n, z, dtype=np.float32)
    return synth.Queries(f(u), f(v), f(du0), f(dv0), f(du1), f(dv1))


def test_ewa_magnification_at_texel_centre_is_point_sample():
    # zero footprint at a texel centre: the unit circle holds only that texel (its
    # neighbours are at r^2 = 1, outside), so every EWA mode returns that texel exactly
    tex = _tiny_tex(8, seed=23)
    img = tex.levels[0].astype(np.float64)
    q = synth.Queries(np.array([2.5 / 8], np.float32), np.array([5.5 / 8], np.float32))
    want = oracle.shade_batch(img[5, 2, :3][None], [img[5, 2, 3]], [[0, 0, 1]])[0]
    for mode in ("ntap_before", "ntap_after", "stochastic"):
        r = oracle.filter_shade(tex, q, "ewa", mode, spp=2, want_picks=True)
        np.testing.assert_allclose(r.rgb[0], want, rtol=1e-12)
        if mode == "stochastic":
            assert np.all(r.picks64[0, :, 0] == ((5 << 14) | 2))


def test_ewa_constant_texture_reproduced():
    c = np.zeros((16, 16, 4), dtype=np.float32)
    c[...] = [0.3, 0.5, 0.1, 0.6]
    tex = oracle.Texture([c])
    q = synth.queries_aniso(200, 3, res=16, lod_range=1.0, max_aniso=16)
    want = oracle.shade_batch(c[0, 0, :3].astype(np.float64)[None], [c[0, 0, 3]], [[0, 0, 1]])[0]
    for mode in ("ntap_before", "ntap_after", "stochastic"):
        r = oracle.filter_shade(tex, q, "ewa", mode, spp=3)
        np.testing.assert_allclose(r.rgb, np.broadcast_to(want, r.rgb.shape), rtol=1e-12)


def test_ewa_stochastic_pick_frequencies_follow_weights():
    # the reservoir pick over the ellipse chooses texel i with probability w_i / sum w:
    # chi-square of 2^16 picks of one query (one level) against the table weights
    tex = _tiny_tex(64, seed=5)
    q = _ewa_query(5 / 64, 1.5 / 64, -0.8 / 64, 2.2 / 64)
    spp = 1 << 16
    r = oracle.filter_shade(tex, q, "ewa", "stochastic", spp=spp, seed=9, flags=oracle.FLAG_LOD0, want_picks=True)
    box, w = oracle.ewa_box(q.u[0], q.v[0], q.dudx[0], q.dvdx[0], q.dudy[0], q.dvdy[0], 64, 64)
    s0, s1, t0, t1 = box
    pk = r.picks64[0, :, 0]
    ix, iy = pk & 0x3FFF, (pk >> 14) & 0x3FFF
    counts = np.zeros_like(w, dtype=np.float64)
    ss = (np.arange(s0, s1 + 1) % 64)
    tt = (np.arange(t0, t1 + 1) % 64)
    for j, t in enumerate(tt):
        for i, s in enumerate(ss):
            counts[j, i] = np.count_nonzero((ix == s) & (iy == t))
    assert counts[w == 0].sum() == 0
    p = w[w > 0].astype(np.float64) / w.sum(dtype=np.float64)
    e = spp * p
    chi2 = float(((counts[w > 0] - e) ** 2 / e).sum())
    dof = p.size - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_ewa_stochastic_mean_converges_to_filter_after():
    # unbiasedness: with the same seeds the stochastic level choice is shared, and the
    # single-tap mean converges to the N-tap filter-after value (3 sigma on the difference)
    m = synth.material_rgba8(32, 6, octaves=4, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_aniso(6, 8, res=32, lod_range=2.0, max_aniso=8)
    spp = 1 << 14
    s = oracle.filter_shade(tex, q, "ewa", "stochastic", spp=spp, seed=4)
    a = oracle.filter_shade(tex, q, "ewa", "ntap_after", spp=1, seed=4)
    small = np.array([oracle.filter_shade(tex, q, "ewa", "stochastic", spp=1, seed=500 + k).rgb for k in range(256)])
    sd = small.std(axis=0) + 1e-6
    z = np.abs(s.rgb - a.rgb) / (sd / math.sqrt(spp))
    assert z.max() < 4.5, z.max()


def test_lod0_flag_uses_the_finest_level_only():
    m = synth.material_rgba8(32, 6, octaves=4, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_aniso(200, 11, res=32, lod_range=4.0)
    for f in ("bspline", "ewa"):
        r = oracle.filter_shade(tex, q, f, "stochastic", spp=2, flags=oracle.FLAG_LOD0, want_picks=True)
        assert np.all((r.picks64[..., 0] >> 28) == 0)
        base = oracle.filter_shade(tex, q, f, "stochastic", spp=2, want_picks=True)
        assert np.any((base.picks64[..., 0] >> 28) > 0)


# ------------------------------------------------------------------------ DCT texture compression
def _dct_coeffs(word):
    # dequantised 8 x 8 coefficient array X[v, u] of one channel word (zeros elsewhere)
    X = np.zeros((8, 8))
    X[0, 0] = (word & 127) * 8.0 / 127.0
    for j, (u, v) in enumerate(synth.DCT_AC):
        X[v, u] = (((word >> (7 + 5 * j)) & 31) - 15) * 2.0 / 15.0
    return X


def test_dct_decode_matches_scipy_inverse_dct():
    # the oracle's restricted basis sum equals scipy's orthonormal 2-D inverse DCT of the
    # dequantised coefficients, at every texel of the block
    from scipy.fft import idctn
    rng = np.random.default_rng(3)
    for word in rng.integers(0, 1 << 32, 12, dtype=np.uint64):
        word = int(word) & 0xFFFFFFFF
        ref = idctn(_dct_coeffs(word), type=2, norm="ortho")    # ref[y, x]
        got = np.array([[oracle.dct_texel(word, x, y) for x in range(8)] for y in range(8)])
        np.testing.assert_allclose(got, ref, atol=1e-12)


def test_dct_roundtrip_and_constant_blocks():
    # smooth content survives within the quantisation error; a constant on the DC grid is exact
    n = 64
    yy, xx = np.mgrid[0:n, 0:n] / n
    smooth = 0.5 + 0.25 * np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * yy)
    b = synth._rne_u8(255 * smooth)
    m = synth.Material([np.repeat(b[..., None], 4, axis=2)], [np.repeat(b[..., None], 2, axis=2)], smooth)
    blk = synth.dct_compress(m)[0].view(np.uint32).reshape(n // 8, n // 8, 8)
    dec = np.array([[oracle.dct_texel(int(blk[y // 8, x // 8, 0]), x % 8, y % 8) for x in range(n)] for y in range(n)])
    # quantisation bound: half a DC step times 1/8 plus five half AC steps times the largest
    # basis value 1/4 (~0.087), and the truncated higher frequencies of the sine are small
    err = dec - b / 255.0
    assert np.abs(err).max() < 0.087 and np.sqrt(np.mean(err ** 2)) < 0.02, (np.abs(err).max(), np.sqrt(np.mean(err ** 2)))
    c = 64 / 127                        # DC = 8 c lands on the 7-bit grid
    m2 = synth.Material([np.full((16, 16, 4), 0, np.uint8)], [np.full((16, 16, 2), 0, np.uint8)], None)
    word = (64 | (15 << 7) | (15 << 12) | (15 << 17) | (15 << 22) | (15 << 27))
    assert all(abs(oracle.dct_texel(word, x, y) - c) < 1e-15 for x in range(8) for y in range(8))
    blk2 = synth.dct_compress(m2)[0].view(np.uint32)
    assert np.all(blk2[..., :6] == (15 << 7) | (15 << 12) | (15 << 17) | (15 << 22) | (15 << 27))


def test_dct_texture_filters_reproduce_a_constant():
    # every stored word decodes to the same constant: all estimators return its shade
    word = (64 | (15 << 7) | (15 << 12) | (15 << 17) | (15 << 22) | (15 << 27))
    blocks = [np.tile(np.array([word] * 6 + [0, 0], np.uint32), (2, 2, 1)).view(np.uint8)]
    tex = oracle.Texture([(16, 16)], dct=blocks)
    c = 64 / 127
    nx = 2 * c - 1
    nz = math.sqrt(max(0.0, 1 - 2 * nx * nx))
    want = oracle.shade_batch(np.array([[c, c, c]]), [0.05 + 0.95 * c], [[nx, nx, nz]])[0]
    q = synth.queries_uniform(200, 4, const_derivs=(1 / 64, 0.0, 0.0, 1 / 64))
    for f, mode in (("linear", "stochastic"), ("bspline", "ntap_before"), ("linear", "ntap_after")):
        r = oracle.filter_shade(tex, q, f, mode, spp=2)
        np.testing.assert_allclose(r.rgb, np.broadcast_to(want, r.rgb.shape), rtol=1e-12)


# ------------------------------------------------------------------------ Gaussian filters and FIS
@pytest.mark.parametrize("sigma", [0.3, 0.5, 0.8])
def test_gauss_ntap_matches_scipy_gaussian_filter(sigma):
    # the discrete Gaussian filter at texel centres (t = 0) is scipy's sampled, normalised
    # Gaussian kernel with periodic addressing; our window reaches ceil(5 sigma) + 1 texels
    tex = _tiny_tex(16, seed=19)
    img = tex.levels[0].astype(np.float64)
    iy, ix = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    q = synth.Queries(((ix.ravel() + 0.5) / 16).astype(np.float32), ((iy.ravel() + 0.5) / 16).astype(np.float32))
    r = oracle.filter_shade(tex, q, "gauss", "ntap_before", "linear", sigma=sigma)
    s32 = float(np.float32(sigma))             # the API's sigma is FP32
    R = math.ceil(5 * s32) + 1
    for c in range(3):
        ref = ndimage.gaussian_filter(img[..., c], s32, mode="wrap", truncate=(R + 0.25) / s32)
        np.testing.assert_allclose(r.rgb[:, c].reshape(16, 16), ref, atol=1e-10)


def test_box_gaussian_weights_integrate_the_density():
    # the FIS Gaussian's N-tap form weighs texel i by the Gaussian mass over its cell
    # [i - 1/2, i + 1/2] (in texel-centre coordinates): checked against scipy's quadrature
    tex = _tiny_tex(16, seed=20)
    img = tex.levels[0].astype(np.float64)
    q = synth.queries_uniform(6, 22)
    sigma = float(np.float32(0.6))
    r = oracle.filter_shade(tex, q, "gauss", "ntap_before", "linear", sampler="fis", sigma=sigma)
    pdf = lambda z: math.exp(-0.5 * (z / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))
    for i in range(q.n):
        px, py = float(np.float32(q.u[i]) * np.float32(16)) - 0.5, float(np.float32(q.v[i]) * np.float32(16)) - 0.5
        ks = np.arange(math.floor(px) - 8, math.floor(px) + 10)
        wx = np.array([integrate.quad(pdf, k - 0.5 - px, k + 0.5 - px)[0] for k in ks])
        ls = np.arange(math.floor(py) - 8, math.floor(py) + 10)
        wy = np.array([integrate.quad(pdf, l - 0.5 - py, l + 0.5 - py)[0] for l in ls])
        w = np.outer(wy / wy.sum(), wx / wx.sum())
        ref = np.einsum("yx,yxc->c", w, img[np.ix_(ls % 16, ks % 16)][..., :3])
        np.testing.assert_allclose(r.rgb[i], ref, atol=1e-9)


@pytest.mark.parametrize("filter,sampler,target,sigma", [
    ("linear", "fis", ("linear", "frs"), 0.5), ("bspline", "fis", ("bspline", "frs"), 0.5),
    ("gauss", "fis", ("gauss", "fis"), 0.4), ("gauss", "fis", ("gauss", "fis"), 0.8),
    ("gauss", "frs", ("gauss", "frs"), 0.5)])
def test_fis_and_frs_gaussian_means_converge(filter, sampler, target, sigma):
    # unbiasedness: the 1-tap mean converges to the N-tap filter it samples.  FIS with a
    # nearest lookup realises the sampled density convolved with the box: the tent from a
    # box, the cubic B-spline from the quadratic one (Cox-de Boor), the box-convolved Gaussian
    # from the Gaussian.  FRS's 4 x 4 Gaussian window is exact to ~3e-4 at sigma 0.5.
    tex = _tiny_tex(16, seed=21)
    q = synth.queries_uniform(8, 23)
    spp = 1 << 15
    s = oracle.filter_shade(tex, q, filter, "stochastic", "linear", spp=spp, seed=3, sampler=sampler, sigma=sigma)
    a = oracle.filter_shade(tex, q, target[0], "ntap_after", "linear", sampler=target[1], sigma=sigma)
    small = np.array([oracle.filter_shade(tex, q, filter, "stochastic", "linear", spp=1, seed=900 + k,
                                          sampler=sampler, sigma=sigma).rgb for k in range(256)])
    sd = small.std(axis=0) + 1e-6
    z = np.abs(s.rgb - a.rgb) / (sd / math.sqrt(spp))
    tol = 4.5 + (0 if filter != "gauss" or sampler != "frs" else 3e-4 / (sd.min() / math.sqrt(spp)))
    assert z.max() < tol, z.max()


def test_gaussian_and_fis_reproduce_a_constant():
    c = np.zeros((16, 16, 4), dtype=np.float32)
    c[...] = [0.2, 0.7, 0.4, 0.5]
    tex = oracle.Texture([c])
    q = synth.queries_uniform(100, 5, const_derivs=(1 / 64, 0.0, 0.0, 1 / 64))
    want = oracle.shade_batch(c[0, 0, :3].astype(np.float64)[None], [c[0, 0, 3]], [[0, 0, 1]])[0]
    for f, sm, mode in (("gauss", "frs", "stochastic"), ("gauss", "frs", "ntap_after"), ("gauss", "fis", "stochastic"),
                        ("gauss", "fis", "ntap_before"), ("bspline", "fis", "stochastic"), ("linear", "fis", "stochastic")):
        r = oracle.filter_shade(tex, q, f, mode, spp=3, sampler=sm, sigma=0.7)
        np.testing.assert_allclose(r.rgb, np.broadcast_to(want, r.rgb.shape), rtol=1e-12)
