"""Pins of the algebraic rewrites the float32 sweep makes (stream_x2.cuh),
checked on the host with numpy against the formulas they replace (ppm.cuh
and the oracle follow the formulas as written):

* the limited slope with its sign test folded into the minimum;
* the two-shock solver's shock-curve quantities with shared reciprocals;
* the parabola averages of tracing from the right and left edges with the
  wave's coefficients negated or sign-flipped, as the lane pairs use them.

No GPU: these are statements about real arithmetic (and float32 rounding
where the rewrite claims equality)."""
import numpy as np

RNG = np.random.default_rng(7)
F32 = np.float32


def _triples(n):
    cont = [RNG.standard_normal(n) for _ in range(3)]
    rounded = [np.round(RNG.standard_normal(n), 1) for _ in range(3)]   # many exact ties and zeros
    am, a0, ap = [np.where(RNG.random(n) < 0.5, c, r).astype(np.float32) for c, r in zip(cont, rounded)]
    am[: n // 20] = a0[: n // 20]
    ap[n // 20: n // 10] = a0[n // 20: n // 10]
    return am, a0, ap


def test_sign_folded_limiter_equals_the_select_form():
    """s = sign(da): s*dl and s*dr are both positive exactly where dl*dr > 0,
    so s * max(min(|da|, 2 min(s dl, s dr)), 0) equals the select form
    (dl*dr > 0 ? copysign(min(|da|, 2|dl|, 2|dr|), da) : 0) in float32, up to
    the sign of a zero slope."""
    am, a0, ap = _triples(400_000)
    dl, dr = a0 - am, ap - a0
    da = F32(0.5) * (ap - am)
    sel = np.where(dl * dr > 0,
                   np.copysign(np.minimum(np.abs(da), np.minimum(F32(2) * np.abs(dl), F32(2) * np.abs(dr))), da),
                   F32(0))
    s = np.copysign(F32(1), da)
    fold = s * np.maximum(np.minimum(np.abs(da), F32(2) * np.minimum(s * dl, s * dr)), F32(0))
    assert sel.dtype == fold.dtype == np.float32
    assert np.array_equal(sel, fold)                      # equal as values (-0 == +0)
    nonzero = sel != 0
    assert np.array_equal(sel[nonzero].view(np.int32), fold[nonzero].view(np.int32))
    assert nonzero.mean() > 0.2 and (~nonzero).mean() > 0.2


def test_limiter_fold_keeps_the_sign_test_when_da_is_zero():
    """da = 0 with dl, dr of opposite signs (a local extremum): slope 0."""
    dl = np.array([1.0, -2.0, 0.0], dtype=np.float32)
    dr = np.array([-1.0, 2.0, 3.0], dtype=np.float32)
    da = F32(0.5) * (dl + dr)
    s = np.copysign(F32(1), da)
    fold = s * np.maximum(np.minimum(np.abs(da), F32(2) * np.minimum(s * dl, s * dr)), F32(0))
    assert np.all(fold == 0)


def _states(n):
    r = np.exp(RNG.uniform(-6, 3, n))
    p = np.exp(RNG.uniform(-8, 4, n))
    ps = p * np.exp(RNG.uniform(-3, 3, n))    # a trial star pressure on either side of p
    return r, p, ps


def test_shock_curve_rewrite_matches_the_literal_formulas():
    """With C = sqrt(gamma p rho) and x = 1 + g1 (p*/p - 1) = (g1/p) p* + (1 -
    g1): W = C sqrt(x), (p* - p)/W = (p* - p) rsqrt(x)/C and Z = 2 W^3 / (W^2
    + C^2) = 2 W x / (x + 1), in float64 to rounding."""
    gamma = 5.0 / 3.0
    g1 = (gamma + 1.0) / (2.0 * gamma)
    r, p, ps = _states(200_000)
    C = np.sqrt(gamma * p * r)
    W_lit = C * np.sqrt(1.0 + g1 * (ps / p - 1.0))
    du_lit = (ps - p) / W_lit
    Z_lit = 2.0 * W_lit ** 3 / (W_lit ** 2 + C ** 2)
    q = gamma * p * r
    iC = 1.0 / np.sqrt(q)
    C2 = q * iC
    x = (g1 / p) * ps + (1.0 - g1)
    rx = 1.0 / np.sqrt(x)
    W = C2 * (x * rx)
    du = (ps - p) * (iC * rx)
    Z = 2.0 * W * x / (x + 1.0)
    for got, want in ((C2, C), (W, W_lit), (Z, Z_lit)):
        assert np.max(np.abs(got - want) / np.abs(want)) < 1e-13
    scale = np.maximum(np.abs(du_lit), 1e-300)
    assert np.max(np.abs(du - du_lit) / scale) < 1e-12


def test_edge_averages_with_negated_coefficients():
    """The right-edge average aR - (s/2)(da - (1 - 2s/3) a6) as fma(nh,
    fma(nk, a6, da), aR) with nk = 2s/3 - 1, nh = -s/2; the left-edge average
    over t = -s, aL + (t/2)(da + (1 - 2t/3) a6), as fma(nh, fma(kp, a6, da),
    aL) with kp = 1 + 2s/3.  The coefficients are exact negations or the same
    rounded values, so in float64 the rewrites agree with the formulas to
    rounding."""
    n = 100_000
    aL, aR, a6 = (RNG.standard_normal(n) for _ in range(3))
    s = RNG.uniform(-1, 1, n)
    da = aR - aL
    right = aR - (0.5 * s) * (da - (1.0 - (2.0 / 3.0) * s) * a6)
    t = -s
    left = aL + (0.5 * t) * (da + (1.0 - (2.0 / 3.0) * t) * a6)
    nk, kp, nh = (2.0 / 3.0) * s - 1.0, 1.0 + (2.0 / 3.0) * s, -0.5 * s
    right2 = nh * (nk * a6 + da) + aR
    left2 = nh * (kp * a6 + da) + aL
    mag = 1.0 + np.abs(aL) + np.abs(aR) + np.abs(a6)
    assert np.max(np.abs(right2 - right) / mag) < 1e-14
    assert np.max(np.abs(left2 - left) / mag) < 1e-14
    # the negation identities themselves are exact in binary floating point
    assert np.array_equal(-(1.0 - (2.0 / 3.0) * s), (2.0 / 3.0) * s - 1.0)
    assert np.array_equal(1.0 - (2.0 / 3.0) * t, 1.0 + (2.0 / 3.0) * s)
