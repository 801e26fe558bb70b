"""Pins of the oracle's interpolation (Def. 2 / Eqs. 3-4 B-spline, Def. 3 /
Eqs. 5-7 Akima, straight-line interpolation) against textbook properties and
scipy's independent spline routines."""
import os

import numpy as np
import pytest
from scipy.interpolate import Akima1DInterpolator, BSpline

from paper_2505_01059_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("M,H", [(6, 17), (8, 64), (16, 256), (7, 5)])
def test_bspline_basis_matches_scipy(orc, p, M, H):
    """Cox-de Boor (Eq. 4) on the Def. 2 knots t_i = i/(M+p+1) equals scipy's
    B-spline basis elements at every evaluation time, both time readings."""
    if M < p + 1:
        pytest.skip("valid span needs M >= p + 1")
    knots = np.arange(M + p + 1) / (M + p + 1)
    for mapping in ("valid_span", "paper_literal"):
        Bm = orc.bspline_basis(M, p, H, mapping)
        ts = np.array([orc.bspline_time(M, p, H, mapping, j) for j in range(H)])
        for m in range(M):
            elem = BSpline.basis_element(knots[m:m + p + 2], extrapolate=False)
            ref = np.nan_to_num(elem(ts))
            # Eq. 4's indicator is half-open: zero at the right end of the support
            ref[ts == knots[m + p + 1]] = 0.0
            if mapping == "valid_span" and H > 1:
                # right end of the valid span: the last interval is closed (left limit)
                ref[-1] = np.nan_to_num(elem(np.nextafter(ts[-1], -1.0)))
                if p == 0:
                    ref[-1] = 1.0 if m == M - 1 else 0.0
            np.testing.assert_allclose(Bm[m], ref, atol=1e-12)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
def test_bspline_partition_of_unity_valid_span(orc, p):
    # Eq. 3: the weights sum to one on the valid span, and are >= 0.
    for M in range(p + 1, 17):
        for H in (1, 2, 3, 64, 129):
            Bm = orc.bspline_basis(M, p, H, "valid_span")
            np.testing.assert_allclose(Bm.sum(axis=0), 1.0, atol=1e-12)
            assert Bm.min() >= -1e-15


def test_bspline_paper_literal_loses_unity_at_ends(orc):
    # With t_j = j/T (Def. 2 as printed) the sum drops below 1 near t = 0.
    Bm = orc.bspline_basis(8, 3, 64, "paper_literal")
    s = Bm.sum(axis=0)
    assert s[0] < 1e-12 and s[len(s) // 2] == pytest.approx(1.0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_bspline_reproduces_linear_data(orc, p):
    """Control points on a line at the Greville abscissae reproduce the line
    exactly (Marsden's identity), a textbook consequence of Eq. 3."""
    M, H = 9, 37
    K = M + p + 1
    knots = np.arange(K) / K
    greville = np.array([knots[i + 1:i + p + 1].mean() for i in range(M)])
    a, b = 0.3, -1.7
    spec = W.pointmass(k=1, M=M, N=2, H=H, interp="bspline", degree=p, u_min=[-10], u_max=[10])
    C = (a + b * greville)[None, :, None]
    U = orc.interpolate(spec, C)
    ts = np.array([orc.bspline_time(M, p, H, "valid_span", j) for j in range(H)])
    np.testing.assert_allclose(U[0, :, 0], a + b * ts, atol=1e-13)


def test_bspline_convex_hull(orc):
    spec = W.pointmass(k=3, M=8, N=16, H=50, interp="bspline", degree=3)
    rng = np.random.default_rng(1)
    C = rng.uniform(-1, 1, size=(40, 8, 3))
    U = orc.interpolate(spec, C)
    for b in range(40):
        lo = C[b].min(axis=0)
        hi = C[b].max(axis=0)
        assert np.all(U[b] >= lo - 1e-12) and np.all(U[b] <= hi + 1e-12)


def test_bspline_degree0_is_piecewise_constant(orc):
    M, H = 5, 21
    Bm = orc.bspline_basis(M, 0, H, "valid_span")
    assert set(np.unique(Bm)) <= {0.0, 1.0}
    # each time step picks the layer whose knot interval contains it
    ts = np.array([orc.bspline_time(M, 0, H, "valid_span", j) for j in range(H)])
    expect = np.minimum(np.floor(ts * (M + 1)).astype(int), M - 1)
    np.testing.assert_array_equal(Bm.argmax(axis=0), expect)


def _hand_slopes():
    rows = []
    with open(os.path.join(GOLDEN, "akima_hand_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            i, s = line.split()
            rows.append(float(s))
    return np.array(rows)


def test_akima_slopes_hand_example(orc):
    tk = np.arange(7.0)
    z = np.array([0, 0, 1, 1, 0, 0, 0], float)
    coef = orc.akima_coeffs(tk, z)
    s = np.append(coef[:, 1], 0.0)  # b_i = s_i (Eq. 7); s_M from the last piece below
    # slope at the right end of the last piece is s_M
    a, b, c, d = coef[-1]
    s[-1] = b + 2 * c * 1.0 + 3 * d * 1.0
    np.testing.assert_allclose(s, _hand_slopes(), atol=1e-14)


def test_akima_interior_slopes_match_scipy(orc):
    """Eq. 6 at the interior knots 3..M-2 equals scipy's Akima slopes (scipy
    uses other end rules, so only the interior is compared)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        M = int(rng.integers(6, 16))
        tk = np.sort(rng.uniform(0, 1, M))
        tk[0], tk[-1] = 0.0, 1.0
        z = rng.normal(size=M)
        coef = orc.akima_coeffs(tk, z)
        ref = Akima1DInterpolator(tk, z)
        deriv = ref.derivative()(tk)
        # paper index i (1-based) 3..M-2 -> 0-based 2..M-3
        for i in range(2, M - 2):
            assert coef[i, 1] == pytest.approx(deriv[i], rel=1e-11, abs=1e-12)


def test_akima_end_rules_literal(orc):
    rng = np.random.default_rng(4)
    M = 9
    tk = np.linspace(0, 1, M)
    z = rng.normal(size=M)
    coef = orc.akima_coeffs(tk, z)
    m = np.diff(z) / np.diff(tk)
    s1, s2, sM1 = coef[0, 1], coef[1, 1], coef[M - 2, 1]
    a, b, c, d = coef[-1]
    h = tk[-1] - tk[-2]
    sM = b + 2 * c * h + 3 * d * h * h
    assert s1 == pytest.approx(m[0], rel=1e-13)
    assert s2 == pytest.approx((m[0] + m[1]) / 2, rel=1e-13)
    assert sM1 == pytest.approx((m[M - 2] + m[M - 3]) / 2, rel=1e-13)
    assert sM == pytest.approx(m[M - 2], rel=1e-10)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 8, 16])
def test_akima_through_knots_and_c1(orc, M):
    rng = np.random.default_rng(M)
    tk = np.linspace(0, 1, M)
    z = rng.normal(size=M)
    coef = orc.akima_coeffs(tk, z)
    for i in range(M - 1):
        h = tk[i + 1] - tk[i]
        a, b, c, d = coef[i]
        # interpolation at both ends of each piece (Eq. 5)
        assert a == z[i]
        assert a + b * h + c * h * h + d * h ** 3 == pytest.approx(z[i + 1], abs=1e-12)
        if i + 1 < M - 1:
            # C1: the right derivative of piece i equals the slope of piece i+1
            right = b + 2 * c * h + 3 * d * h * h
            assert right == pytest.approx(coef[i + 1, 1], abs=1e-11)


@pytest.mark.parametrize("M", [2, 3, 4, 6, 11])
def test_akima_exact_on_linear_data(orc, M):
    spec = W.pointmass(k=2, M=M, N=2, H=33, interp="akima", u_min=[-10, -10], u_max=[10, 10])
    tk = np.array([orc.akima_knot(M, "valid_span", i) for i in range(M)])
    C = np.stack([0.5 - 2.0 * tk, 1.0 + 0.25 * tk], axis=-1)[None]
    U = orc.interpolate(spec, C)
    ts = np.array([orc.akima_time(33, "valid_span", j) for j in range(33)])
    np.testing.assert_allclose(U[0, :, 0], 0.5 - 2.0 * ts, atol=1e-13)
    np.testing.assert_allclose(U[0, :, 1], 1.0 + 0.25 * ts, atol=1e-13)


def test_akima_paper_literal_extrapolates(orc):
    # Def. 3 as printed: knots i/M, times j/T; times past the last knot use the last cubic.
    M, H = 4, 16
    spec = W.pointmass(k=1, M=M, N=2, H=H, interp="akima", time_mapping="paper_literal",
                       u_min=[-10], u_max=[10])
    z = np.array([0.0, 1.0, 0.0, 2.0])
    U = orc.interpolate(spec, z[None, :, None])
    tk = np.arange(M) / M
    coef = orc.akima_coeffs(tk, z)
    t = (H - 1) / H
    a, b, c, d = coef[-1]
    dt = t - tk[-2]
    assert U[0, -1, 0] == pytest.approx(a + b * dt + c * dt * dt + d * dt ** 3, abs=1e-14)
    assert U[0, 0, 0] == 0.0


def test_linear_interpolation(orc):
    M, H = 5, 41
    spec = W.pointmass(k=1, M=M, N=2, H=H, interp="linear", u_min=[-10], u_max=[10])
    z = np.array([0.0, 1.0, -1.0, 0.5, 2.0])
    U = orc.interpolate(spec, z[None, :, None])
    ts = np.linspace(0, 1, H)
    np.testing.assert_allclose(U[0, :, 0], np.interp(ts, np.linspace(0, 1, M), z), atol=1e-14)


# ----------------------------------------------------------------------------
# BF16 operands of the B-spline contraction
# ----------------------------------------------------------------------------

def _bf16_bits(x):
    """Independent reference: round float32 values to bfloat16 through their
    IEEE-754 encoding (keep the high 16 bits, round half to even)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_round_known_values(orc):
    # published bfloat16 encodings: pi = 0x4049, 0.1 = 0x3DCD
    assert orc.bf16_round(np.pi)[0] == 3.140625
    assert orc.bf16_round(0.1)[0] == 0.10009765625
    # ties go to the even significand (ulp of [1, 2) is 2^-7)
    assert orc.bf16_round(1 + 2.0 ** -8)[0] == 1.0
    assert orc.bf16_round(1 + 3 * 2.0 ** -8)[0] == 1 + 2.0 ** -6
    assert orc.bf16_round(-(1 + 3 * 2.0 ** -8))[0] == -(1 + 2.0 ** -6)
    assert orc.bf16_round(65408.0)[0] == 65536.0  # 255.5 * 256 -> 256 * 256
    assert orc.bf16_round(0.0)[0] == 0.0


def test_bf16_round_matches_bit_rounding(orc):
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(4000) * 10.0 ** rng.uniform(-6, 6, 4000)).astype(np.float32)
    assert np.array_equal(orc.bf16_round(x.astype(np.float64)), _bf16_bits(x))


@pytest.mark.parametrize("p", [2, 3])
def test_bf16_bspline_within_operand_rounding(orc, p):
    """Each operand moves by at most 2^-8 of itself (the unit roundoff of an
    8-bit significand), so with a non-negative basis summing to one the
    result moves by at most ~2^-7 max|C|."""
    spec = W.pointmass(k=3, M=8, H=64, degree=p)
    rng = np.random.default_rng(p)
    Cc = rng.uniform(-1, 1, size=(40, spec["M"], 3))
    U64 = orc.interpolate(spec, Cc)
    U16 = orc.interpolate(dict(spec, flags=0x4), Cc)
    err = np.abs(U16 - U64).max()
    assert 0 < err <= 2.0 ** -7 * np.abs(Cc).max() * 1.01
    assert np.abs(U16 - U64).max() / np.abs(U64).max() < 1e-2


def test_bf16_bspline_exact_when_operands_are_bf16(orc):
    """Degree 1, M = 5, H = 9 (valid span) samples the piecewise-linear
    interpolant at the knots and the midpoints (basis values 0, 1/2, 1); with
    knots on a 2^-6 grid every BF16 operand is exact, so the result is the
    closed form exactly (the FP64 basis itself is only within 1e-16 of 1/2)."""
    spec = W.pointmass(k=2, M=5, H=9, degree=1)
    rng = np.random.default_rng(3)
    Cc = rng.integers(-64, 65, size=(7, 5, 2)) / 64.0
    want = np.empty((7, 9, 2))
    want[:, 0::2] = Cc
    want[:, 1::2] = 0.5 * (Cc[:, :-1] + Cc[:, 1:])
    assert np.array_equal(orc.interpolate(dict(spec, flags=0x4), Cc), want)
