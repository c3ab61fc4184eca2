"""The error bounds the GPU filters rest on, checked against emulated
roundings on the CPU (no GPU): a filter only rules candidates out, so each
bound must hold for every input, or the exact result could be lost.

- E4M3 operand rows (the FP8 distance tiles): a row x' is scaled by the
  power of two s = 2^e, e the smallest with max|x'_t| <= 448 s, and rounded
  to E4M3 (3 mantissa bits, exponent bias 7, subnormal spacing 2^-9,
  saturating at 448). The tile's certificate assumes |x^ . y^ - x' . y'|
  <= (2u + u^2 + 2 sqrt(d)(1 + u) c + d c^2) ||x'|| ||y'|| with u = 2^-4,
  c = 2^-10 2/448 (products exact, accumulation counted separately).
- BF16 rows of the refinement and Alg. 3 filters: h = bf16(fl(x - m)) and
  the per-row bound eb = sqrt_ru(sum (h - fl(x - m))^2)(1 + 2^-12) +
  ||fl(x - m)||(1 + 2^-12) 2^-22 must bound ||h - (x - m)|| (x - m exact).
"""
import numpy as np

RNG = np.random.default_rng(20260)


def e4m3(v):
    """Round float64 values to E4M3 (round to nearest, ties to even,
    saturating at +-448)."""
    v = np.asarray(v, np.float64)
    a = np.abs(v)
    with np.errstate(divide="ignore"):
        ex = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    ex = np.maximum(ex, -6.0)            # below 2^-6: subnormal spacing 2^-9
    q = np.exp2(ex - 3.0)
    r = np.round(a / q) * q              # numpy rounds half to even
    r = np.minimum(r, 448.0)
    return np.sign(v) * r


def row_scale(x):
    amax = np.max(np.abs(x))
    if amax == 0:
        return 1.0
    e = int(np.floor(np.log2(amax / 448.0)))
    while 448.0 * 2.0 ** (e - 1) >= amax:
        e -= 1
    while 448.0 * 2.0 ** e < amax:
        e += 1
    return 2.0 ** max(min(e, 127), -126)


def eps_e4m3(d):
    u, c = 1.0 / 16.0, 2.0 / 448.0 / 1024.0
    return 2 * u + u * u + 2 * np.sqrt(d) * (1 + u) * c + d * c * c


def _rows(kind, d):
    if kind == "gauss":
        return RNG.standard_normal(d)
    if kind == "heavy":
        return RNG.standard_cauchy(d)
    if kind == "spiky":   # one large coordinate, the rest tiny: subnormal codes
        x = 1e-6 * RNG.standard_normal(d)
        x[RNG.integers(d)] = 1e3
        return x
    if kind == "ties":    # exact halfway points of the E4M3 grid
        return (RNG.integers(0, 16, d) + 0.5) * 2.0 ** RNG.integers(-8, 4, d)
    return RNG.uniform(-1, 1, d) * 10.0 ** RNG.integers(-20, 20)


def test_e4m3_dot_error_bound_holds():
    worst = 0.0
    for d in (3, 32, 128, 200, 512):
        for kind in ("gauss", "heavy", "spiky", "ties", "scaled"):
            for _ in range(40):
                x, y = _rows(kind, d), _rows(kind, d)
                sx, sy = row_scale(x), row_scale(y)
                xq, yq = e4m3(x / sx) * sx, e4m3(y / sy) * sy
                assert np.all(np.abs(x / sx) <= 448.0) and np.all(np.abs(y / sy) <= 448.0)
                err = abs(float(xq @ yq) - float(x @ y))
                bound = eps_e4m3(d) * np.linalg.norm(x) * np.linalg.norm(y)
                assert err <= bound * (1 + 1e-12), (d, kind, err, bound)
                worst = max(worst, err / bound if bound > 0 else 0.0)
    assert worst > 0.05   # the bound is not vacuous on these rows


def test_e4m3_scale_is_the_smallest_that_fits():
    for amax in (1e-30, 3.5, 448.0, 448.0000001, 1e30, 2.0 ** -100):
        x = np.array([amax, -amax / 3])
        s = row_scale(x)
        assert np.max(np.abs(x)) <= 448 * s and np.max(np.abs(x)) > 448 * s / 2


def bf16(v32):
    """Round float32 values to BF16 (nearest, ties to even), as float32."""
    b = np.asarray(v32, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_bf16_row_error_bound_holds():
    for d in (1, 33, 128, 256):
        for _ in range(200):
            scale = 10.0 ** RNG.integers(-6, 6)
            x = (RNG.standard_normal(d) * scale).astype(np.float32)
            m = (RNG.standard_normal(d) * scale).astype(np.float32)
            xc = (x - m).astype(np.float32)                   # fl(x - m)
            h = bf16(xc)
            exact = x.astype(np.float64) - m.astype(np.float64)
            rnd = np.sqrt(np.sum((h.astype(np.float64) - xc) ** 2)) * (1 + 2.0 ** -12)
            nrm = np.sqrt(np.sum(xc.astype(np.float64) ** 2)) * (1 + 2.0 ** -12)
            eb = rnd + nrm * 2.0 ** -22 + 1e-30
            assert np.linalg.norm(h.astype(np.float64) - exact) <= eb
            # and it is tight to within the BF16 rounding itself
            assert eb <= np.linalg.norm(h.astype(np.float64) - exact) * 1.01 + nrm * 2.0 ** -21 + 1e-29
