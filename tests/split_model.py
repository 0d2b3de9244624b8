"""A CPU model of the split-BF16 arithmetic of the tensor-core path (tests
only): what the kernels compute, written with numpy on exact basis values,
to size the numerical choices (digit grids, number of products) against the
tolerances before they are built.

Leading digit x0 = rint(x / unit) * unit on a power-of-two grid per row
(H) or per point (density), the remainder split into two BF16 terms
(round to nearest even), products accumulated in FP32 per 16 contraction
steps (one MMA, the accumulator update truncated), x0 * y0 exact.  Not a test of the CUDA code: the parity
tests are.
"""
import numpy as np


def bf16(x):
    """Round FP32 values to BF16 (nearest even), returned as FP32."""
    x = np.asarray(x, np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def fixed_bits(depth):
    """Digit width b with depth * 2^(2b) <= 2^24 (at most 7)."""
    b = 7
    while b > 1 and (depth << (2 * b)) > (1 << 24):
        b -= 1
    return b


def grid_units(mx, sm, depth):
    """Grid unit per row: 2^(e - b) with 2^e >= mx (1 + 2^-12); b = 8 when
    the row sum allows it (sum / 2^e <= 200), else the depth rule.  sm=None
    means no sum is known (the depth rule alone)."""
    mx = np.asarray(mx, np.float64)
    unit = np.zeros_like(mx)
    ok = mx > 1e-30
    _, e = np.frexp(mx[ok] * (1 + 1 / 4096))
    if sm is None:
        bits = fixed_bits(depth)
    else:
        S = np.asarray(sm, np.float64)[ok] * np.exp2(-e.astype(np.float64)) * 1.001
        bits = np.where(S <= 200, 8, fixed_bits(depth))
    unit[ok] = np.exp2((e - bits).astype(np.float64))
    return unit


def split3(x, unit):
    """x0 (fixed digit), x1, x2 (BF16) of x (float64) on the given units."""
    xh = x.astype(np.float32)
    xl = (x - xh.astype(np.float64)).astype(np.float32)
    safe = np.where(unit > 0, unit, 1.0).astype(np.float32)
    x0 = np.where(unit > 0, np.rint(xh / safe) * unit, 0.0).astype(np.float32)
    d = (xh - x0).astype(np.float32)
    a, b = bf16(x0), bf16(d)
    c = bf16((d - b) + xl)
    return a.astype(np.float64), b.astype(np.float64), c.astype(np.float64)


def to_f32_rz(x):
    """Round float64 values to FP32 toward zero (the accumulator update of
    the tensor cores is modelled as truncating)."""
    y = np.asarray(x, np.float64).astype(np.float32)
    over = np.abs(y.astype(np.float64)) > np.abs(x)
    return np.where(over, np.nextafter(y, np.float32(0)), y)


def _fp32_steps(pairs, K, truncate=True):
    """Products accumulated in FP32 per 16 contraction steps (one MMA): the
    16-step partial sums exact, each added to the accumulator with one
    rounding (toward zero by default, to nearest with truncate=False)."""
    rnd = to_f32_rz if truncate else (lambda v: np.asarray(v).astype(np.float32))
    acc = None
    for k0 in range(0, K, 16):
        part = sum(a[:, k0:k0 + 16] @ b[k0:k0 + 16] for a, b in pairs)
        acc = rnd(part) if acc is None else rnd(acc.astype(np.float64) + part)
    return acc.astype(np.float64)


def h_block(psi, unit, n_products=8):
    """psi^T psi of one batch (psi: points x functions) with row grids `unit`
    per function: x0 y0 exact, the other products in FP32."""
    x0, x1, x2 = split3(psi, unit[None, :])
    pairs = [(x0.T, x1), (x1.T, x0), (x0.T, x2), (x1.T, x1), (x2.T, x0)]
    if n_products == 8:
        pairs += [(x1.T, x2), (x2.T, x1)]
    return x0.T @ x0 + _fp32_steps(pairs, psi.shape[0])


def density_e(D, dunit, Phi, punit, n_products=8):
    """E = D Phi (functions x points): D rows on `dunit`, Phi columns (points)
    on `punit`; the 8 products of combined order <= 3 except d2 p2 (as the
    kernels), or the 6 of order <= 2."""
    d0, d1, d2 = split3(D, dunit[:, None])
    p0, p1, p2 = split3(Phi, punit[None, :])
    pairs = [(d0, p1), (d1, p0), (d0, p2), (d1, p1), (d2, p0)]
    if n_products == 8:
        pairs += [(d1, p2), (d2, p1)]
    return d0 @ p0 + _fp32_steps(pairs, D.shape[1])


def table_lookup(tab, h, nk, d):
    """The kernels' lookup of a suffix-bound table at distances d: knot index
    floor(d (1 - 1e-6) / h) clamped to [0, nk - 2], zero beyond the cutoff."""
    ki = np.clip((d * 0.999999 / h).astype(np.int64), 0, nk - 2)
    return np.where(d < (nk - 1) * h * 1.00001, tab[ki], 0.0)
