"""CPU pin of the E4M3 rounding bound used by the 8-bit layer test.

E4M3 (sign, 4 exponent bits with bias 7, 3 mantissa bits, no infinities; the
all-ones exponent with mantissa 111 is NaN): normal values 2^(e-7) (1 + m/8)
for e = 1..15 (e = 15 only up to mantissa 110, i.e. 448), subnormals
2^-6 (m / 8).  Rounding to nearest (ties to even) with saturation at 448, the
error of v is at most 2^-4 |v| for 2^-6 <= |v| <= 448 and at most half the
subnormal spacing 2^-9 below: |dv| <= 2^-4 |v| + 2^-10 covers both, which
is the per-operand bound of tests/test_gpu_e4m3.py (in units of the scale).
The grid here is built from that definition alone.
"""
import numpy as np


def e4m3_values():
    vals = [0.0]
    for m in range(1, 8):                       # subnormals
        vals.append(2.0 ** -6 * m / 8)
    for e in range(1, 16):
        for m in range(8):
            if e == 15 and m == 7:              # NaN encoding
                continue
            vals.append(2.0 ** (e - 7) * (1 + m / 8))
    v = np.array(sorted(set(vals)))
    return np.concatenate([-v[:0:-1], v])


def round_e4m3(x, grid):
    """Nearest grid value, ties to the one with an even mantissa (even index
    among the positive values), saturating at +-448."""
    x = np.clip(x, grid[0], grid[-1])
    i = np.searchsorted(grid, x)
    i = np.clip(i, 1, len(grid) - 1)
    lo, hi = grid[i - 1], grid[i]
    dlo, dhi = x - lo, hi - x
    pick_hi = dhi < dlo
    tie = dhi == dlo
    # even mantissa <=> even position in the magnitude-ordered list of positive codes
    pos = np.searchsorted(grid[grid >= 0], np.abs(hi))
    pick_hi = np.where(tie, pos % 2 == 0, pick_hi)
    return np.where(pick_hi, hi, lo)


def test_e4m3_grid_matches_the_format():
    g = e4m3_values()
    pos = g[g > 0]
    assert pos.max() == 448.0
    assert pos.min() == 2.0 ** -9                        # smallest subnormal
    assert len(pos) == 7 + 15 * 8 - 1                    # 126 positive finite values
    sub = pos[pos < 2.0 ** -6]
    assert np.allclose(np.diff(sub), 2.0 ** -9)          # subnormal spacing


def test_e4m3_rounding_error_bound():
    g = e4m3_values()
    rng = np.random.default_rng(5)
    # dense log-uniform magnitudes over the whole range, plus every midpoint and its neighbours
    x = np.concatenate([
        np.exp(rng.uniform(np.log(2.0 ** -14), np.log(448.0), 200000)) * rng.choice([-1, 1], 200000),
        (g[:-1] + g[1:]) / 2,
        np.nextafter((g[:-1] + g[1:]) / 2, np.inf),
        np.nextafter((g[:-1] + g[1:]) / 2, -np.inf),
    ])
    r = round_e4m3(x, g)
    err = np.abs(r - x)
    assert (err <= 2.0 ** -4 * np.abs(x) + 2.0 ** -10 + 1e-15).all()
    # the bound is tight: both terms are reached
    normal = np.abs(x) >= 2.0 ** -6
    assert (err[normal] / np.abs(x[normal])).max() > 0.9 * 2.0 ** -4
    assert err[~normal].max() > 0.99 * 2.0 ** -10
    # a scale of max|x| / 448 maps the largest magnitude onto the largest finite value
    v = rng.standard_normal(1000)
    s = np.abs(v).max() / 448.0
    assert np.abs(round_e4m3(v / s, g)).max() == 448.0
