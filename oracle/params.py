"""PSWF bandlimit c from the tolerance eps (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Table 2 (Sec. 7) lists 3c/pi for the prolate split at eps = 1e-3, 1e-6, 1e-9,
1e-12.  The paper selects parameters for other eps by a regression whose
coefficients it does not print.  Reading used here: interpolate 3c/pi linearly
in log10(eps) between the table rows and round up to an integer; when both the
Stokeslet and the stresslet are requested, take the larger c.
"""
import math

TABLE2_3C_OVER_PI = {
    "stokeslet": {-3: 10, -6: 17, -9: 25, -12: 31},
    "stresslet": {-3: 9, -6: 17, -9: 25, -12: 32},
}


def three_c_over_pi(eps, kernel="stokeslet"):
    rows = TABLE2_3C_OVER_PI[kernel]
    e = math.log10(eps)
    if not (-12.0 - 1e-9 <= e <= -3.0 + 1e-9):
        raise ValueError("eps outside Table 2 range [1e-12, 1e-3]")
    keys = sorted(rows)                  # [-12, -9, -6, -3]
    for lo, hi in zip(keys[:-1], keys[1:]):
        if lo - 1e-9 <= e <= hi + 1e-9:
            t = (e - lo) / (hi - lo)
            v = rows[lo] + t * (rows[hi] - rows[lo])
            return int(math.ceil(v - 1e-9))
    raise AssertionError


def bandlimit_c(eps, stokeslet=True, stresslet=False):
    v = 0
    if stokeslet:
        v = max(v, three_c_over_pi(eps, "stokeslet"))
    if stresslet:
        v = max(v, three_c_over_pi(eps, "stresslet"))
    return v * math.pi / 3.0
