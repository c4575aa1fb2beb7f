"""Writes rounding_cases.txt and knn_rounding_cases.txt: kernel-test and kNN-order cases
whose outcome depends on how the binary32 distance is evaluated.

Section 3.2 defines the kernels with a strict "<"; the reading taken everywhere in this
library evaluates d = p - c per axis, then ((dx*dx + dy*dy) + dz*dz) < r*r for the
sphere (circle: dx*dx + dy*dy < r*r) and max(|d|) < r for the cube and square, every
operation a binary32 operation rounded to nearest-even, nothing fused.  Section 3.3 orders
kNN candidates by that squared distance, ties by the smaller index.

Every decision written here is taken by exact rational arithmetic (fractions.Fraction)
with explicit round-to-nearest-even to binary32 (or binary64) after each operation, so no
floating-point unit, compiler or oracle code is involved.  Beside the reading's decision
each row records what plausible mistakes would decide: a different summation order, a
fused multiply-add, and (for the boundary report) the binary64 evaluation.  Rows are
kept only where at least one of those differs from the reading, so a test that matches
the reading's column on every row fails for each of the mistakes.

Run from the repository root:  python tests/golden/make_rounding_cases.py
"""
import os
import random
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def rnd(x, p, emin):
    """Round the rational x to the nearest binary float with p significand bits and
    minimum normal exponent emin, ties to even (subnormals included, no overflow)."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, emin)
    ulp = Fraction(2) ** (e - (p - 1))
    q = a / ulp
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return s * n * ulp


def r32(x):
    return rnd(x, 24, -126)


def r64(x):
    return rnd(x, 53, -1022)


def f32_hex(v):
    """Exact hexadecimal of a binary32 value held as a Fraction."""
    assert r32(v) == v
    return float(v).hex()


def to32(x):
    """The binary32 value nearest to the Python float x, as a Fraction."""
    return r32(Fraction(x))


# ----------------------------------------------------------------------------- decisions
def sphere_decisions(p, c, r):
    d = [r32(p[a] - c[a]) for a in range(3)]
    xx, yy, zz = (r32(v * v) for v in d)
    r2 = r32(r * r)
    out = {
        "inside": r32(r32(xx + yy) + zz) < r2,                 # the reading
        "o2": r32(xx + r32(yy + zz)) < r2,                     # x + (y + z)
        "o3": r32(r32(xx + zz) + yy) < r2,                     # (x + z) + y
        "fma1": r32(r32(xx + yy) + d[2] * d[2]) < r2,          # fma(dz, dz, xx + yy)
        "fma2": r32(r32(xx + d[1] * d[1]) + d[2] * d[2]) < r2,  # fma(dz, dz, fma(dy, dy, xx))
    }
    e = [r64(p[a] - c[a]) for a in range(3)]
    out["f64"] = r64(r64(r64(e[0] * e[0]) + r64(e[1] * e[1])) + r64(e[2] * e[2])) < r64(r * r)
    return out


def circle_decisions(p, c, r):
    d = [r32(p[a] - c[a]) for a in range(2)]
    xx, yy = (r32(v * v) for v in d)
    r2 = r32(r * r)
    out = {
        "inside": r32(xx + yy) < r2,
        "o2": None, "o3": None,
        "fma1": r32(xx + d[1] * d[1]) < r2,                    # fma(dy, dy, xx)
        "fma2": r32(d[0] * d[0] + yy) < r2,                    # fma(dx, dx, yy)
    }
    e = [r64(p[a] - c[a]) for a in range(2)]
    out["f64"] = r64(r64(e[0] * e[0]) + r64(e[1] * e[1])) < r64(r * r)
    return out


def maxnorm_decisions(p, c, r, axes):
    d = [abs(r32(p[a] - c[a])) for a in range(axes)]
    e = [abs(r64(p[a] - c[a])) for a in range(axes)]
    return {"inside": max(d) < r, "o2": None, "o3": None, "fma1": None, "fma2": None, "f64": max(e) < r}


DECIDE = {
    "sphere": sphere_decisions,
    "circle": circle_decisions,
    "cube": lambda p, c, r: maxnorm_decisions(p, c, r, 3),
    "square": lambda p, c, r: maxnorm_decisions(p, c, r, 2),
}
ALTS = ("o2", "o3", "fma1", "fma2", "f64")


# ----------------------------------------------------------------------------- search
def candidates(rng, c, r, axes, grid):
    """Points p = c + off near the kernel's boundary, off on a grid of 2^grid (so that the
    subtraction is exact when grid is fine enough) or rounded when it is not."""
    while True:
        v = [rng.gauss(0.0, 1.0) for _ in range(3)]
        if axes == 2:
            v[2] = rng.uniform(-3.0, 3.0) * float(r)
        nrm = sum(x * x for x in v[:axes]) ** 0.5
        if nrm == 0.0:
            continue
        if rng.random() < 0.5:                                  # sphere-like boundary
            s = float(r) / nrm * (1.0 + rng.uniform(-3e-7, 3e-7))
            off = [x * s for x in v[:axes]] + v[axes:]
        else:                                                   # max-norm boundary
            m = max(abs(x) for x in v[:axes])
            s = float(r) / m * (1.0 + rng.uniform(-3e-7, 3e-7))
            off = [x * s for x in v[:axes]] + v[axes:]
        if grid is not None:
            off = [round(x * 2.0 ** grid) / 2.0 ** grid for x in off]
        p = [to32(float(c[a]) + off[a]) for a in range(3)]
        yield p


def find_kernel_cases(rng, kern, c, r, axes, grid, want):
    """Rows where each alternative of ALTS that exists for the kernel differs from the
    reading at least want[alt] times; each row once."""
    need = dict(want)
    rows = []
    seen = set()
    for n, p in enumerate(candidates(rng, c, r, axes, grid)):
        if n > 400000:
            raise RuntimeError("search did not find enough %s cases: %r" % (kern, need))
        dec = DECIDE[kern](p, c, r)
        hits = [a for a in ALTS if dec[a] is not None and dec[a] != dec["inside"] and need.get(a, 0) > 0]
        if not hits:
            continue
        key = tuple(p)
        if key in seen:
            continue
        seen.add(key)
        for a in hits:
            need[a] -= 1
        rows.append((p, dec))
        if all(v <= 0 for v in need.values()):
            break
    # a few plain rows on either side, where every evaluation agrees
    for p in candidates(rng, c, r * 1.001 if rng.random() < 0.5 else r * 0.999, axes, grid):
        dec = DECIDE[kern](p, c, r)
        if all(dec[a] is None or dec[a] == dec["inside"] for a in ALTS):
            rows.append((p, dec))
            if len(rows) >= len(seen) + 2:
                break
    return rows


def fmt(v):
    return "-" if v is None else str(int(v))


def write_kernel_cases(path):
    rng = random.Random(20260312)
    specs = [
        # kernel, centre, radius, axes, offset grid (2^-k), minimum rows per mistake
        ("sphere", (311.7, 905.3, 17.2), 2.0, 3, 17, dict(o2=3, o3=3, fma1=3, fma2=3, f64=4)),
        ("circle", (311.7, 905.3, 17.2), 2.0, 2, 17, dict(fma1=3, fma2=3, f64=4)),
        ("cube", (0.000371, -0.000213, 0.0000977), 700.0, 3, None, dict(f64=4)),
        ("square", (0.000371, -0.000213, 0.0000977), 700.0, 2, None, dict(f64=4)),
    ]
    lines = [
        "# Section 3.2 kernels at the rounding boundary (written by make_rounding_cases.py;",
        "# decided by exact rational arithmetic with round-to-nearest-even after every step).",
        "# Values are binary32 in hexadecimal.  Columns: kernel px py pz cx cy cz r, then the",
        "# reading's decision (d = p - c; ((dx*dx + dy*dy) + dz*dz) < r*r, or max|d| < r; every",
        "# operation binary32, nothing fused) and what these would decide instead:",
        "#   o2 = dx*dx + (dy*dy + dz*dz), o3 = (dx*dx + dz*dz) + dy*dy,",
        "#   fma1 = the last addition fused with its product, fma2 = both additions fused,",
        "#   f64 = the same expression in binary64 (the boundary report's other side).",
        "# '-' where a variant does not exist for the kernel.",
        "# kernel px py pz cx cy cz r inside o2 o3 fma1 fma2 f64",
    ]
    for kern, c0, r0, axes, grid, want in specs:
        c = [to32(v) for v in c0]
        r = to32(r0)
        for p, dec in find_kernel_cases(rng, kern, c, r, axes, grid, want):
            cols = [kern] + [f32_hex(v) for v in p] + [f32_hex(v) for v in c] + [f32_hex(r)]
            cols += [fmt(dec["inside"])] + [fmt(dec[a]) for a in ALTS]
            lines.append(" ".join(cols))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


# ----------------------------------------------------------------------------- kNN order
def sq_dists(p, c):
    d = [r32(p[a] - c[a]) for a in range(3)]
    xx, yy, zz = (r32(v * v) for v in d)
    return {
        "d2": r32(r32(xx + yy) + zz),
        "o2": r32(xx + r32(yy + zz)),
        "o3": r32(r32(xx + zz) + yy),
        "fma1": r32(r32(xx + yy) + d[2] * d[2]),
        "fma2": r32(r32(xx + d[1] * d[1]) + d[2] * d[2]),
    }


def order_of(d0, d1):
    """Section 3.3 order of the two points: by distance, ties to the smaller index."""
    return "01" if (d0 < d1 or d0 == d1) else "10"


def write_knn_cases(path):
    rng = random.Random(20260313)
    c = [to32(v) for v in (100.0, 200.0, 50.0)]
    grid = 2.0 ** 17                                   # ulp of 100..256: offsets add exactly
    need = {"o2": 2, "o3": 2, "fma1": 2, "fma2": 2}
    ties = 0
    rows = []
    tries = 0
    while any(v > 0 for v in need.values()) or ties < 2:
        tries += 1
        if tries > 500000:
            raise RuntimeError("kNN search did not converge: %r" % need)
        a, b, z = (round(rng.uniform(0.3, 1.7) * grid) / grid for _ in range(3))
        off0 = [a, b, z]
        off1 = [z, b, a] if rng.random() < 0.5 else [b, z, a]  # the same real distance
        p0 = [to32(float(c[i]) + off0[i]) for i in range(3)]
        p1 = [to32(float(c[i]) + off1[i]) for i in range(3)]
        s0, s1 = sq_dists(p0, c), sq_dists(p1, c)
        want = order_of(s0["d2"], s1["d2"])
        differ = [k for k in need if order_of(s0[k], s1[k]) != want]
        useful = [k for k in differ if need[k] > 0]
        tie = s0["d2"] == s1["d2"] and ties < 2 and differ
        if not useful and not tie:
            continue
        for k in useful:
            need[k] -= 1
        if tie:
            ties += 1
        rows.append((p0, p1, s0, s1, want))
    lines = [
        "# Section 3.3 order of two candidates whose binary32 squared distances (the reading:",
        "# ((dx*dx + dy*dy) + dz*dz), every operation binary32, nothing fused) tie or nearly",
        "# tie; written by make_rounding_cases.py with exact rational arithmetic.  Point 0 is",
        "# the first of the cloud, point 1 the second; the order puts the smaller distance",
        "# first, a tie to point 0.  Columns: cx cy cz  p0x p0y p0z  p1x p1y p1z  order d2_0 d2_1",
        "# then the order the variants would give: o2 o3 fma1 fma2 (see rounding_cases.txt).",
    ]
    for p0, p1, s0, s1, want in rows:
        cols = [f32_hex(v) for v in c] + [f32_hex(v) for v in p0] + [f32_hex(v) for v in p1]
        cols += [want, f32_hex(s0["d2"]), f32_hex(s1["d2"])]
        cols += [order_of(s0[k], s1[k]) for k in ("o2", "o3", "fma1", "fma2")]
        lines.append(" ".join(cols))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    write_kernel_cases(os.path.join(HERE, "rounding_cases.txt"))
    write_knn_cases(os.path.join(HERE, "knn_rounding_cases.txt"))
