"""Bulk statistics of a sphere packing: packing fraction and mean coordination number.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): these measure the outputs of a
run, the oracle's and the CUDA library's alike, and are never called by the library.

The paper judges its long runs by bulk quantities of the granular bed (Sec. 5); the two
used here are
  * the packing fraction of a window: the volume of the spheres inside the window (each
    sphere clipped exactly to it) over the window's volume;
  * the mean coordination number: over the spheres centred in the window, the mean number
    of sphere-sphere contacts (overlap > 0; walls excluded).

The clipped volume of a sphere is the integral over z of the area of its horizontal disc
slice inside the window's rectangle.  That area has a closed form (``disc_rect_area``);
the z integral is done by quadrature in the polar angle, on panels split at every angle
where the slice's radius meets an edge or a corner distance of the rectangle, with nodes
clustered at the panel ends (where the area has fractional-power kinks), so the result is
exact to about 1e-13 relative.
"""
from __future__ import annotations

import math

import numpy as np


def _clustered_rule(n, m):
    """Gauss-Legendre nodes in u on [-1, 1] mapped by x(u) = c * int_0^u (1 - v^2)^m dv
    (c so that x(1) = 1): the weights carry dx/du = c (1 - u^2)^m, which vanishes to
    order m at both ends, so an integrand with a fractional-power kink at a panel end
    (a circular segment's area grows like (rho - d)^(3/2)) becomes smooth in u."""
    u, wu = np.polynomial.legendre.leggauss(n)
    poly = np.polynomial.polynomial
    p = poly.polypow([1.0, 0.0, -1.0], m)           # (1 - v^2)^m
    P = poly.polyint(p)                             # antiderivative, P(0) = 0
    c = 1.0 / poly.polyval(1.0, P)
    return c * poly.polyval(u, P), wu * c * poly.polyval(u, p)


_GL_X, _GL_W = _clustered_rule(40, 4)


def _prim(x, r):
    """Antiderivative of sqrt(r^2 - x^2) on [-r, r]."""
    x = min(max(x, -r), r)
    return 0.5 * (x * math.sqrt(max(r * r - x * x, 0.0)) + r * r * math.asin(x / r))


def _int_s(a, b, r):
    """Integral of sqrt(r^2 - x^2) over [a, b] intersected with [-r, r]."""
    lo, hi = max(a, -r), min(b, r)
    return _prim(hi, r) - _prim(lo, r) if hi > lo else 0.0


def _quadrant(a, b, r):
    """Area of the disc x^2 + y^2 <= r^2 with x <= a and y <= b."""
    if r <= 0.0 or a <= -r or b <= -r:
        return 0.0
    a = min(a, r)
    if b >= r:
        return 2.0 * _int_s(-r, a, r)
    xb = math.sqrt(r * r - b * b)     # |x| <= xb: the line y = b cuts the disc
    lo, hi = -xb, min(xb, a)
    inner = hi - lo if hi > lo else 0.0
    if b >= 0.0:
        # 2 s(x) everywhere, less (s(x) - b) where the line cuts
        return 2.0 * _int_s(-r, a, r) - (_int_s(lo, hi, r) - b * inner)
    # b < 0: only |x| <= xb contributes, with s(x) + b
    return _int_s(lo, hi, r) + b * inner


def disc_rect_area(r, x0, x1, y0, y1):
    """Area of the disc of radius r about the origin inside [x0, x1] x [y0, y1]."""
    if r <= 0.0 or x1 <= x0 or y1 <= y0:
        return 0.0
    return (_quadrant(x1, y1, r) - _quadrant(x0, y1, r) - _quadrant(x1, y0, r) + _quadrant(x0, y0, r))


def sphere_box_volume(c, R, lo, hi):
    """Volume of the ball of radius R about c inside the box [lo, hi] (3-vectors)."""
    c = np.asarray(c, np.float64)
    lo = np.asarray(lo, np.float64) - c
    hi = np.asarray(hi, np.float64) - c
    if np.any(hi <= -R) or np.any(lo >= R):
        return 0.0
    if np.all(lo <= -R) and np.all(hi >= R):
        return 4.0 / 3.0 * math.pi * R ** 3
    # z = R sin(t): slice radius R cos(t), dz = R cos(t) dt
    t0 = -0.5 * math.pi if lo[2] <= -R else math.asin(lo[2] / R)
    t1 = 0.5 * math.pi if hi[2] >= R else math.asin(hi[2] / R)
    cuts = [t0, t1]
    dists = [abs(lo[0]), abs(hi[0]), abs(lo[1]), abs(hi[1])]
    dists += [math.hypot(x, y) for x in (lo[0], hi[0]) for y in (lo[1], hi[1])]
    for d in dists:
        if d < R:
            t = math.acos(d / R)
            cuts += [t, -t]
    cuts = sorted(t for t in cuts if t0 <= t <= t1)
    vol = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b <= a:
            continue
        half, mid = 0.5 * (b - a), 0.5 * (b + a)
        for xg, wg in zip(_GL_X, _GL_W):
            t = mid + half * xg
            rho = R * math.cos(t)
            vol += wg * half * disc_rect_area(rho, lo[0], hi[0], lo[1], hi[1]) * R * math.cos(t)
    return vol


def packing_fraction(centres, radii, lo, hi):
    """Sum of the spheres' volumes inside the window [lo, hi] over its volume."""
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    radii = np.asarray(radii, np.float64).reshape(-1)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    inside = np.all(centres - radii[:, None] >= lo, axis=1) & np.all(centres + radii[:, None] <= hi, axis=1)
    vol = float(np.sum(4.0 / 3.0 * math.pi * radii[inside] ** 3))
    touch = ~inside & np.all(centres + radii[:, None] > lo, axis=1) & np.all(centres - radii[:, None] < hi, axis=1)
    for k in np.nonzero(touch)[0]:
        vol += sphere_box_volume(centres[k], radii[k], lo, hi)
    return vol / float(np.prod(hi - lo))


def coordination(centres, contact_i, contact_j, lo, hi):
    """Mean number of sphere-sphere contacts of the spheres centred in [lo, hi].

    contact_i, contact_j: sphere ids of the touching pairs (each pair once; wall contacts,
    given with a negative j, are ignored).  Returns (mean, number of spheres counted)."""
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    ci = np.asarray(contact_i, np.int64)
    cj = np.asarray(contact_j, np.int64)
    keep = cj >= 0
    ci, cj = ci[keep], cj[keep]
    inwin = np.all((centres >= lo) & (centres <= hi), axis=1)
    deg = np.bincount(ci, minlength=len(centres)) + np.bincount(cj, minlength=len(centres))
    n = int(inwin.sum())
    return (float(deg[inwin].sum()) / n if n else 0.0), n
