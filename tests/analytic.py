"""Closed-form equilibrium shapes used by the physics tests (host only)."""
import math

from scipy.optimize import brentq


def lens_area(R, r, d):
    """Area of the intersection of two circles of radii R, r at centre distance d."""
    if d >= R + r:
        return 0.0
    if d <= abs(R - r):
        return math.pi * min(R, r) ** 2
    c1 = min(1.0, max(-1.0, (d * d + r * r - R * R) / (2 * d * r)))
    c2 = min(1.0, max(-1.0, (d * d + R * R - r * r) / (2 * d * R)))
    k = max(0.0, (-d + r + R) * (d + r - R) * (d - r + R) * (d + r + R))
    return r * r * math.acos(c1) + R * R * math.acos(c2) - 0.5 * math.sqrt(k)


def drop_on_circle(A, R, theta):
    """Circular-arc drop of area A (outside the solid) meeting a circle of radius R at
    contact angle theta: returns (r, d) with d^2 = R^2 + r^2 - 2 R r cos(theta);
    the apex height above the circle centre is d + r (Sec. III B)."""
    def f(r):
        d = math.sqrt(R * R + r * r - 2 * R * r * math.cos(theta))
        return math.pi * r * r - lens_area(R, r, d) - A
    r = brentq(f, 1e-3 * R, 1e3 * R)
    return r, math.sqrt(R * R + r * r - 2 * R * r * math.cos(theta))


def cap_on_plane(A, theta):
    """Circular cap of area A on a flat wall at contact angle theta:
    R_c = sqrt(2A / (2 theta - sin 2 theta)) (Sec. III A); centre at -R_c cos(theta)."""
    Rc = math.sqrt(2 * A / (2 * theta - math.sin(2 * theta)))
    return Rc, -Rc * math.cos(theta)
