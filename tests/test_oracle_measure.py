"""The oracle's contact-angle measurement (diagnostics with a circle, sphere or
plane probe) on color fields whose contact angle is known exactly: the
equilibrium tanh profile of a circle or sphere of radius r cut by the solid.
The expected angle comes from the geometry alone -- a contact point P found by
bisection on the drop circle, and the angle between the outward normals of the
drop and of the solid at P (cos theta = n_drop . n_solid: 180 deg for a drop
just touching the wall, 0 for one lying flat on it) -- not from the formula
the measurement uses.  The measurement takes each interface point's nearest
periodic image from the probe's centre, so every drop here lies within half
a box of it."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import workloads as wl

W = 4.0


def _params(lattice, shape):
    nz, ny, nx = shape
    return dict(lattice=lattice, nx=nx, ny=ny, nz=nz, periodic=7, rho_l=1.0, rho_g=1.0, mu_l=0.1, mu_g=0.1,
                sigma=0.01, W=W, M_phi=0.02, theta=math.radians(90.0), g=(0, 0, 0))


def _bisect(f, a, b, n=200):
    fa = f(a)
    for _ in range(n):
        m = 0.5 * (a + b)
        fm = f(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def _angle_on_circle(cs, R, cd, r):
    """Contact angle of a drop circle (cd, r) on a solid circle (cs, R), both in
    the plane through the symmetry axis: P on the drop circle where the
    distance to cs equals R, then the angle between the outward normals."""
    cs, cd = np.asarray(cs, float), np.asarray(cd, float)
    axis = (cd - cs) / np.linalg.norm(cd - cs)
    side = np.array([-axis[1], axis[0]])
    point = lambda t: cd + r * (math.cos(t) * side + math.sin(t) * axis)      # noqa: E731
    # t = -pi/2 points from the drop centre toward the solid centre
    t = _bisect(lambda t: np.linalg.norm(point(t) - cs) - R, -math.pi / 2, math.pi / 2)
    P = point(t)
    n_d, n_s = (P - cd) / r, (P - cs) / R
    return math.degrees(math.acos(float(np.clip(n_d @ n_s, -1, 1))))


@pytest.mark.parametrize("d_over_R", [1.2, 1.45, 1.75])
def test_circle_probe_on_an_exact_cap(d_over_R):
    shape = (1, 112, 112)
    R, r = 18.0, 22.0
    cs = (56.0, 40.0)
    cd = (56.0, 40.0 + d_over_R * R)
    solid, ghosts = wl.sphere_domain(9, shape, (cs[0], cs[1], 0.0), R)
    z, y, x = wl.node_coords(shape)
    phi = wl.tanh_field(r - np.hypot(x - cd[0], y - cd[1]), W).reshape(-1)
    o = oracle.Oracle(_params(9, shape), solid, ghosts)
    o.init_phi(phi)
    d = o.diagnostics(oracle.make_probe(1, (cs[0], cs[1], 0.0), R, (0, 1, 0), 1.5 * W))
    want = _angle_on_circle(cs, R, cd, r)
    got = math.degrees(d["contact_angle"])
    print("circle cap: d/R %.2f  exact %.4f deg  measured %.4f deg  fit r %.4f (%.1f)  points %d"
          % (d_over_R, want, got, d["fit_radius"], r, d["n_fit"]))
    assert abs(got - want) < 0.1
    assert abs(d["fit_radius"] / r - 1) < 2e-3


def test_sphere_probe_on_an_exact_cap():
    shape = (80, 64, 64)                 # the cap reaches 32.8 above the sphere centre
    R, r = 12.0, 16.0
    cs = (32.0, 32.0, 20.0)
    cd = (32.0, 32.0, 20.0 + 1.4 * R)
    solid, ghosts = wl.sphere_domain(19, shape, cs, R)
    z, y, x = wl.node_coords(shape)
    dist = np.sqrt((x - cd[0]) ** 2 + (y - cd[1]) ** 2 + (z - cd[2]) ** 2)
    phi = wl.tanh_field(r - dist, W).reshape(-1)
    o = oracle.Oracle(_params(19, shape), solid, ghosts)
    o.init_phi(phi)
    d = o.diagnostics(oracle.make_probe(1, cs, R, (0, 0, 1), 1.5 * W))
    # the cross-section through the axis is the 2D configuration
    want = _angle_on_circle((cs[0], cs[2]), R, (cd[0], cd[2]), r)
    got = math.degrees(d["contact_angle"])
    print("sphere cap: exact %.4f deg  measured %.4f deg  fit r %.4f (%.1f)  points %d"
          % (want, got, d["fit_radius"], r, d["n_fit"]))
    assert abs(got - want) < 0.1
    assert abs(d["fit_radius"] / r - 1) < 2e-3


@pytest.mark.parametrize("h", [-8.0, 0.0, 9.0])
def test_plane_probe_on_an_exact_cap(h):
    """A drop circle whose centre lies h above a flat wall (bottom solid rows
    0..b-1, halfway bounce-back puts the surface at y = b - 1/2)."""
    shape = (1, 96, 128)
    b, r = 3, 24.0
    solid, ghosts = wl.wall_domain(9, shape, bottom=b, top=1)
    wall = b - 0.5
    cd = (64.0, wall + h)
    z, y, x = wl.node_coords(shape)
    phi = wl.tanh_field(r - np.hypot(x - cd[0], y - cd[1]), W).reshape(-1)
    o = oracle.Oracle(_params(9, shape), solid, ghosts)
    o.init_phi(phi)
    d = o.diagnostics(oracle.make_probe(2, (cd[0], wall, 0.0), 0.0, (0, 1, 0), 1.5 * W))
    # contact point where the circle meets y = wall, normals at it
    P = np.array([cd[0] + math.sqrt(r * r - h * h), wall])
    n_d, n_s = (P - np.asarray(cd)) / r, np.array([0.0, 1.0])
    want = math.degrees(math.acos(float(n_d @ n_s)))
    got = math.degrees(d["contact_angle"])
    print("plane cap: h %.1f  exact %.4f deg  measured %.4f deg  fit r %.4f (%.1f)  points %d"
          % (h, want, got, d["fit_radius"], r, d["n_fit"]))
    assert abs(got - want) < 0.1
