"""Seeded synthetic inputs: solid masks, ghost lists with analytic normals,
initial color fields and random states.

This module holds geometry and random numbers only -- none of the lattice
Boltzmann arithmetic.  Both the CUDA library's tests and the FP64 oracle's
tests draw their inputs from here, so a geometry handed to the two sides is
the same array.

Conventions (shared by the C ABI):
  * node index = x + nx*(y + ny*z); arrays have numpy shape (nz, ny, nx)
  * a node is solid iff |x - c|^2 <= R^2 with integer node coordinates
  * a ghost node is a solid node with at least one fluid neighbour in the
    lattice stencil (D2Q9: 8 neighbours, D3Q19: 18 neighbours) -- the solid
    boundary nodes of Sec. I of the paper
  * ghost normals are the analytic unit normals out of the solid (Sec. III)
"""
import math

import numpy as np

# neighbour offsets of the lattice stencils (order irrelevant here)
_OFF2 = [(dx, dy, 0) for dx in (-1, 0, 1) for dy in (-1, 0, 1) if (dx, dy) != (0, 0)]
_OFF3 = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
         if 0 < abs(dx) + abs(dy) + abs(dz) <= 2]


def offsets(lattice):
    return _OFF2 if lattice == 9 else _OFF3


def node_coords(shape):
    """(z, y, x) integer coordinate grids for a (nz, ny, nx) shape."""
    return np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")


def ghost_mask(solid, lattice):
    """Solid nodes with a fluid stencil neighbour (periodic wrap)."""
    solid = solid.astype(bool)
    fluid = ~solid
    has_fluid_nb = np.zeros_like(solid)
    for dx, dy, dz in offsets(lattice):
        has_fluid_nb |= np.roll(fluid, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    return solid & has_fluid_nb


def ghost_list(solid, lattice, normal_fn):
    """(nodes int64[n], normals float64[n,3]) for every ghost node; normal_fn maps
    (x, y, z) float arrays to unit normals of shape (n, 3)."""
    g = ghost_mask(solid, lattice)
    z, y, x = np.nonzero(g)
    nz, ny, nx = solid.shape
    nodes = (x + nx * (y + ny * z)).astype(np.int64)
    order = np.argsort(nodes)
    nodes, x, y, z = nodes[order], x[order], y[order], z[order]
    n = normal_fn(x.astype(float), y.astype(float), z.astype(float))
    n = np.asarray(n, dtype=np.float64).reshape(-1, 3)
    return nodes, n


def _radial_normals(center, dims):
    def fn(x, y, z):
        r = np.stack([x - center[0], y - center[1], (z - center[2]) if dims == 3 else 0 * z], axis=1)
        norm = np.linalg.norm(r, axis=1, keepdims=True)
        norm[norm == 0] = 1.0
        return r / norm
    return fn


def _plane_normals(normal):
    n = np.asarray(normal, dtype=float)
    n = n / np.linalg.norm(n)

    def fn(x, y, z):
        return np.tile(n, (len(x), 1))
    return fn


def sphere_domain(lattice, shape, center, R):
    """Solid circle (D2Q9, shape (1, ny, nx)) or sphere (D3Q19) of radius R."""
    z, y, x = node_coords(shape)
    d2 = (x - center[0]) ** 2 + (y - center[1]) ** 2
    if lattice == 19:
        d2 = d2 + (z - center[2]) ** 2
    solid = (d2 <= R * R).astype(np.uint8)
    return solid, ghost_list(solid, lattice, _radial_normals(center, 2 if lattice == 9 else 3))


def multi_sphere_domain(lattice, shape, centers, radii):
    """Several solid spheres; each ghost takes the normal of the sphere whose
    surface is nearest to it."""
    z, y, x = node_coords(shape)
    nz, ny, nx = shape
    solid = np.zeros(shape, dtype=bool)
    dims = np.array([nx, ny, nz], dtype=float)
    for c, R in zip(centers, radii):
        d2 = np.zeros(shape)
        for a, q in enumerate((x, y, z)[: 2 if lattice == 9 else 3]):
            d = q - c[a]
            d = d - dims[a] * np.round(d / dims[a])
            d2 += d * d
        solid |= d2 <= R * R
    centers = np.asarray(centers, dtype=float)
    radii = np.asarray(radii, dtype=float)

    def fn(xg, yg, zg):
        pts = np.stack([xg, yg, zg], axis=1)
        best = np.full(len(xg), np.inf)
        out = np.zeros((len(xg), 3))
        for c, R in zip(centers, radii):
            d = pts - c[None, :]
            if lattice == 9:
                d[:, 2] = 0
            d = d - dims[None, :] * np.round(d / dims[None, :])
            r = np.linalg.norm(d, axis=1)
            gap = np.abs(r - R)
            sel = gap < best
            rr = np.where(r == 0, 1.0, r)
            out[sel] = d[sel] / rr[sel, None]
            best = np.where(sel, gap, best)
        return out
    solid = solid.astype(np.uint8)
    return solid, ghost_list(solid, lattice, fn)


def wall_domain(lattice, shape, bottom=1, top=1):
    """Flat solid walls: `bottom` solid rows at low y and `top` at high y (D2Q9),
    or solid layers at low/high z (D3Q19).  Ghost normals point into the fluid."""
    solid = np.zeros(shape, dtype=np.uint8)
    axis = 1 if lattice == 9 else 0          # numpy axis of y (2D) or z (3D)
    n_ax = shape[axis]
    idx = [slice(None)] * 3
    for k in range(bottom):
        idx[axis] = k
        solid[tuple(idx)] = 1
    for k in range(top):
        idx[axis] = n_ax - 1 - k
        solid[tuple(idx)] = 1
    comp = 1 if lattice == 9 else 2
    mid = n_ax / 2.0

    def fn(x, y, z):
        coord = y if lattice == 9 else z
        out = np.zeros((len(x), 3))
        out[:, comp] = np.where(coord < mid, 1.0, -1.0)
        return out
    return solid, ghost_list(solid, lattice, fn)


def tilted_wall_domain(shape, normal, offset):
    """2D half-plane solid {n.x <= offset} with unit normal n pointing into the fluid."""
    z, y, x = node_coords(shape)
    n = np.asarray(normal, dtype=float)
    n = n / np.linalg.norm(n)
    solid = ((x * n[0] + y * n[1]) <= offset).astype(np.uint8)
    return solid, ghost_list(solid, 9, _plane_normals((n[0], n[1], 0.0)))


def tanh_field(signed_distance, W):
    """Equilibrium color profile of width W as a function of signed distance
    (positive inside the liquid), Sec. II."""
    return 0.5 * (1.0 + np.tanh(2.0 * signed_distance / W))


def droplet_on_sphere_center(sphere_center, R, R0, theta, axis=2):
    """Centre of a spherical cap of radius R0 meeting a sphere of radius R at
    contact angle theta, on the +axis pole: d^2 = R^2 + R0^2 - 2 R R0 cos(theta)."""
    d = math.sqrt(R * R + R0 * R0 - 2.0 * R * R0 * math.cos(theta))
    c = list(sphere_center)
    c[axis] += d
    return c


# ---------------------------------------------------------------- named workloads

def cylinder_config(nx=64, ny=64, R=12.0, R0=10.0, theta_deg=60.0):
    """D2Q9 drop on a circular cylinder: cylinder R=12 at the box centre of a
    64x64 periodic box, drop R0=10 tangent on its top, theta=60 deg, density
    and viscosity ratio 1, sigma=0.01, tau=1, FP64."""
    center = (nx / 2.0, ny / 2.0, 0.0)
    solid, ghosts = sphere_domain(9, (1, ny, nx), center, R)
    nu = 1.0 / 6.0                                   # tau = 1/2 + 3 nu = 1
    params = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=7, rho_l=1.0, rho_g=1.0, mu_l=nu, mu_g=nu,
                  sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(theta_deg), g=(0, 0, 0))
    drop = (center[0], center[1] + R + R0, 0.0)
    return dict(params=params, solid=solid, ghosts=ghosts, drop_center=drop, R0=R0,
                solid_center=center, R=R)


def sphere_config(n=192, R=32.0, R0=24.0, theta_deg=60.0, rho_ratio=1000.0, mu_ratio=100.0,
                  sigma=0.005, precision=1):
    """D3Q19 drop on a sphere: sphere R=32 at the centre of an n^3 periodic box,
    drop R0=24 on its +z pole placed at the prescribed contact angle,
    rho_g=1, mu_g=0.1, rho_l/rho_g=1000, mu_l/mu_g=100, sigma=0.005."""
    center = (n / 2.0, n / 2.0, n / 2.0)
    solid, ghosts = sphere_domain(19, (n, n, n), center, R)
    rho_g, mu_g = 1.0, 0.1
    params = dict(lattice=19, nx=n, ny=n, nz=n, periodic=7, rho_l=rho_g * rho_ratio, rho_g=rho_g,
                  mu_l=mu_g * mu_ratio, mu_g=mu_g, sigma=sigma, W=4.0, M_phi=0.02,
                  theta=math.radians(theta_deg), g=(0, 0, 0), precision=precision)
    drop = droplet_on_sphere_center(center, R, R0, math.radians(theta_deg))
    return dict(params=params, solid=solid, ghosts=ghosts, drop_center=tuple(drop), R0=R0,
                solid_center=center, R=R)


def random_state(Q, nn, fluid, seed, base=None, amp=1e-3):
    """Seeded random populations for one-step checks: N = base + amp*U(-1,1),
    B = phi N with phi ~ U(0,1) smoothed; zero at solid nodes.  base defaults
    to a uniform 1/Q (no lattice arithmetic)."""
    rng = np.random.default_rng(seed)
    if base is None:
        base = np.full(Q, 1.0 / Q)
    N = base[:, None] + amp * rng.uniform(-1, 1, size=(Q, nn))
    phi = rng.uniform(0, 1, size=nn)
    B = N * phi[None, :] * (1.0 + 0.01 * rng.uniform(-1, 1, size=(Q, nn)))
    N[:, ~fluid] = 0
    B[:, ~fluid] = 0
    u = 1e-3 * rng.uniform(-1, 1, size=(3, nn))
    u[:, ~fluid] = 0
    p = 1e-4 * rng.uniform(-1, 1, size=nn)
    p[~fluid] = 0
    return N, B, u, p


# ---------------------------------------------------------------- porous medium

def sphere_packing(n=256, r_min=8.0, r_max=16.0, porosity=0.45, reservoir=24, seed=1, max_iter=4000,
                   tol=0.02):
    """Seeded non-overlapping polydisperse sphere packing in a periodic n^3 box.

    Radii ~ U(r_min, r_max); sphere count from the target solid fraction
    (1 - porosity) of the region x >= reservoir (x < reservoir stays free, the
    inlet reservoir).  Random sequential placement jams well below a 0.55 solid
    fraction, so the spheres are placed at random and then pushed apart pair by
    pair (periodic in y, z; confined to the region in x) until no two overlap by
    more than tol.  Returns (centers [m,3], radii [m])."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    L = float(n)
    span = L - reservoir
    vol = span * L * L * (1.0 - porosity)
    mean_r3 = (r_max ** 4 - r_min ** 4) / (4.0 * (r_max - r_min))
    m = int(round(vol / (4.0 / 3.0 * math.pi * mean_r3)))
    radii = rng.uniform(r_min, r_max, m)
    c = np.stack([reservoir + radii + rng.uniform(0, 1, m) * (span - 2 * radii),
                  rng.uniform(0, L, m), rng.uniform(0, L, m)], axis=1)
    box = np.array([4.0 * L, L, L])          # x never wraps: the big box length disables x periodicity
    for _ in range(max_iter):
        tree = cKDTree(c, boxsize=box)
        pairs = tree.query_pairs(2.0 * r_max, output_type="ndarray")
        if len(pairs) == 0:
            break
        i, j = pairs[:, 0], pairs[:, 1]
        d = c[j] - c[i]
        d[:, 1:] -= L * np.round(d[:, 1:] / L)
        dist = np.linalg.norm(d, axis=1)
        ov = radii[i] + radii[j] - dist
        sel = ov > 0
        if not sel.any() or ov.max() <= tol:
            break
        i, j, d, dist, ov = i[sel], j[sel], d[sel], dist[sel], ov[sel]
        u = d / np.maximum(dist, 1e-9)[:, None]
        push = 0.5 * (ov + tol)[:, None] * u
        delta = np.zeros_like(c)
        np.add.at(delta, i, -push)
        np.add.at(delta, j, push)
        c += delta
        c[:, 0] = np.clip(c[:, 0], reservoir + radii, L - radii)
        c[:, 1:] %= L
    return c, radii


def packing_domain(centers, radii, n=256):
    """Staircase mask (|x - c|^2 <= r^2 with periodic images in y, z) of a
    sphere packing and its D3Q19 ghost list; each ghost takes the normal of the
    sphere surface nearest to it."""
    from scipy.spatial import cKDTree
    shape = (n, n, n)
    solid = np.zeros(shape, dtype=bool)
    for (cx, cy, cz), r in zip(centers, radii):
        lo = np.floor(np.array([cx, cy, cz]) - r).astype(int)
        hi = np.ceil(np.array([cx, cy, cz]) + r).astype(int)
        xs = np.arange(lo[0], hi[0] + 1)
        ys = np.arange(lo[1], hi[1] + 1)
        zs = np.arange(lo[2], hi[2] + 1)
        dz, dy, dx = np.meshgrid(zs - cz, ys - cy, xs - cx, indexing="ij")
        inside = dx * dx + dy * dy + dz * dz <= r * r
        zi, yi, xi = np.meshgrid(zs % n, ys % n, xs % n, indexing="ij")
        solid[zi[inside], yi[inside], xi[inside]] = True
    solid = solid.astype(np.uint8)
    tree = cKDTree(centers, boxsize=np.array([4.0 * n, n, n]))
    radii = np.asarray(radii)

    def fn(x, y, z):
        pts = np.stack([x, y, z], axis=1)
        k = min(8, len(radii))
        _, idx = tree.query(pts, k=k, workers=-1)       # each point's answer is independent of the split
        idx = idx.reshape(len(pts), k)
        best = np.full(len(pts), np.inf)
        out = np.zeros((len(pts), 3))
        for col in range(k):
            cid = idx[:, col]
            d = pts - centers[cid]
            d[:, 1:] -= n * np.round(d[:, 1:] / n)
            r = np.linalg.norm(d, axis=1)
            gap = np.abs(r - radii[cid])
            sel = gap < best
            rr = np.where(r == 0, 1.0, r)
            out[sel] = d[sel] / rr[sel, None]
            best = np.where(sel, gap, best)
        return out
    return solid, ghost_list(solid, 19, fn)
