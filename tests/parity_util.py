"""Comparison of a GPU state with the FP64 oracle's, shared by the GPU parity tests.

Populations N, B and the color phi are compared by their relative L-infinity
error over fluid nodes, max|gpu - oracle| / max|oracle|, against the bound of
the precision: 1e-12 (FP64), 1e-4 (FP32), 2e-3 (FP16 population storage).

u and p are compared on their own scale.  Both are small results of sums of
much larger terms, so a relative bound alone would demand more than the
arithmetic can give; each gets the same relative bound plus the rounding
budget of the sums that produce it:

    |u_gpu - u_oracle| <= tol * max|u_oracle| + E_u,
    |p_gpu - p_oracle| <= tol * max|p_oracle| + E_p,

with E from the step's arithmetic (Eqs. velUpdate, pressureUpdate,
surfaceTensionForce, pressCorrection, viscCorrection), per step taken:

    u = sum_i N_i c_i + F / (2 rho)            (Eq. velUpdate)
    p = (sum_{i>0} N_i / 3 - ...) / (1 - w_0)   (Eq. pressureUpdate)

  * the population sums round at the unit roundoff u_r of the arithmetic
    (2^-53 in FP64, 2^-24 in float) times S_N = max_x sum_i |N_i - b_i|, where
    b_i is what the storage subtracts (0 in FP64, chi_i in the float modes,
    which compute on deviations from the rest state);
  * the force is a sum of terms far larger than itself at equilibrium:
    S_F = sigma (48/W |phi(1-phi)(phi-1/2)| + 3W/2 |lap phi|) |grad phi|
    + drho |grad phi| (|p| + 2 nu_max |grad u|) + rho_l |g|;
  * E_u = 8 u_r (S_N + S_F / (2 rho_g)), E_p = 8 u_r S_N / (3 (1 - w_0)) +
    2 w_0 / (1 - w_0) max|u| E_u, the factor 8 covering the operations of
    each sum; n steps from the same start add n such budgets;
  * every step also reads a color the GPU holds in its own precision (the
    initial or written color included; the oracle keeps it in double): half a
    unit roundoff per node, which the Laplacian stencil gains by 12 (1 - w_0)
    and the surface tension carries into u as
    2 u_r sigma 3W/2 12 (1 - w_0) |grad phi| / (2 rho_g) (twice the stencil
    bound, for the rounding of the rest of the chemical potential there);
    steps add linearly (the worst case: the velocity integrates the force),
    and the pressure, which integrates the velocity's divergence
    (dp/dt = -c_s^2 div u), gathers D/3 du n (n - 1)/2 of it;
  * FP16 population storage also rounds every stored moving value to 11
    significant bits, the initial or written state included (chi itself is
    not on the FP16 grid): 2^-12 max|N - chi| per N value and
    2^-12 max|B - chi/2| per B value, which enter u directly (Q - 1 N values)
    and through phi (Q - 1 B values) and the force's Laplacian.

A term, a sign or a factor of 2 wrong in the float force or moments of the
GPU step moves u or p by a fraction of their own size, far above E.
"""
import numpy as np

import oracle

TOL = {0: 1e-12, 1: 1e-4, 2: 2e-3}          # FP64, FP32, FP16 population storage
U_R = {0: 2.0 ** -53, 1: 2.0 ** -24, 2: 2.0 ** -24}


def rel(a, b, mask=None):
    """max|a - b| / max|b| over the masked entries (last axis)."""
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def _stencil(Q):
    t = oracle.lattice_tables(Q)
    return t["c"], t["w"]


def _grad_lap(f, c, w, shape):
    """Isotropic lattice gradient 3 sum w_i c_i f(x + c_i) and Laplacian
    6 sum w_i (f(x + c_i) - f(x)) of a field on the periodic grid (nz, ny, nx)."""
    f = f.reshape(shape)
    g = np.zeros((3,) + shape)
    lap = np.zeros(shape)
    for ci, wi in zip(c, w):
        if not ci.any():
            continue
        nb = np.roll(f, shift=(-int(ci[2]), -int(ci[1]), -int(ci[0])), axis=(0, 1, 2))
        for a in range(3):
            if ci[a]:
                g[a] += 3.0 * wi * ci[a] * nb
        lap += 6.0 * wi * (nb - f)
    return g.reshape(3, -1), lap.reshape(-1)


def budget(params, precision, state, fluid, steps):
    """Rounding budgets (E_u, E_p) of u and p after `steps` steps (see the module
    docstring); state holds the oracle's N, B, phi, u, p."""
    Q = params["lattice"]
    shape = (params.get("nz", 1), params["ny"], params["nx"])
    c, w = _stencil(Q)
    w0 = w[0]
    chi = oracle.lattice_tables(Q, params.get("M_phi", 0.02))["chi"]
    N, B, phi, u, p = (state[k] for k in ("N", "B", "phi", "u", "p"))
    base = np.zeros(Q) if precision == 0 else chi
    S_N = np.abs(N[:, fluid] - base[:, None]).sum(0).max()
    gphi, lap = _grad_lap(phi, c, w, shape)
    G = np.sqrt((gphi[:, fluid] ** 2).sum(0)).max()
    L = np.abs(lap[fluid]).max()
    ph = np.clip(phi[fluid], 0.0, 1.0)
    mu0 = (48.0 / params["W"]) * np.abs(ph * (1 - ph) * (ph - 0.5)).max()
    sigma, W = params["sigma"], params["W"]
    rho_l, rho_g = params["rho_l"], params["rho_g"]
    drho = abs(rho_l - rho_g)
    Gu = 0.0
    for a in range(3):
        ga, _ = _grad_lap(u[a], c, w, shape)
        Gu = max(Gu, np.abs(ga[:, fluid]).max())
    nu_max = max(params["mu_l"] / rho_l, params["mu_g"] / rho_g)
    g = np.asarray(params.get("g", (0, 0, 0)), float)
    S_F = (sigma * (mu0 + 1.5 * W * L) * G
           + drho * G * (np.abs(p[fluid]).max() + 2.0 * nu_max * Gu) + max(rho_l, rho_g) * np.abs(g).max())
    ur = U_R[precision]
    rho_min = min(rho_l, rho_g)
    umax = np.abs(u[:, fluid]).max()
    to_p = 2.0 * w0 / (1 - w0) * umax                   # p depends on u through w_0 u^2 / 2
    E_u = 8.0 * ur * (S_N + S_F / (2.0 * rho_min))
    E_p = 8.0 * ur * S_N / (3.0 * (1 - w0)) + to_p * E_u
    E_u, E_p = steps * E_u, steps * E_p
    # every step reads a color the GPU holds in its own precision (the initial
    # or written one included, which the oracle keeps in double): one unit
    # roundoff, gained 12 (1 - w_0) by the Laplacian
    du = 2.0 * ur * sigma * 1.5 * W * 12.0 * (1 - w0) * G / (2.0 * rho_min)
    du_later = 0.0
    if precision == 2:
        # and populations stored with 11 significant bits: N from the first
        # step on (the initial or written state too: chi itself is not on the
        # FP16 grid), B through the color that the next steps gather from it
        nm = Q - 1
        dN = 2.0 ** -12 * np.abs(N[1:, fluid] - chi[1:, None]).max()
        dB = 2.0 ** -12 * np.abs(B[1:, fluid] - 0.5 * chi[1:, None]).max()
        du += nm * dN
        du_later = sigma * 1.5 * W * 12.0 * (1 - w0) * nm * dB * G / (2.0 * rho_min)
        E_p += steps * nm * dN / (3.0 * (1 - w0))
    later = max(steps - 1, 0)
    E_u += steps * du + later * du_later
    E_p += to_p * (steps * du + later * du_later)
    # the pressure integrates the divergence of the velocity error
    # (dp/dt = -c_s^2 div u, a lattice divergence at most D times the error):
    # a velocity error growing by du per step adds D/3 du n (n - 1)/2 to p
    D = 2 if Q == 9 else 3
    E_p += D / 3.0 * (du + du_later) * steps * later / 2.0
    return E_u, E_p


def errors(got, want, params, precision, fluid, steps):
    """Per field: (error, bound).  N, B, phi: relative L-infinity error against
    the precision's bound; u, p: max|diff| against tol * max|oracle| + E."""
    out = {}
    tol = TOL[precision]
    for f in ("N", "B", "phi"):
        if f in got:
            out[f] = (rel(got[f], want[f], fluid), tol)
    if "u" in got or "p" in got:
        E = dict(zip(("u", "p"), budget(params, precision, want, fluid, steps)))
        for f in ("u", "p"):
            if f in got:
                diff = np.abs(got[f][..., fluid] - want[f][..., fluid]).max()
                scale = np.abs(want[f][..., fluid]).max()
                out[f] = (diff, tol * scale + E[f])
                out[f + "/own scale"] = (diff / scale if scale > 0 else 0.0, None)
    return out


def check(got, want, params, precision, fluid, steps, label=""):
    """Assert every field within its bound; returns the errors (printed too)."""
    err = errors(got, want, params, precision, fluid, steps)
    bad = {k: v for k, v in err.items() if v[1] is not None and not v[0] <= v[1]}
    shown = {k: ("%.2e" % v[0]) + ("" if v[1] is None else " (<= %.2e)" % v[1]) for k, v in err.items()}
    print("parity", label, "precision", precision, shown)
    assert not bad, "%s: above the bound: %s" % (label, shown)
    return err


def read_gpu(dom, fields=("N", "B", "phi", "u", "p")):
    return {f: dom.read(f) for f in fields}


def read_oracle(o, fields=("N", "B", "phi", "u", "p")):
    return {f: o.get(f) for f in fields}
