"""ctypes front end of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product package never imports it, and it
never imports the product package.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

GMAX = 8
FIELDS = {"N": 0, "B": 1, "phi": 2, "u": 3, "p": 4}


class Params(C.Structure):
    _fields_ = [("lattice", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("periodic", C.c_uint32), ("ghost_rule", C.c_int32),
                ("rho_l", C.c_double), ("rho_g", C.c_double), ("mu_l", C.c_double), ("mu_g", C.c_double),
                ("sigma", C.c_double), ("W", C.c_double), ("M_phi", C.c_double), ("theta", C.c_double),
                ("g", C.c_double * 3)]


class Ghost(C.Structure):
    _fields_ = [("node", C.c_int64), ("n", C.c_double * 3)]


class Probe(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("center", C.c_double * 3),
                ("radius", C.c_double), ("normal", C.c_double * 3), ("exclude", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("phi_sum", C.c_double), ("mass_liquid", C.c_double), ("mass_gas", C.c_double),
                ("pop_sum", C.c_double), ("max_u", C.c_double), ("p_in", C.c_double), ("p_out", C.c_double),
                ("fit_center", C.c_double * 3), ("fit_radius", C.c_double), ("contact_angle", C.c_double),
                ("apex", C.c_double), ("n_in", C.c_int64), ("n_out", C.c_int64), ("n_iface", C.c_int64),
                ("n_fit", C.c_int64), ("n_fluid", C.c_int64), ("step", C.c_int64),
                ("nan_flag", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if not isinstance(v, (int, float)) else v
        return d


_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_create.argtypes = [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_int64,
                                 C.POINTER(C.c_void_p), C.c_char_p, C.c_int]
        L.orc_create.restype = C.c_int
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_init_phi.argtypes = [C.c_void_p, _dp]
        L.orc_init_droplet.argtypes = [C.c_void_p, _dp, C.c_double]
        L.orc_step.argtypes = [C.c_void_p, C.c_int64]
        L.orc_get.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_set.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_diagnostics.argtypes = [C.c_void_p, C.POINTER(Probe), C.POINTER(Diag)]
        L.orc_step_sample.argtypes = [C.c_void_p, _i64p, C.c_int64, _dp, _dp, _dp, _dp, _dp]
        L.orc_ghost_fallbacks.argtypes = [C.c_void_p]
        L.orc_ghost_fallbacks.restype = C.c_int64
        L.orc_update_ghosts.argtypes = [C.c_void_p]
        L.orc_ghost_table.argtypes = [C.c_void_p, _i64p, _dp, C.POINTER(C.c_int32)]
        L.orc_node_class.argtypes = [C.c_void_p, C.c_int64]
        L.orc_node_class.restype = C.c_int
        L.orc_lattice_tables.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int32), _dp, _dp,
                                         C.POINTER(C.c_int32), _dp, _dp, C.POINTER(C.c_int32)]
        L.orc_lattice_tables.restype = C.c_int
        L.orc_equilibrium.argtypes = [C.c_int, C.c_double, _dp, C.c_double, _dp]
        L.orc_macro.argtypes = [C.c_int, C.c_double, _dp, _dp, C.c_double, _dp, _dp]
        L.orc_collide.argtypes = [C.c_int, C.c_double, _dp, _dp, C.c_double, _dp, C.c_double,
                                  C.c_double, _dp]
        L.orc_segregate.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp, C.c_double, _dp, _dp]
        L.orc_ghost_rule.argtypes = [C.c_double, C.c_double]
        L.orc_ghost_rule.restype = C.c_double
        L.orc_ghost_rule_fakhari.argtypes = [C.c_double, C.c_double]
        L.orc_ghost_rule_fakhari.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _vec3(v):
    a = np.zeros(3)
    a[:len(v)] = v
    return a


def make_params(spec):
    """spec: a mapping with the keys of Params (g may have 2 or 3 entries)."""
    p = Params()
    for name, _ in Params._fields_:
        if name == "g":
            p.g[:] = list(_vec3(spec.get("g", (0, 0, 0))))
        elif name in spec:
            setattr(p, name, spec[name])
    return p


def make_probe(kind=0, center=(0, 0, 0), radius=0.0, normal=(0, 0, 0), exclude=0.0):
    pr = Probe()
    pr.kind = kind
    pr.center[:] = list(_vec3(center))
    pr.radius = radius
    pr.normal[:] = list(_vec3(normal))
    pr.exclude = exclude
    return pr


# ---------------------------------------------------------------- single-node pieces

def lattice_tables(lattice, M_phi=0.02, gram_schmidt=False):
    Q = lattice
    c = np.zeros(3 * Q, np.int32)
    w, chi = np.zeros(Q), np.zeros(Q)
    opp, st = np.zeros(Q, np.int32), np.zeros(Q, np.int32)
    M, Minv = np.zeros(Q * Q), np.zeros(Q * Q)
    r = lib().orc_lattice_tables(lattice, M_phi, int(gram_schmidt), c.ctypes.data_as(C.POINTER(C.c_int32)),
                                 _d(w), _d(chi), opp.ctypes.data_as(C.POINTER(C.c_int32)), _d(M), _d(Minv),
                                 st.ctypes.data_as(C.POINTER(C.c_int32)))
    if r != Q:
        raise RuntimeError("lattice construction failed")
    return dict(c=c.reshape(Q, 3), w=w, chi=chi, opp=opp, M=M.reshape(Q, Q), Minv=Minv.reshape(Q, Q),
                is_stress=st.astype(bool))


def equilibrium(lattice, u, p, M_phi=0.02):
    out = np.zeros(lattice)
    lib().orc_equilibrium(lattice, M_phi, _d(_vec3(u)), p, _d(out))
    return out


def macro(lattice, N, F, rho, M_phi=0.02):
    u = np.zeros(3)
    p = C.c_double()
    lib().orc_macro(lattice, M_phi, _d(np.ascontiguousarray(N, dtype=np.float64)), _d(_vec3(F)), rho,
                    _d(u), C.byref(p))
    return u, p.value


def collide(lattice, N, u, p, F, rho, tau, M_phi=0.02):
    out = np.zeros(lattice)
    lib().orc_collide(lattice, M_phi, _d(np.ascontiguousarray(N, dtype=np.float64)), _d(_vec3(u)), p,
                      _d(_vec3(F)), rho, tau, _d(out))
    return out


def segregate(lattice, Nst, phi, gphi, p, W=4.0, M_phi=0.02):
    """Eq. (segragationStepBlue) at one node: the post-collision color
    populations B* from N*, phi, grad phi and the pressure p."""
    out = np.zeros(lattice)
    lib().orc_segregate(lattice, M_phi, W, phi, _d(_vec3(gphi)), p,
                        _d(np.ascontiguousarray(Nst, dtype=np.float64)), _d(out))
    return out


def ghost_rule(phiF, eps):
    return lib().orc_ghost_rule(float(phiF), float(eps))


def ghost_rule_fakhari(phiF, eps):
    return lib().orc_ghost_rule_fakhari(float(phiF), float(eps))


# ---------------------------------------------------------------- whole grid

class Oracle:
    """One simulation domain on the host, FP64, literal formulation."""

    def __init__(self, params, solid, ghosts):
        """params: mapping (see make_params); solid: uint8 array of shape (nz, ny, nx) or flat;
        ghosts: structured array / list of (node, (nx, ny, nz)) with unit normals."""
        self.params = make_params(params)
        P = self.params
        self.Q = P.lattice
        self.shape = (P.nz, P.ny, P.nx)
        self.nn = P.nx * P.ny * P.nz
        solid = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
        if solid.size != self.nn:
            raise ValueError("mask size mismatch")
        nodes, normals = ghosts
        nodes = np.asarray(nodes, dtype=np.int64)
        normals = np.asarray(normals, dtype=np.float64).reshape(-1, 3)
        arr = (Ghost * max(1, len(nodes)))()
        for k in range(len(nodes)):
            arr[k].node = int(nodes[k])
            arr[k].n[:] = list(normals[k])
        self.n_ghosts = len(nodes)
        err = C.create_string_buffer(512)
        h = C.c_void_p()
        r = lib().orc_create(C.byref(P), solid.ctypes.data, C.cast(arr, C.c_void_p), len(nodes),
                             C.byref(h), err, 512)
        if r != 0:
            raise ValueError(err.value.decode())
        self.h = h
        self.solid = solid

    def __del__(self):
        if lib is None:
            return
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def init_phi(self, phi):
        a = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        lib().orc_init_phi(self.h, _d(a))

    def init_droplet(self, centre, R0):
        lib().orc_init_droplet(self.h, _d(_vec3(centre)), float(R0))

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    def _count(self, field):
        return {"N": self.Q * self.nn, "B": self.Q * self.nn, "phi": self.nn, "u": 3 * self.nn,
                "p": self.nn}[field]

    def get(self, field):
        out = np.zeros(self._count(field))
        lib().orc_get(self.h, FIELDS[field], _d(out))
        if field in ("N", "B"):
            return out.reshape(self.Q, self.nn)
        if field == "u":
            return out.reshape(3, self.nn)
        return out

    def set(self, field, values):
        a = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1))
        if a.size != self._count(field):
            raise ValueError("size mismatch for field %s" % field)
        lib().orc_set(self.h, FIELDS[field], _d(a))

    def diagnostics(self, probe=None):
        d = Diag()
        lib().orc_diagnostics(self.h, C.byref(probe) if probe is not None else None, C.byref(d))
        return d.as_dict()

    def step_sample(self, nodes):
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        n = len(nodes)
        N, B = np.zeros((n, self.Q)), np.zeros((n, self.Q))
        u, p, phi = np.zeros((n, 3)), np.zeros(n), np.zeros(n)
        lib().orc_step_sample(self.h, nodes.ctypes.data_as(_i64p), n, _d(N), _d(B), _d(u), _d(p), _d(phi))
        return dict(N=N, B=B, u=u, p=p, phi=phi)

    def update_ghosts(self):
        lib().orc_update_ghosts(self.h)

    def ghost_fallbacks(self):
        return lib().orc_ghost_fallbacks(self.h)

    def node_class(self, node):
        return lib().orc_node_class(self.h, int(node))

    def ghost_table(self):
        n = max(1, self.n_ghosts)
        cor = np.zeros(n * GMAX, np.int64)
        wt = np.zeros(n * GMAX)
        nc = np.zeros(n, np.int32)
        lib().orc_ghost_table(self.h, cor.ctypes.data_as(_i64p), _d(wt), nc.ctypes.data_as(C.POINTER(C.c_int32)))
        return cor.reshape(n, GMAX)[:self.n_ghosts], wt.reshape(n, GMAX)[:self.n_ghosts], nc[:self.n_ghosts]
