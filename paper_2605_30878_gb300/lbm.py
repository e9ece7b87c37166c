"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the simulation runs in the CUDA library _build/liblbm.so; this
module converts Python/numpy arguments, hands the library a PyTorch-owned
device workspace and the current PyTorch stream, and raises on error codes.
There is no CPU fallback: without the compiled library every call raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY=debug selects the bounds-checked build of the same sources
# (liblbm_debug.so: every index the kernels compute is range-checked, a bad
# one is reported as LBM_ERR_BOUNDS and its access skipped); anything else the
# production library.
LIB_PATH = os.path.join(_HERE, "_build", "liblbm_debug.so" if os.environ.get("LBM_LIBRARY") == "debug"
                        else "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6
LBM_ERR_BOUNDS = -7
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_UNSTABLE",
                -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_UNSUPPORTED", -7: "LBM_ERR_BOUNDS"}
FP64, FP32, FP16 = 0, 1, 2     # FP16: FP32 arithmetic, FP16 population storage
BATCH_TILE_SHAPES = 6          # LBM_BATCH_TILE_SHAPES: tile shapes / block sizes of the batched kernels
GHOST_PRESENT, GHOST_FAKHARI = 0, 1
FIELDS = {"N": 0, "B": 1, "phi": 2, "u": 3, "p": 4}

# Every entry point include/lbm.h declares.
EXPORTS = ("lbm_domain_bytes", "lbm_create_domain", "lbm_init_droplet", "lbm_init_phi", "lbm_step", "lbm_sync",
           "lbm_diagnostics", "lbm_read_state", "lbm_write_state", "lbm_profile_steps", "lbm_ghost_table", "lbm_ghost_fallbacks",
           "lbm_launches_per_step", "lbm_bytes_per_fluid_node", "lbm_fluid_nodes", "lbm_last_error", "lbm_destroy",
           "lbm_release_cached_memory", "lbm_phase_sums_noalloc", "lbm_debug_expire_halo_wait", "lbm_debug_bounds_checked",
           "lbm_debug_plant_bad_index", "lbm_batch_create", "lbm_batch_step", "lbm_batch_sync", "lbm_batch_tune",
           "lbm_batch_variant", "lbm_batch_set_variant", "lbm_batch_launches_per_step", "lbm_batch_last_error",
           "lbm_batch_destroy")


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Params(C.Structure):
    _fields_ = [("lattice", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("periodic", C.c_uint32), ("precision", C.c_int32), ("ghost_rule", C.c_int32),
                ("reserved", C.c_int32), ("rho_l", C.c_double), ("rho_g", C.c_double), ("mu_l", C.c_double), ("mu_g", C.c_double),
                ("sigma", C.c_double), ("W", C.c_double), ("M_phi", C.c_double), ("theta", C.c_double),
                ("g", C.c_double * 3)]


class Ghost(C.Structure):
    _fields_ = [("node", C.c_int64), ("n", C.c_double * 3)]


class Probe(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("center", C.c_double * 3), ("radius", C.c_double),
                ("normal", C.c_double * 3), ("exclude", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("phi_sum", C.c_double), ("mass_liquid", C.c_double), ("mass_gas", C.c_double),
                ("pop_sum", C.c_double), ("max_u", C.c_double), ("p_in", C.c_double), ("p_out", C.c_double),
                ("fit_center", C.c_double * 3), ("fit_radius", C.c_double), ("contact_angle", C.c_double),
                ("apex", C.c_double), ("n_in", C.c_int64), ("n_out", C.c_int64), ("n_iface", C.c_int64),
                ("n_fit", C.c_int64), ("n_fluid", C.c_int64), ("step", C.c_int64), ("nan_flag", C.c_int32),
                ("reserved", C.c_int32)]


_lib = None
_dp = C.POINTER(C.c_double)


def load():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library %s is missing: run `python -c 'import __graft_entry__ as g; g.build()'`"
                           % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    L.lbm_domain_bytes.argtypes = [C.POINTER(Params), C.c_int64]
    L.lbm_domain_bytes.restype = C.c_size_t
    L.lbm_create_domain.argtypes = [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t,
                                    C.c_void_p, C.POINTER(C.c_void_p)]
    L.lbm_create_domain.restype = C.c_int
    L.lbm_init_droplet.argtypes = [C.c_void_p, _dp, C.c_double]
    L.lbm_init_droplet.restype = C.c_int
    L.lbm_init_phi.argtypes = [C.c_void_p, _dp]
    L.lbm_init_phi.restype = C.c_int
    L.lbm_step.argtypes = [C.c_void_p, C.c_int64]
    L.lbm_step.restype = C.c_int
    L.lbm_sync.argtypes = [C.c_void_p]
    L.lbm_sync.restype = C.c_int
    L.lbm_diagnostics.argtypes = [C.c_void_p, C.POINTER(Probe), C.POINTER(Diag)]
    L.lbm_diagnostics.restype = C.c_int
    L.lbm_read_state.argtypes = [C.c_void_p, C.c_int32, _dp]
    L.lbm_read_state.restype = C.c_int
    L.lbm_write_state.argtypes = [C.c_void_p, C.c_int32, _dp]
    L.lbm_write_state.restype = C.c_int
    L.lbm_profile_steps.argtypes = [C.c_void_p, C.c_int64, _dp]
    L.lbm_profile_steps.restype = C.c_int
    L.lbm_ghost_table.argtypes = [C.c_void_p, C.POINTER(C.c_int64), _dp, C.POINTER(C.c_int32)]
    L.lbm_ghost_table.restype = C.c_int
    L.lbm_ghost_fallbacks.argtypes = [C.c_void_p]
    L.lbm_ghost_fallbacks.restype = C.c_int64
    L.lbm_launches_per_step.argtypes = [C.c_void_p]
    L.lbm_launches_per_step.restype = C.c_int32
    L.lbm_bytes_per_fluid_node.argtypes = [C.c_void_p]
    L.lbm_bytes_per_fluid_node.restype = C.c_double
    L.lbm_fluid_nodes.argtypes = [C.c_void_p]
    L.lbm_fluid_nodes.restype = C.c_int64
    L.lbm_last_error.argtypes = [C.c_void_p]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_destroy.argtypes = [C.c_void_p]
    L.lbm_destroy.restype = None
    L.lbm_release_cached_memory.argtypes = []
    L.lbm_release_cached_memory.restype = C.c_int
    L.lbm_phase_sums_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int64,
                                         C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_char_p,
                                         C.c_size_t]
    L.lbm_phase_sums_noalloc.restype = C.c_int
    L.lbm_debug_expire_halo_wait.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
    L.lbm_debug_expire_halo_wait.restype = C.c_int
    L.lbm_debug_bounds_checked.argtypes = []
    L.lbm_debug_bounds_checked.restype = C.c_int32
    L.lbm_debug_plant_bad_index.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_debug_plant_bad_index.restype = C.c_int
    L.lbm_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]
    L.lbm_batch_create.restype = C.c_int
    L.lbm_batch_step.argtypes = [C.c_void_p, C.c_int64]
    L.lbm_batch_step.restype = C.c_int
    L.lbm_batch_sync.argtypes = [C.c_void_p]
    L.lbm_batch_sync.restype = C.c_int
    L.lbm_batch_tune.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), _dp]
    L.lbm_batch_tune.restype = C.c_int
    L.lbm_batch_variant.argtypes = [C.c_void_p]
    L.lbm_batch_variant.restype = C.c_int32
    L.lbm_batch_set_variant.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_batch_set_variant.restype = C.c_int
    L.lbm_batch_launches_per_step.argtypes = [C.c_void_p]
    L.lbm_batch_launches_per_step.restype = C.c_int32
    L.lbm_batch_last_error.argtypes = [C.c_void_p]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_batch_destroy.argtypes = [C.c_void_p]
    L.lbm_batch_destroy.restype = None
    _lib = L
    return L


def make_params(spec):
    """Params from a mapping with the lbm_params field names (g may be 2 or 3 long;
    precision defaults to FP32)."""
    p = Params()
    p.precision = FP32
    for name, _ in Params._fields_:
        if name == "g":
            g = list(spec.get("g", (0.0, 0.0, 0.0))) + [0.0] * 3
            p.g[:] = [float(v) for v in g[:3]]
        elif name in spec:
            setattr(p, name, spec[name])
    return p


def make_probe(kind=0, center=(0, 0, 0), radius=0.0, normal=(0, 0, 0), exclude=0.0):
    pr = Probe()
    pr.kind = kind
    pr.center[:] = [float(v) for v in (list(center) + [0.0] * 3)[:3]]
    pr.radius = float(radius)
    pr.normal[:] = [float(v) for v in (list(normal) + [0.0] * 3)[:3]]
    pr.exclude = float(exclude)
    return pr


def bounds_checked():
    """True when the loaded library is the bounds-checked build."""
    return bool(load().lbm_debug_bounds_checked())


def domain_bytes(params, n_ghosts):
    P = params if isinstance(params, Params) else make_params(params)
    return load().lbm_domain_bytes(C.byref(P), int(n_ghosts))


def last_error(handle=None):
    m = load().lbm_last_error(handle)
    return m.decode() if m else ""


def _check(status, handle=None):
    if status != LBM_OK:
        raise LbmError(status, last_error(handle))


def phase_sums_noalloc(dev_class, dev_phi, dev_u, precision, n_components, n_nodes, plane, rho_l, rho_g,
                       dev_out, stream=None):
    """Per-phase sums of caller-owned device buffers (raw device addresses as
    ints), written to dev_out (6 doubles) without any device allocation; see
    lbm_phase_sums_noalloc in include/lbm.h.  Raises LbmError on a bad status."""
    err = C.create_string_buffer(256)
    st = load().lbm_phase_sums_noalloc(dev_class, dev_phi, dev_u, int(precision), int(n_components), int(n_nodes),
                                       int(plane), float(rho_l), float(rho_g), dev_out, stream, err, 256)
    if st != LBM_OK:
        raise LbmError(st, err.value.decode())


_GHOST_DTYPE = np.dtype([("node", "<i8"), ("n", "<f8", (3,))])       # the layout of lbm_ghost


def release_cached_memory():
    """Give the workspaces of destroyed library-allocated domains, which the
    library keeps for the next domain, back to the devices."""
    _check(load().lbm_release_cached_memory())


def ghost_array(nodes, normals):
    """A contiguous lbm_ghost array (as a numpy record array) and its length."""
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1)
    normals = np.asarray(normals, dtype=np.float64).reshape(-1, 3)
    arr = np.zeros(max(1, len(nodes)), dtype=_GHOST_DTYPE)
    arr["node"][:len(nodes)] = nodes
    arr["n"][:len(nodes)] = normals
    return arr, len(nodes)


class Domain:
    """One simulation domain on the GPU.

    params: mapping with the lbm_params fields; solid: uint8 array (nz, ny, nx);
    ghosts: (nodes, normals).  workspace: "torch" (a PyTorch uint8 tensor holds the
    device state), "library" (the library calls cudaMalloc), or a torch tensor.
    stream: None for torch's current stream (or the default stream without torch),
    or a torch.cuda.Stream / raw cudaStream_t integer."""

    def __init__(self, params, solid, ghosts, workspace="torch", stream=None):
        L = load()
        self.params = params if isinstance(params, Params) else make_params(params)
        P = self.params
        self.Q = P.lattice
        self.nn = P.nx * P.ny * P.nz
        solid = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
        if solid.size != self.nn:
            raise ValueError("solid mask has %d entries, grid has %d" % (solid.size, self.nn))
        garr, ng = ghost_array(*ghosts)
        self.n_ghosts = ng
        self._ws = None
        ws_ptr, ws_bytes = None, 0
        need = L.lbm_domain_bytes(C.byref(P), ng)
        if need == 0:
            raise LbmError(LBM_ERR_ARG, "invalid parameters")
        torch = None
        if (isinstance(workspace, str) and workspace == "torch") or stream is None:
            try:
                import torch
            except ImportError:
                torch = None
        if isinstance(workspace, str):
            if workspace == "torch":
                if torch is None:
                    raise RuntimeError("workspace='torch' needs PyTorch")
                self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            elif workspace != "library":
                raise ValueError("workspace must be 'torch', 'library' or a device tensor")
        else:
            self._ws = workspace
        if self._ws is not None:
            ws_ptr, ws_bytes = self._ws.data_ptr(), self._ws.numel() * self._ws.element_size()
        if stream is None:
            stream_ptr = torch.cuda.current_stream().cuda_stream if torch is not None else None
        elif hasattr(stream, "cuda_stream"):
            stream_ptr = stream.cuda_stream
        else:
            stream_ptr = int(stream)
        self.stream_ptr = stream_ptr
        h = C.c_void_p()
        st = L.lbm_create_domain(C.byref(P), solid.ctypes.data, garr.ctypes.data, ng,
                                 ws_ptr, ws_bytes, stream_ptr, C.byref(h))
        _check(st, None)
        self.h = h

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            load().lbm_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- simulation
    def init_droplet(self, centre, R0):
        c = np.zeros(3)
        c[:len(centre)] = centre
        _check(load().lbm_init_droplet(self.h, c.ctypes.data_as(_dp), float(R0)), self.h)

    def init_phi(self, phi):
        a = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        _check(load().lbm_init_phi(self.h, a.ctypes.data_as(_dp)), self.h)

    def step(self, n=1):
        _check(load().lbm_step(self.h, int(n)), self.h)

    def sync(self):
        _check(load().lbm_sync(self.h), self.h)

    def diagnostics(self, probe=None):
        d = Diag()
        st = load().lbm_diagnostics(self.h, C.byref(probe) if probe is not None else None, C.byref(d))
        out = {}
        for name, _ in Diag._fields_:
            v = getattr(d, name)
            out[name] = list(v) if not isinstance(v, (int, float)) else v
        if st != LBM_OK and st != LBM_ERR_UNSTABLE:
            _check(st, self.h)
        out["status"] = st
        return out

    def _count(self, field):
        return {"N": self.Q * self.nn, "B": self.Q * self.nn, "phi": self.nn, "u": 3 * self.nn, "p": self.nn}[field]

    def read(self, field):
        out = np.zeros(self._count(field))
        _check(load().lbm_read_state(self.h, FIELDS[field], out.ctypes.data_as(_dp)), self.h)
        if field in ("N", "B"):
            return out.reshape(self.Q, self.nn)
        if field == "u":
            return out.reshape(3, self.nn)
        return out

    def write(self, field, values):
        a = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1))
        if a.size != self._count(field):
            raise ValueError("field %s needs %d values" % (field, self._count(field)))
        _check(load().lbm_write_state(self.h, FIELDS[field], a.ctypes.data_as(_dp)), self.h)

    def profile_steps(self, n):
        """Run n steps kernel by kernel; return milliseconds in (ghost, step, phi)."""
        ms = np.zeros(3)
        _check(load().lbm_profile_steps(self.h, int(n), ms.ctypes.data_as(_dp)), self.h)
        return ms

    def ghost_table(self):
        GK = 4 if self.Q == 9 else 8
        n = max(1, self.n_ghosts)
        cor = np.zeros(n * GK, np.int64)
        wt = np.zeros(n * GK)
        nc = np.zeros(n, np.int32)
        _check(load().lbm_ghost_table(self.h, cor.ctypes.data_as(C.POINTER(C.c_int64)), wt.ctypes.data_as(_dp),
                                      nc.ctypes.data_as(C.POINTER(C.c_int32))), self.h)
        return cor.reshape(n, GK)[:self.n_ghosts], wt.reshape(n, GK)[:self.n_ghosts], nc[:self.n_ghosts]

    def debug_expire_halo_wait(self, timeout_ns, measure=False):
        """Make one block's bounded halo-copy wait run out on the domain stream
        (no copy is issued); the next sync reports LBM_ERR_TIMEOUT.  With
        measure=True, synchronises and returns the measured wait in ns."""
        w = C.c_int64(-1)
        _check(load().lbm_debug_expire_halo_wait(self.h, int(timeout_ns), C.byref(w) if measure else None), self.h)
        return w.value if measure else None

    def debug_plant_bad_index(self, which=0):
        """Bounds-checked library only: make the next step meet an index its
        checks must catch (see lbm_debug_plant_bad_index)."""
        _check(load().lbm_debug_plant_bad_index(self.h, int(which)), self.h)

    def ghost_fallbacks(self):
        return load().lbm_ghost_fallbacks(self.h)

    def launches_per_step(self):
        return load().lbm_launches_per_step(self.h)

    def bytes_per_fluid_node(self):
        return load().lbm_bytes_per_fluid_node(self.h)

    def fluid_nodes(self):
        return load().lbm_fluid_nodes(self.h)


class Batch:
    """Several domains (same lattice and precision) advanced by one launch per
    phase; see lbm_batch_* in include/lbm.h.  Keeps references to
    its domains so they outlive it."""

    def __init__(self, domains, stream=None):
        L = load()
        self.domains = list(domains)
        arr = (C.c_void_p * len(self.domains))(*[d.h.value for d in self.domains])
        if stream is None:
            stream = self.domains[0].stream_ptr
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = C.c_void_p()
        st = L.lbm_batch_create(arr, len(self.domains), stream, C.byref(h))
        if st != LBM_OK:
            raise LbmError(st, L.lbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, load().lbm_batch_last_error(self.h).decode())

    def step(self, n=1):
        self._check(load().lbm_batch_step(self.h, int(n)))

    def sync(self):
        self._check(load().lbm_batch_sync(self.h))

    def tune(self, steps_per_trial=20):
        """Time every tile shape, keep the fastest; returns (chosen, ms per step of each)."""
        ch = C.c_int32()
        ms = np.zeros(BATCH_TILE_SHAPES)
        self._check(load().lbm_batch_tune(self.h, int(steps_per_trial), C.byref(ch), ms.ctypes.data_as(_dp)))
        return ch.value, ms

    @property
    def variant(self):
        return load().lbm_batch_variant(self.h)

    def set_variant(self, v):
        self._check(load().lbm_batch_set_variant(self.h, int(v)))

    def launches_per_step(self):
        return load().lbm_batch_launches_per_step(self.h)

    def close(self):
        """Wait for the batch's launches and give its constant-table slots back."""
        if getattr(self, "h", None):
            load().lbm_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
