/*
 * lbm.h -- C ABI of the GB300 color-gradient lattice Boltzmann wetting step.
 *
 * The library advances a two-phase color-gradient lattice Boltzmann model
 * (D2Q9 as in Appendix A of Bhattacharya et al., arXiv 2605.30878, or its
 * D3Q19 extension) with the ghost-node wetting boundary condition of
 * Eq. (ghost-nodePrescription) on staircase solids of any shape.  Every step
 * of the time integration runs in CUDA kernels for sm_103a; nothing here
 * falls back to the CPU.
 *
 * Conventions shared by every call:
 *   - node index      node = x + nx*(y + ny*z), 0 <= x < nx, ...; nz = 1 in 2D
 *   - lattice units   dx = dt = 1, c_s^2 = 1/3 (Appendix A)
 *   - host arrays     owned by the caller, read or written during the call only
 *   - device memory   owned by the library, or carved from a caller workspace
 *   - errors          no call aborts or throws; each returns an lbm_status and
 *                     lbm_last_error() gives a one-line message.  Device-side
 *                     failures (non-finite values, a halo copy that did not
 *                     complete) are latched on the device and reported by the
 *                     next synchronising call (lbm_diagnostics, lbm_sync,
 *                     lbm_batch_sync).  After LBM_ERR_TIMEOUT the domain is
 *                     poisoned: a tile of some step was skipped, so its state
 *                     is wrong, and every later call that would change or
 *                     advance it (lbm_step, lbm_init_*, lbm_write_state,
 *                     lbm_profile_steps, lbm_batch_create/step/tune with it)
 *                     returns LBM_ERR_TIMEOUT; destroy it and create another.
 *   - threads         one host thread per domain at a time
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain lbm_domain;      /* opaque */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,          /* invalid argument, mask or ghost list */
    LBM_ERR_OOM = -2,          /* device allocation failed or workspace too small */
    LBM_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    LBM_ERR_UNSTABLE = -4,     /* a step produced a non-finite velocity or color */
    LBM_ERR_TIMEOUT = -5,      /* a bounded device wait gave up (a step kernel's TMA halo copy did not
                                  complete within 1 s or 2^22 polls); the domain is poisoned, see above */
    LBM_ERR_UNSUPPORTED = -6,  /* valid request the library does not implement */
    LBM_ERR_BOUNDS = -7        /* debug bounds-check library only (liblbm_debug.so): a kernel computed an
                                  index outside its array; the access was skipped, the state is not valid */
} lbm_status;

typedef enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 } lbm_lattice;

/* Ghost-node color rule: the paper's Eq. (ghost-nodePrescription), or the
 * comparison scheme of Fakhari et al., Eq. (ghostNodeFakhari), evaluated in
 * the conjugate form 4 phi_F/(a + sqrt(a^2 - 2 eps phi_F)) - phi_F,
 * a = 1 + eps/2, which is exact algebra and stays accurate at theta -> 90 deg. */
typedef enum { LBM_GHOST_PRESENT = 0, LBM_GHOST_FAKHARI = 1 } lbm_ghost_rule;

/* Arithmetic and storage type of the step.  LBM_FP64: double throughout.
 * LBM_FP32: float arithmetic; populations stored in float as deviations from
 * the rest state (N_i - chi_i, B_i - chi_i/2), which keeps the small pressure
 * p = p_h/rho of a dense liquid representable.  LBM_FP32_STORE_FP16: float
 * arithmetic, the moving populations' deviations stored in FP16 scaled by
 * 2^16 (N) and 2^7 (B), the rest populations in float; the collision fixes
 * each node's totals (sum of N_i - chi_i is 0, sum of B_i - chi_i/2 is
 * phi - 1/2) and the rest populations are written as those totals less the
 * rounded moving populations, so storage conserves mass.  phi, u, p stay
 * float.  Diagnostics reduce in double in every mode. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP32_STORE_FP16 = 2 } lbm_precision;

/* Physical and numerical parameters (lattice units).  The model of Sec. II
 * and Appendix A: phi = 1 is the liquid (heavier) phase, phi = 0 the gas;
 * rho = rho_l phi + rho_g (1-phi), 1/nu = phi/nu_l + (1-phi)/nu_g with
 * nu_k = mu_k/rho_k, tau = 1/2 + nu/c_s^2.  Interface mobility M_phi fixes
 * the rest color weight alpha (Appendix A, taken at reference pressure 0).
 * W >= 4 (Eq. ghost-nodePrescription keeps |eps| <= 1).  theta is the
 * contact angle measured through the liquid (Eq. sharpWettingCondition).  A
 * non-periodic axis must have solid nodes on both end layers. */
typedef struct {
    int32_t lattice;        /* lbm_lattice */
    int32_t nx, ny, nz;     /* grid; nz = 1 for D2Q9 */
    uint32_t periodic;      /* bit0 x, bit1 y, bit2 z */
    int32_t precision;      /* lbm_precision */
    int32_t ghost_rule;     /* lbm_ghost_rule */
    int32_t reserved;       /* must be 0 */
    double rho_l, rho_g;    /* phase densities, > 0 */
    double mu_l, mu_g;      /* dynamic viscosities, > 0 */
    double sigma;           /* surface tension, Eq. (surfaceTensionForce) */
    double W;               /* interface width */
    double M_phi;           /* interface mobility, 0 < M_phi (alpha in (0,1)) */
    double theta;           /* contact angle, radians */
    double g[3];            /* body acceleration; F_b = rho g */
} lbm_params;

/* One solid boundary node (a solid node with at least one fluid neighbour
 * in the lattice stencil, Sec. I) and its unit normal pointing out of the
 * solid into the fluid (Fig. 2).  In 2D n[2] must be 0. */
typedef struct {
    int64_t node;
    double n[3];
} lbm_ghost;

/* Optional analytic description of the solid surface, used only by
 * lbm_diagnostics to measure the contact angle and the apex height.  Each
 * phi = 1/2 interface point is taken at its nearest periodic image from
 * center, so the drop must lie within half a box of it in every periodic
 * direction. */
typedef struct {
    int32_t kind;           /* 0 none, 1 circle (2D) / sphere (3D), 2 plane */
    int32_t reserved;
    double center[3];       /* circle/sphere centre, or a point on the plane near the drop */
    double radius;          /* circle/sphere radius */
    double normal[3];       /* plane: unit normal out of the solid; circle/sphere: apex axis */
    double exclude;         /* interface points closer than this to the surface are not fitted */
} lbm_probe;

/* Reductions over fluid nodes, accumulated in FP64 on the device. */
typedef struct {
    double phi_sum;         /* sum of phi: liquid volume (area in 2D) */
    double mass_liquid;     /* rho_l * sum phi */
    double mass_gas;        /* rho_g * sum (1 - phi) */
    double pop_sum;         /* sum of all N_i: equals the fluid node count after each step */
    double max_u;           /* max |u| (spurious currents at rest) */
    double p_in, p_out;     /* mean p_h = rho p over nodes with phi > 1-1e-3 / phi < 1e-3 */
    double fit_center[3];   /* least-squares circle/sphere through the phi = 1/2 crossings */
    double fit_radius;
    double contact_angle;   /* radians, from the fit and the probe surface; NaN without probe */
    double apex;            /* max over phi = 1/2 crossings of (x - center).normal */
    int64_t n_in, n_out, n_iface, n_fit, n_fluid;
    int64_t step;           /* steps taken since the last init */
    int32_t nan_flag;       /* 1 if any fluid node holds a non-finite value */
    int32_t reserved;
} lbm_diag;

/* State fields for lbm_read_state / lbm_write_state (host arrays of doubles). */
typedef enum {
    LBM_FIELD_N = 0,        /* [Q][nodes]  color-blind populations after streaming */
    LBM_FIELD_B = 1,        /* [Q][nodes]  liquid-phase populations after streaming */
    LBM_FIELD_PHI = 2,      /* [nodes]     color; ghost nodes hold their last ghost value */
    LBM_FIELD_U = 3,        /* [3][nodes]  velocity of the last step, 0 at solid nodes */
    LBM_FIELD_P = 4         /* [nodes]     auxiliary pressure p = p_h/rho of the last step */
} lbm_field;

/* Device bytes a domain with these parameters and n_ghosts ghost nodes
 * needs (state, ghost table and reduction scratch); 0 if the parameters are
 * invalid.  Use it to size a caller workspace or to admit work. */
size_t lbm_domain_bytes(const lbm_params* params, int64_t n_ghosts);

/* Create a domain (Sec. II-III).  solid: host uint8[nx*ny*nz], nonzero =
 * solid.  ghosts: host array listing every solid node with a fluid stencil
 * neighbour exactly once, with unit normals (|n| within 1e-6 of 1).  The
 * library computes, in FP64, each ghost's fluid point x_F = x_G + n
 * (Fig. 2) and its bilinear (2D) / trilinear (3D) weights over the fluid
 * corners of the cell holding x_F, renormalised; a ghost with no fluid
 * corner uses its fluid stencil neighbour most aligned with n.
 * dev_workspace: NULL to let the library allocate (from a memory pool of the
 * current device that keeps destroyed domains' workspaces for later domains;
 * see lbm_release_cached_memory), else a device pointer of
 * ws_bytes >= lbm_domain_bytes(...) that the caller keeps alive until
 * lbm_destroy.  cuda_stream: cudaStream_t every device call is issued on
 * (NULL = default stream).  The step kernel copies each tile's color and
 * velocity halo with tiled TMA copies where the tile needs no periodic image
 * in y and z; with the environment variable LBM_HALO_COPY=elements set when
 * the domain is created, every tile copies its halo element by element
 * instead (same results; the reference the tiled copies are tested
 * against).  Errors: LBM_ERR_ARG (parameters, mask or ghost list),
 * LBM_ERR_OOM, LBM_ERR_CUDA.  On error *out is NULL. */
lbm_status lbm_create_domain(const lbm_params* params, const uint8_t* solid,
                             const lbm_ghost* ghosts, int64_t n_ghosts,
                             void* dev_workspace, size_t ws_bytes,
                             void* cuda_stream, lbm_domain** out);

/* Initial state with a circular/spherical drop (Eq. equilibriumPhaseField):
 * phi = (1 + tanh(2 (R0 - |x - centre|)/W))/2 at fluid nodes, |x - centre|
 * taken to the nearest periodic image on periodic axes; ghost nodes hold
 * (1 + cos theta)/2 (Sec. III); N_i = chi_i (the equilibrium at u = 0,
 * p = 0), B_i = phi N_i; u = 0, p = 0.  Asynchronous on the domain stream. */
lbm_status lbm_init_droplet(lbm_domain* dom, const double centre[3], double R0);

/* Same initial state from a host color field phi[nodes] (values at solid
 * nodes are ignored). */
lbm_status lbm_init_phi(lbm_domain* dom, const double* phi_host);

/* Advance n >= 0 time steps, asynchronously on the domain stream.  One step:
 * ghost update, Eq. (ghost-nodePrescription); at every fluid node the
 * isotropic stencils of phi (and of the previous velocity), the forces of
 * Eqs. (surfaceTensionForce), (pressCorrection), (viscCorrection),
 * (totalForce), the fields of Eqs. (velUpdate), (pressureUpdate), the
 * collision of Eq. (MRTCOLL) with Eq. (forceGuo), the segregation of Eq.
 * (segragationStepBlue); streaming, Eqs. (propTotal), (propBlue), with
 * halfway bounce-back at solid neighbours; the color of Eq. (phiUpdate).
 * The steps are replayed from a captured CUDA graph.  Errors: LBM_ERR_ARG
 * (n < 0), LBM_ERR_CUDA. */
lbm_status lbm_step(lbm_domain* dom, int64_t n);

/* Wait for the domain stream; LBM_ERR_UNSTABLE if a step since the last
 * check produced a non-finite velocity or color. */
lbm_status lbm_sync(lbm_domain* dom);

/* Reductions of the current state (see lbm_diag); probe may be NULL.
 * Synchronises the domain stream. */
lbm_status lbm_diagnostics(lbm_domain* dom, const lbm_probe* probe, lbm_diag* out);

/* Copy one state field to / from a host double array laid out as in
 * lbm_field (FP32 domains convert).  read synchronises; write is ordered
 * before later work on the domain stream and returns after the copy.
 * Populations read back as 0 at non-fluid nodes; a written velocity is taken
 * as 0 there (the stencils read it as the wall's velocity). */
lbm_status lbm_read_state(lbm_domain* dom, int32_t field, double* host_out);
lbm_status lbm_write_state(lbm_domain* dom, int32_t field, const double* host_in);

/* Instrumented stepping: advance n >= 1 steps launching the three kernels one
 * by one (no graph) with CUDA events around each, and add to kernel_ms[0..2]
 * the milliseconds spent in the ghost update, the fused step kernel and the
 * color kernel.  Same arithmetic and results as lbm_step; synchronises. */
lbm_status lbm_profile_steps(lbm_domain* dom, int64_t n, double kernel_ms[3]);

/* Ghost table as computed by lbm_create_domain: per ghost up to 4 (2D) or
 * 8 (3D) corner node indices and weights (unused slots: weight 0). */
lbm_status lbm_ghost_table(lbm_domain* dom, int64_t* corner, double* weight, int32_t* n_corner);

/* Number of ghosts that used the most-aligned-neighbour fallback. */
int64_t lbm_ghost_fallbacks(const lbm_domain* dom);

/* Kernel launches one lbm_step(dom, 1) issues, and the algorithmic device
 * bytes one step moves per fluid node (populations, fields, node type). */
int32_t lbm_launches_per_step(const lbm_domain* dom);
double  lbm_bytes_per_fluid_node(const lbm_domain* dom);
int64_t lbm_fluid_nodes(const lbm_domain* dom);

/* Per-phase sums of a color field that already sits in the caller's device
 * memory, for callers that cannot allocate device memory when they need them
 * (a program whose device memory all belongs to its own pool allocator, a
 * real-time loop that forbids allocation after start-up, a plugin whose host
 * reserves every allocation).  The paper has no counterpart: this is a
 * service of this library, not a step of the method.
 *   dev_class  uint8[n_nodes] node classes, 0 = fluid (others are skipped)
 *   dev_phi    T[n_nodes] color, T = float (LBM_FP32) or double (LBM_FP64)
 *   dev_u      T[n_components][plane] velocity components (may be NULL if
 *              n_components = 0), plane >= n_nodes
 *   dev_out    double[6], written: fluid node count, sum phi, rho_l sum phi,
 *              rho_g sum (1-phi), max |u| over the nodes where |u|^2 is
 *              finite, count of fluid nodes whose phi or |u|^2 is NaN or
 *              infinite (the sums include such values as they are)
 * Everything is device memory owned by the caller; the call only enqueues two
 * kernels on cuda_stream (NULL = default stream) and returns.  It allocates
 * nothing: its scratch is a static 64 KiB array inside the library that each
 * GPU loading the library keeps until the process exits.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call outside any stream capture.  The cached
 * address belongs to the device's primary context: after cudaDeviceReset
 * (or any reset of that context) the library reloads and the array may
 * move, so do not call this entry point again in that process.  All calls on a
 * GPU share the array, so calls whose kernels overlap on the GPU (different
 * streams, no ordering between them) race and give wrong sums; calls on one
 * stream are safe.  n_nodes above 16,777,216 (the array's capacity of 1024
 * blocks x 16384 nodes) is rejected with LBM_ERR_ARG.  Errors: LBM_ERR_ARG,
 * LBM_ERR_CUDA; a message goes to err[err_len] when err is not NULL. */
lbm_status lbm_phase_sums_noalloc(const uint8_t* dev_class, const void* dev_phi, const void* dev_u,
                                  int32_t precision, int32_t n_components, int64_t n_nodes,
                                  int64_t plane, double rho_l, double rho_g, double* dev_out,
                                  void* cuda_stream, char* err, size_t err_len);

/* Fault-path check of the bounded halo-copy wait (no counterpart in the
 * paper: a service of this library for testing its error reporting).  The
 * step kernel waits for each tile's TMA halo copy on a shared-memory mbarrier
 * with a bounded wait; if that wait gives up, the kernel sets the domain's
 * timeout bit instead of hanging.  A copy that never lands cannot be made
 * without faulting the GPU, so this call enqueues on the domain stream one
 * block that arms an mbarrier for 4096 bytes no copy will deliver (no TMA or
 * bulk copy is issued at all), waits on it with the step kernel's own wait
 * function and a limit of timeout_ns (1e3 .. 1e9 ns), sets the same timeout
 * bit and exits with nothing in flight.  The next synchronising call then
 * returns LBM_ERR_TIMEOUT and the domain is poisoned exactly as after a real
 * timeout.  waited_ns (may be NULL) receives the block's measured wait, which
 * makes the call synchronise the stream (it then also allocates and frees 8
 * bytes of device memory with cudaMallocAsync/cudaFreeAsync).  Errors:
 * LBM_ERR_ARG (timeout_ns out of range), LBM_ERR_TIMEOUT (already
 * poisoned), LBM_ERR_CUDA, LBM_ERR_OOM. */
lbm_status lbm_debug_expire_halo_wait(lbm_domain* dom, int64_t timeout_ns, int64_t* waited_ns);

/* The bounds-checked build of this library (liblbm_debug.so, the same sources
 * compiled with LBM_DEBUG_BOUNDS; no counterpart in the paper) tests every
 * index its kernels compute against the array it addresses -- streaming pull
 * sources, bounce-back slots, halo slots, ghost corners and nodes, tiled-copy
 * boxes, batch tiles -- before the access.  A bad index sets a bit that the
 * next synchronising call reports as LBM_ERR_BOUNDS, and the access is
 * skipped (a load reads element 0, a store is dropped); nothing traps.
 * lbm_debug_bounds_checked returns 1 in that build and 0 in the production
 * library.  lbm_debug_plant_bad_index(dom, 0) points the first corner of the
 * domain's first ghost past the end of the color array, so that the next
 * step's ghost update meets an index its check must catch; it synchronises,
 * and in the production library it returns LBM_ERR_UNSUPPORTED and writes
 * nothing.  Errors: LBM_ERR_ARG (which != 0, no ghost nodes), LBM_ERR_CUDA. */
int32_t lbm_debug_bounds_checked(void);
lbm_status lbm_debug_plant_bad_index(lbm_domain* dom, int32_t which);

/* ---- Batches: several domains advanced together (no counterpart in the
 * paper, which runs one case at a time).  A batch advances domains of the same
 * lattice and precision with one launch per phase (ghost update; step, split
 * into domains with and without density contrast; color), one block per tile
 * of a flat list of the tiles of every domain, replayed from CUDA graphs.
 * Each domain keeps its own state, parameters and error flag;
 * results are bitwise identical to stepping each domain alone.  While a
 * domain belongs to a batch it must only be stepped through the batch
 * (lbm_batch_step reports LBM_ERR_ARG otherwise); reading its state and
 * diagnostics stay available. */
typedef struct lbm_batch lbm_batch;

/* Build a batch over doms[0..n-1] (not owned; they must outlive the batch).
 * Launches go to cuda_stream (NULL = default stream).  Errors: LBM_ERR_ARG
 * (mixed lattice/precision, repeated domain), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_batch_create(lbm_domain* const* doms, int32_t n, void* cuda_stream, lbm_batch** out);

/* Advance every domain of the batch n >= 0 steps, asynchronously. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t n);

/* Wait for the batch stream; LBM_ERR_UNSTABLE if any domain went non-finite. */
lbm_status lbm_batch_sync(lbm_batch* b);

/* Block tile shapes of the batched step kernels, in nodes (shape 0 is the
 * tile of the single-domain one-node kernel, shape 5 that of the two-node
 * kernel, whose threads update two x-adjacent nodes each; float arithmetic
 * runs shapes 0, 3 and 5 with two nodes per thread):
 *                    0        1        2        3        4        5
 *   D3Q19          32x4x2   32x2x4   32x8x1   32x2x2   32x4x4   64x2x2
 *   D2Q9           32x8     64x4     128x2    32x4     32x16    64x4
 *   threads float   128      256      256      64       512      128
 *   threads FP64    256      256      256      128      512      256 */
enum { LBM_BATCH_TILE_SHAPES = 6 };

/* Autotuner: time steps_per_trial batched steps with each tile shape and block
 * size above, keep the fastest; ms_per_step[LBM_BATCH_TILE_SHAPES] (may be
 * NULL) receives the timings.  Tuning advances every domain by
 * LBM_BATCH_TILE_SHAPES * (steps_per_trial + 1) steps and synchronises. */
lbm_status lbm_batch_tune(lbm_batch* b, int32_t steps_per_trial, int32_t* chosen, double* ms_per_step);

/* Current tile shape of the batch, or set one directly (0 .. LBM_BATCH_TILE_SHAPES-1). */
int32_t lbm_batch_variant(const lbm_batch* b);
lbm_status lbm_batch_set_variant(lbm_batch* b, int32_t variant);

/* Kernel launches one batched step makes: ghost update (when any domain has
 * ghost nodes), step kernel once per contrast class present, color kernel. */
int32_t lbm_batch_launches_per_step(const lbm_batch* b);

/* Message of the last failed call on b (of the last failed create if b is NULL). */
const char* lbm_batch_last_error(const lbm_batch* b);

void lbm_batch_destroy(lbm_batch* b);

/* Message of the last failed call on dom, or of the last failed
 * lbm_create_domain when dom is NULL. */
const char* lbm_last_error(const lbm_domain* dom);

/* Free the domain.  Like cudaFree it first waits for all work on the
 * device; a workspace the library allocated goes back to the device's
 * workspace pool (not to the device), ready for the next domain. */
void lbm_destroy(lbm_domain* dom);

/* Give the memory cached in the workspace pools (workspaces of destroyed
 * domains) back to the devices, e.g. before other code in the process
 * allocates device memory.  Waits for all work on those devices.  Not part of
 * the paper: a memory-management call of this library.  Errors:
 * LBM_ERR_CUDA. */
lbm_status lbm_release_cached_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
