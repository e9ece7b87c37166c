// Host side of the C ABI declared in include/lbm.h: validation, ghost-table
// preparation (x_F = x_G + n_s, Fig. 2), device memory layout, CUDA-graph
// step replay, state transfer and diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <unistd.h>

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_domain_access.h"
#include "lbm_launch.cuh"

using namespace lbmgpu;

static_assert(kTileVariants == LBM_BATCH_TILE_SHAPES, "tile shapes of the kernels and of the header");

namespace {

thread_local std::string g_create_error;

constexpr size_t ALIGN = 256;
constexpr int GRAPH_STEPS = 8;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    int px = 0;                      // row pitch of the device fields: nx rounded up to 4 (16-byte rows)
    int64_t nn = 0, plane = 0;       // device nodes px * ny * nz (columns nx..px-1 are solid padding)
    int64_t nn_dense = 0;            // grid nodes nx * ny * nz (host arrays)
    size_t elem = 0;                 // bytes of a field value (phi, u, p, ghost weights)
    size_t pop_elem = 0;             // bytes of a stored moving population
    size_t rest_elem = 0;            // bytes of a stored rest population
    size_t pop_bytes = 0;            // bytes of one population array (Q planes)
    int Q = 0, D = 0, GK = 0;
    size_t off_N[2], off_B[2], off_phi, off_u[2], off_p, off_cls, off_mask, off_gnode, off_gcorner, off_gwt,
        off_err, off_partial, off_dout, off_stage;
    size_t total = 0;
};

bool make_layout(const lbm_params* P, int64_t ng, Layout& L, std::string& err) {
    if (!P) { err = "params is NULL"; return false; }
    if (P->lattice != LBM_D2Q9 && P->lattice != LBM_D3Q19) { err = "lattice must be 9 (D2Q9) or 19 (D3Q19)"; return false; }
    if (P->precision != LBM_FP32 && P->precision != LBM_FP64 && P->precision != LBM_FP32_STORE_FP16) {
        err = "precision must be LBM_FP64, LBM_FP32 or LBM_FP32_STORE_FP16";
        return false;
    }
    if (P->nx < 1 || P->ny < 1 || P->nz < 1) { err = "grid sizes must be positive"; return false; }
    if (P->lattice == LBM_D2Q9 && P->nz != 1) { err = "D2Q9 needs nz == 1"; return false; }
    if (ng < 0) { err = "n_ghosts must be >= 0"; return false; }
    L.px = (int)round_up((size_t)P->nx, 4);
    L.nn_dense = (int64_t)P->nx * P->ny * P->nz;
    const int64_t nn = (int64_t)L.px * P->ny * P->nz;
    if (nn >= ((int64_t)1 << 31)) { err = "grid has 2^31 nodes or more"; return false; }
    L.nn = nn;
    L.plane = (int64_t)round_up((size_t)nn, 64);
    if ((int64_t)P->lattice * L.plane >= ((int64_t)1 << 31)) {
        err = "Q x nodes must stay below 2^31 (32-bit population indexing)";
        return false;
    }
    L.elem = P->precision == LBM_FP64 ? 8 : 4;
    L.pop_elem = P->precision == LBM_FP64 ? 8 : (P->precision == LBM_FP32 ? 4 : 2);
    L.rest_elem = P->precision == LBM_FP64 ? 8 : 4;
    L.Q = P->lattice;
    L.D = P->lattice == LBM_D2Q9 ? 2 : 3;
    L.GK = L.D == 2 ? 4 : 8;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = round_up(o + bytes, ALIGN); return r; };
    const size_t pop = (size_t)L.plane * (L.rest_elem + (size_t)(L.Q - 1) * L.pop_elem);
    L.pop_bytes = pop;
    for (int k = 0; k < 2; ++k) { L.off_N[k] = take(pop); L.off_B[k] = take(pop); }
    L.off_phi = take(L.plane * L.elem);
    for (int k = 0; k < 2; ++k) L.off_u[k] = take((size_t)L.D * L.plane * L.elem);
    L.off_p = take(L.plane * L.elem);
    L.off_cls = take(L.plane);
    L.off_mask = take(L.plane * 4);
    L.off_gnode = take((size_t)(ng + 1) * 4);
    L.off_gcorner = take((size_t)L.GK * (ng + 1) * 4);
    L.off_gwt = take((size_t)L.GK * (ng + 1) * L.elem);
    L.off_err = take(16);
    L.off_partial = take((size_t)DIAG_MAX_BLOCKS * DG_REC * 8);
    L.off_dout = take(DG_REC * 8);
    L.off_stage = take(2 * (size_t)L.plane * L.elem);   // two planes of field-typed values
    L.total = o;
    return true;
}

// Workspaces the library allocates come from one memory pool per device
// that keeps freed memory for the next domain (release threshold: all of
// it), so creating and destroying domains of similar sizes, as a serving loop
// does, costs no cudaMalloc / cudaFree: 0.5 ms and 1 ms for a 2.5 GB
// workspace.  lbm_release_cached_memory hands the cached memory back.
std::mutex g_pool_mutex;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t workspace_pool(int device) {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    auto it = g_pools.find(device);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;                                      // plain cudaMalloc then
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[device] = pool;
    return pool;
}

}  // namespace

struct lbm_domain {
    lbm_params prm;
    Layout lay;
    bool fp64 = false, contrast = false;
    char* ws = nullptr;
    bool own_ws = false;
    bool pooled_ws = false;            // own_ws from the device's workspace pool
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int64_t ng = 0, n_fallback = 0, n_fluid = 0;
    // node classes on the host as row bit masks: row r = y + ny z, W words of
    // 64 nodes each, bit x of fluid[r W + x / 64] (ghost[...]) set for a fluid
    // (ghost) node
    int row_words = 0;
    std::vector<uint64_t> fluid_bits, ghost_bits;
    bool is_fluid(int64_t node) const {          // dense node index
        const int64_t nx = prm.nx, r = node / nx, x = node - r * nx;
        return (fluid_bits[(size_t)(r * row_words + (x >> 6))] >> (x & 63)) & 1u;
    }
    std::vector<int32_t> h_corner;   // [GK][ng], dense node indices
    std::vector<int32_t> h_pcorner;  // [GK][ng], padded (device) node indices
    std::vector<int32_t> h_pnode;    // [ng], padded ghost nodes
    std::vector<double> h_wt;        // [GK][ng]
    std::vector<int32_t> h_nc;
    StepConfig cfg;
    int cur = 0;                     // buffers holding the current state
    int64_t step = 0;
    cudaGraphExec_t g1[2] = {nullptr, nullptr};
    cudaGraphExec_t g8 = nullptr;
    std::string err;
    // tiled TMA maps of phi and of both velocity buffers for the step kernel's
    // halo copies (FP32 arithmetic, rows of a multiple of 16 bytes)
    bool tma = false;
    CUtensorMap tm_phi{}, tm_u[2]{};
    bool tma2 = false;                     // the same with the two-node kernel's box
    CUtensorMap tm2_phi{}, tm2_u[2]{};
    // set once a bounded halo-copy wait gave up (LBM_ERR_TIMEOUT): a skipped
    // tile left the state wrong, so the domain takes no further steps
    bool poisoned = false;

    template <typename P> P* at(size_t off) const { return reinterpret_cast<P*>(ws + off); }
    void* N(int k) const { return at<void>(lay.off_N[k]); }
    void* B(int k) const { return at<void>(lay.off_B[k]); }
    void* U(int k) const { return at<void>(lay.off_u[k]); }
    void* phi() const { return at<void>(lay.off_phi); }
    void* p() const { return at<void>(lay.off_p); }
    uint8_t* cls() const { return at<uint8_t>(lay.off_cls); }
    uint32_t* mask() const { return at<uint32_t>(lay.off_mask); }
    int* errflag() const { return at<int>(lay.off_err); }
};

namespace {
// device index of grid node x + nx * (y + ny * z): x + px * (y + ny * z)

// Host threads for the per-domain set-up work (node classes, ghost
// weights).  Starting a thread costs tens of microseconds, as much as the
// work itself on a 192^3 grid, so the threads are started once, on first
// use, and sleep between calls.  The pool is never destroyed: its threads
// live as long as the process.  run() calls are serialised; the caller's
// thread works too, so a pool whose threads could not be started (or a
// forked child, which has none) still finishes every call.
class HostPool {
public:
    static HostPool& get() {
        // a forked child inherits none of the threads, and perhaps a mutex some
        // thread held at the fork: it gets a pool of its own
        static std::mutex make;
        static HostPool* pool = nullptr;
        static pid_t owner = 0;
        std::lock_guard<std::mutex> lk(make);
        if (!pool || owner != getpid()) {
            pool = new HostPool();
            owner = getpid();
        }
        return *pool;
    }
    int threads() const { return workers_ + 1; }
    // fn(i) for every i in [0, n), on the pool's threads and the caller's
    void run(int n, const std::function<void(int)>& fn) {
        std::lock_guard<std::mutex> one_call(call_);
        {
            std::lock_guard<std::mutex> lk(m_);
            fn_ = &fn;
            n_ = n;
            next_ = 0;
            done_ = 0;
            ++gen_;
        }
        wake_.notify_all();
        work();
        std::unique_lock<std::mutex> lk(m_);
        finished_.wait(lk, [&] { return done_ == n_; });
        fn_ = nullptr;
    }

private:
    HostPool() {
        const unsigned hw = std::thread::hardware_concurrency();
        const int want = std::min<int>(hw > 1 ? (int)hw - 1 : 0, 15);
        for (int t = 0; t < want; ++t) {
            try {
                std::thread(&HostPool::loop, this).detach();
                ++workers_;
            } catch (...) {
                break;
            }
        }
    }
    void work() {
        for (;;) {
            const std::function<void(int)>* fn;
            int i;
            {
                std::lock_guard<std::mutex> lk(m_);
                if (!fn_ || next_ >= n_) return;
                fn = fn_;
                i = next_++;
            }
            (*fn)(i);
            std::lock_guard<std::mutex> lk(m_);
            if (++done_ == n_) finished_.notify_all();
        }
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(m_);
                wake_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
            }
            work();
        }
    }
    std::mutex call_, m_;
    std::condition_variable wake_, finished_;
    const std::function<void(int)>* fn_ = nullptr;
    int n_ = 0, next_ = 0, done_ = 0, workers_ = 0;
    uint64_t gen_ = 0;
};

// The number of chunks for n items of at least min_chunk each, at most one
// per pool thread (and at most 16: the callers keep per-chunk counters).
int64_t chunk_count(int64_t n, int64_t min_chunk) {
    const int64_t k = std::min<int64_t>(HostPool::get().threads(), 16);
    return std::max<int64_t>(1, std::min<int64_t>(k, n / std::max<int64_t>(min_chunk, 1)));
}

// f(begin, end, chunk) over [0, n) in contiguous chunks of at least min_chunk
// items on the pool's threads; returns the number of chunks.
template <class F>
int parallel_chunks(int64_t n, int64_t min_chunk, F f) {
    const int64_t k = chunk_count(n, min_chunk);
    if (k == 1) {
        f((int64_t)0, n, 0);
        return 1;
    }
    HostPool::get().run((int)k, [&](int c) { f(n * c / k, n * (c + 1) / k, c); });
    return (int)k;
}

// f1 over the chunks of [0, n), then, once every f1 has returned, f2 over the
// same chunks.
template <class F1, class F2>
void parallel_phases(int64_t n, int64_t min_chunk, F1 f1, F2 f2) {
    const int64_t k = chunk_count(n, min_chunk);
    if (k == 1) {
        f1((int64_t)0, n, 0);
        f2((int64_t)0, n, 0);
        return;
    }
    HostPool::get().run((int)k, [&](int c) { f1(n * c / k, n * (c + 1) / k, c); });
    HostPool::get().run((int)k, [&](int c) { f2(n * c / k, n * (c + 1) / k, c); });
}

// Bit k of the result: byte k of v (little-endian order, as on every target
// here) is nonzero.  The shifts OR each byte's bits into its bit 0; the
// multiply moves bit 8k to bit 56 + k (the partial products fall on distinct
// bits, so nothing carries).
inline uint64_t nonzero_byte_bits(uint64_t v) {
    v |= v >> 4;
    v |= v >> 2;
    v |= v >> 1;
    return ((v & 0x0101010101010101ull) * 0x0102040810204080ull) >> 56;
}

// Node classes of a grid as row bit masks (see lbm_domain): a solid node with
// a fluid stencil neighbour (periodic wrap on every axis; a non-periodic axis
// has solid end layers, so its wrap finds no fluid) is a ghost.  The stencil
// of a row is the row itself shifted by +/-1 in x, the four rows next to it
// in y and z, shifted by -1, 0, +1 (axis and x-edge directions), and in 3D
// the four rows diagonal in (y, z) (the yz-edge directions).  Rows are split
// over host threads; n_solid and n_ghost count the grid's solid and ghost
// nodes.
void classify_rows(const lbm_params& P, const uint8_t* solid, int W, std::vector<uint64_t>& F,
                   std::vector<uint64_t>& G, int64_t& n_solid, int64_t& n_ghost) {
    const int64_t nx = P.nx, ny = P.ny, nz = P.nz, rows = ny * nz;
    const uint64_t last = (nx & 63) ? (1ull << (nx & 63)) - 1 : ~0ull;   // valid bits of a row's last word
    F.assign((size_t)(rows * W), 0);
    G.assign((size_t)(rows * W), 0);
    const bool three_d = P.lattice == LBM_D3Q19;
    std::vector<int64_t> solid_n(16, 0), ghost_n(16, 0);
    // at least ~1M nodes per chunk (measured: smaller chunks ran slower)
    const int64_t min_rows = std::max<int64_t>(1, ((int64_t)1 << 20) / nx);
    parallel_phases(rows, min_rows, [&](int64_t r0, int64_t r1, int) {
        for (int64_t r = r0; r < r1; ++r) {
            const uint8_t* row = solid + nx * r;
            uint64_t* f = &F[(size_t)(r * W)];
            int64_t x = 0;
            for (; x + 8 <= nx; x += 8) {
                uint64_t v;
                std::memcpy(&v, row + x, 8);
                f[x >> 6] |= nonzero_byte_bits(v) << (x & 63);
            }
            for (; x < nx; ++x) f[x >> 6] |= (uint64_t)(row[x] != 0) << (x & 63);
            for (int w = 0; w < W; ++w) f[w] = ~f[w];                       // solid -> fluid bits
            f[W - 1] &= last;
        }
    }, [&](int64_t r0, int64_t r1, int chunk) {
        std::vector<uint64_t> A(W), B(W);
        int64_t ns = 0, ng = 0;
        for (int64_t r = r0; r < r1; ++r) {
            const int64_t y = r % ny, z = r / ny;
            const int64_t ym = (y + ny - 1) % ny, yp = (y + 1) % ny, zm = (z + nz - 1) % nz, zp = (z + 1) % nz;
            const uint64_t* fr = &F[(size_t)(r * W)];
            auto row_of = [&](int64_t yy, int64_t zz) { return &F[(size_t)((yy + ny * zz) * W)]; };
            const uint64_t *fa = row_of(ym, z), *fb = row_of(yp, z);
            const uint64_t *fc = three_d ? row_of(y, zm) : fr, *fd = three_d ? row_of(y, zp) : fr;
            for (int w = 0; w < W; ++w) {
                A[w] = fa[w] | fb[w] | (three_d ? fc[w] | fd[w] : 0);
                B[w] = fr[w] | A[w];
            }
            // shifted copies of B: bit x <- bit x - 1 and bit x <- bit x + 1, periodic in x
            uint64_t carry = (B[(nx - 1) >> 6] >> ((nx - 1) & 63)) & 1u;
            uint64_t* g = &G[(size_t)(r * W)];
            for (int w = 0; w < W; ++w) {
                const uint64_t up = (B[w] << 1) | carry;
                carry = B[w] >> 63;
                const uint64_t down = (B[w] >> 1) | (w + 1 < W ? B[w + 1] << 63 : 0);
                uint64_t n = up | down | A[w];
                if (three_d) n |= row_of(ym, zm)[w] | row_of(yp, zm)[w] | row_of(ym, zp)[w] | row_of(yp, zp)[w];
                g[w] = ~fr[w] & n;
            }
            g[(nx - 1) >> 6] |= ~fr[(nx - 1) >> 6] & ((B[0] & 1u) << ((nx - 1) & 63));   // x = nx-1 sees x = 0
            g[W - 1] &= last;
            for (int w = 0; w < W; ++w) {
                ns += __builtin_popcountll(~fr[w] & (w == W - 1 ? last : ~0ull));
                ng += __builtin_popcountll(g[w]);
            }
        }
        solid_n[chunk] = ns;
        ghost_n[chunk] = ng;
    });
    n_solid = n_ghost = 0;
    for (int k = 0; k < 16; ++k) { n_solid += solid_n[k]; n_ghost += ghost_n[k]; }
}
}  // namespace

namespace {

lbm_status fail(lbm_domain* d, lbm_status s, const std::string& msg) {
    if (d) d->err = msg; else g_create_error = msg;
    return s;
}
}  // namespace

namespace lbmgpu {
int* domain_error_flag(lbm_domain* d) { return d->errflag(); }
cudaStream_t domain_stream(lbm_domain* d) { return d->stream; }
bool domain_poisoned(const lbm_domain* d) { return d->poisoned; }
int32_t* domain_ghost_corners(lbm_domain* d) { return d->at<int32_t>(d->lay.off_gcorner); }
int64_t domain_ghosts(const lbm_domain* d) { return d->ng; }
int64_t domain_plane(const lbm_domain* d) { return d->lay.plane; }
lbm_status domain_fail(lbm_domain* d, lbm_status s, const char* msg) { return fail(d, s, msg); }
}  // namespace lbmgpu

namespace {

#define CUDA_TRY(dom, call)                                                                        \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(dom, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

// Call f with a value of the Launch type of the domain's precision.
template <typename F>
void dispatch(const lbm_domain* d, F&& f) {
    switch (d->prm.precision) {
    case LBM_FP64: f(Launch<double, double>{}); break;
    case LBM_FP32: f(Launch<float, float>{}); break;
    default: f(Launch<float, __half>{}); break;
    }
}

// Lattice neighbour offsets of a stencil (excluding rest), for node classes.
void stencil_offsets(int Q, std::vector<int>& ox, std::vector<int>& oy, std::vector<int>& oz) {
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int m = std::abs(dx) + std::abs(dy) + std::abs(dz);
                if (m == 0) continue;
                if (Q == 9 && dz != 0) continue;
                if (Q == 19 && m > 2) continue;
                ox.push_back(dx); oy.push_back(dy); oz.push_back(dz);
            }
}

// Color weights chi (Appendix A / Eq. ChiTerm) and alpha from M_phi at p = 0.
void color_weights(int Q, double M_phi, double chi[19], double& alpha, double& c2chi) {
    const double cs2 = 1.0 / 3.0;
    const double w0 = Q == 9 ? 4.0 / 9.0 : 1.0 / 3.0;
    alpha = 1.0 - 2.0 * M_phi * (1.0 - w0) / cs2;
    for (int i = 0; i < 19; ++i) chi[i] = 0.0;
    chi[0] = alpha;
    for (int i = 1; i < Q; ++i) {
        if (Q == 9) {
            chi[i] = (i <= 4) ? (1.0 - alpha) / 5.0 : (1.0 - alpha) / 20.0;     // Eq. (ChiTerm)
        } else {
            chi[i] = (1.0 - alpha) * Lattice<19>::w(i) / (1.0 - w0);          // same rule in 3D
        }
    }
    c2chi = (1.0 - alpha) * cs2 / (1.0 - w0);
}

// f(k) for every fluid node k (dense index) of the domain, from the row bits
template <class F>
void for_fluid_nodes(const lbm_domain* d, F f) {
    const int64_t nx = d->prm.nx, rows = (int64_t)d->prm.ny * d->prm.nz;
    const int W = d->row_words;
    for (int64_t r = 0; r < rows; ++r)
        for (int w = 0; w < W; ++w) {
            uint64_t bits = d->fluid_bits[(size_t)(r * W + w)];
            while (bits) {
                const int b = __builtin_ctzll(bits);
                bits &= bits - 1;
                f(r * nx + 64 * w + b);
            }
        }
}

lbm_status prepare_ghosts(lbm_domain* d, const lbm_ghost* ghosts) {
    const lbm_params& P = d->prm;
    const int D = d->lay.D, GK = d->lay.GK, W = d->row_words;
    const int64_t ng = d->ng, nx = P.nx, ny = P.ny, px = d->lay.px;
    const int dims[3] = {P.nx, P.ny, P.nz};
    d->h_corner.assign((size_t)GK * ng, 0);
    d->h_pcorner.assign((size_t)GK * ng, 0);
    d->h_pnode.assign((size_t)ng, 0);
    d->h_wt.assign((size_t)GK * ng, 0.0);
    d->h_nc.assign(ng, 0);
    std::vector<int> ox, oy, oz;
    stencil_offsets(P.lattice, ox, oy, oz);
    auto fluid_at = [&](int64_t x, int64_t y, int64_t z) {
        return (d->fluid_bits[(size_t)((y + ny * z) * W + (x >> 6))] >> (x & 63)) & 1u;
    };
    // validation, in list order (the first bad entry is the one reported); a
    // listed ghost's bit is cleared in a copy of the ghost bits, which catches
    // a second listing of the same node
    std::vector<uint64_t> unlisted(d->ghost_bits);
    for (int64_t g = 0; g < ng; ++g) {
        const int64_t node = ghosts[g].node;
        bool ghost = false, listed = false;
        if (node >= 0 && node < d->lay.nn_dense) {
            const int64_t r = node / nx, x = node - r * nx;
            const size_t w = (size_t)(r * W + (x >> 6));
            ghost = (d->ghost_bits[w] >> (x & 63)) & 1u;
            listed = ghost && !((unlisted[w] >> (x & 63)) & 1u);
            unlisted[w] &= ~(1ull << (x & 63));
        }
        if (listed) return fail(nullptr, LBM_ERR_ARG, "node " + std::to_string(node) + " is listed twice");
        if (!ghost)
            return fail(nullptr, LBM_ERR_ARG, "ghost " + std::to_string(g) + " (node " + std::to_string(node) +
                                                  ") is not a solid node with a fluid neighbour");
        const double* n = ghosts[g].n;
        const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(std::fabs(len - 1.0) <= 1e-6))
            return fail(nullptr, LBM_ERR_ARG, "ghost " + std::to_string(g) + " normal is not a unit vector");
        if (D == 2 && n[2] != 0.0)
            return fail(nullptr, LBM_ERR_ARG, "ghost " + std::to_string(g) + " has a z normal on a 2D lattice");
    }

    // x_F = x_G + n_s, its cell corners and their bilinear/trilinear weights;
    // independent per ghost, so the list is split over host threads.  Node
    // indices are kept dense (lbm_ghost_table) and padded (the device).
    std::vector<int64_t> fallbacks(16, 0);
    parallel_chunks(ng, 2048, [&](int64_t g0, int64_t g1, int chunk) {
        int64_t n_fb = 0;
        for (int64_t g = g0; g < g1; ++g) {
            const int64_t node = ghosts[g].node;
            const double* n = ghosts[g].n;
            const int64_t xyz[3] = {node % nx, (node / nx) % ny, node / (nx * ny)};
            d->h_pnode[g] = (int32_t)(xyz[0] + px * (xyz[1] + ny * xyz[2]));
            double base[3] = {0, 0, 0}, frac[3] = {0, 0, 0};
            for (int a = 0; a < D; ++a) {
                const double xf = (double)xyz[a] + n[a];
                base[a] = std::floor(xf);
                frac[a] = xf - base[a];
            }
            int kept = 0;
            double wsum = 0.0;
            int64_t cidx[8], cpad[8];
            double cw[8];
            for (int k = 0; k < (1 << D); ++k) {
                int64_t c[3] = {0, 0, 0};
                double wk = 1.0;
                for (int a = 0; a < D; ++a) {
                    const int bit = (k >> a) & 1;
                    int64_t v = (int64_t)base[a] + bit;       // within one cell of the ghost: x - 1 .. x + 2
                    while (v < 0) v += dims[a];
                    while (v >= dims[a]) v -= dims[a];
                    c[a] = v;
                    wk *= bit ? frac[a] : 1.0 - frac[a];
                }
                if (fluid_at(c[0], c[1], c[2])) {
                    cidx[kept] = c[0] + nx * (c[1] + ny * c[2]);
                    cpad[kept] = c[0] + px * (c[1] + ny * c[2]);
                    cw[kept] = wk;
                    wsum += wk;
                    ++kept;
                }
            }
            if (kept > 0 && wsum > 0.0) {
                for (int k = 0; k < kept; ++k) cw[k] /= wsum;
            } else {
                // the fluid stencil neighbour most aligned with n_s; ties -> smaller node index
                int64_t best = -1, best_pad = -1;
                double best_dot = -INFINITY;
                for (size_t j = 0; j < ox.size(); ++j) {
                    int64_t c[3] = {xyz[0] + ox[j], xyz[1] + oy[j], xyz[2] + oz[j]};
                    for (int a = 0; a < 3; ++a) { c[a] %= dims[a]; if (c[a] < 0) c[a] += dims[a]; }
                    if (!fluid_at(c[0], c[1], c[2])) continue;
                    const int64_t cn = c[0] + nx * (c[1] + ny * c[2]);
                    const double dot = ox[j] * n[0] + oy[j] * n[1] + oz[j] * n[2];
                    if (dot > best_dot || (dot == best_dot && cn < best)) {
                        best_dot = dot;
                        best = cn;
                        best_pad = c[0] + px * (c[1] + ny * c[2]);
                    }
                }
                kept = 1;
                cidx[0] = best;
                cpad[0] = best_pad;
                cw[0] = 1.0;
                ++n_fb;
            }
            d->h_nc[g] = kept;
            for (int k = 0; k < GK; ++k) {
                d->h_corner[(size_t)k * ng + g] = (int32_t)(k < kept ? cidx[k] : cidx[0]);
                d->h_pcorner[(size_t)k * ng + g] = (int32_t)(k < kept ? cpad[k] : cpad[0]);
                d->h_wt[(size_t)k * ng + g] = k < kept ? cw[k] : 0.0;
            }
        }
        fallbacks[chunk] = n_fb;
    });
    for (int64_t f : fallbacks) d->n_fallback += f;
    return LBM_OK;
}

// ev: optional events {before ghost, before step, before phi, after phi}
void launch_one_step(lbm_domain* d, int cur, cudaStream_t s, cudaEvent_t* ev = nullptr) {
    const Layout& L = d->lay;
    if (ev) cudaEventRecord(ev[0], s);
    if (d->ng > 0) {
        const void* wt = d->at<void>(L.off_gwt);
        dispatch(d, [&](auto Lx) {
            decltype(Lx)::ghost(L.GK, d->cfg.ghost_rule, d->ng, d->at<int32_t>(L.off_gnode),
                                d->at<int32_t>(L.off_gcorner), wt, d->cfg.exp_eps, d->cfg.eps, d->phi(), L.plane,
                                d->errflag(), s);
        });
    }
    StepPtrs sp;
    sp.Nin = d->N(cur); sp.Bin = d->B(cur); sp.Nout = d->N(1 - cur); sp.Bout = d->B(1 - cur);
    sp.phi = d->phi(); sp.u_in = d->U(cur); sp.u_out = d->U(1 - cur); sp.p = d->p();
    sp.mask = d->mask(); sp.err = d->errflag();
    if (d->tma) { sp.tm_phi = &d->tm_phi; sp.tm_u = &d->tm_u[cur]; }
    if (d->tma2) { sp.tm2_phi = &d->tm2_phi; sp.tm2_u = &d->tm2_u[cur]; }
    if (ev) cudaEventRecord(ev[1], s);
    dispatch(d, [&](auto Lx) { decltype(Lx)::step(d->cfg, sp, s); });
    if (ev) cudaEventRecord(ev[2], s);
    dispatch(d, [&](auto Lx) { decltype(Lx)::phi(d->cfg, d->B(1 - cur), d->mask(), d->phi(), d->errflag(), s); });
    if (ev) cudaEventRecord(ev[3], s);
}

lbm_status capture(lbm_domain* d, int start, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CUDA_TRY(d, cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal));
    int c = start;
    for (int k = 0; k < nsteps; ++k) { launch_one_step(d, c, d->cap); c ^= 1; }
    cudaError_t e = cudaStreamEndCapture(d->cap, &g);
    if (e != cudaSuccess) return fail(d, LBM_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(d, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return LBM_OK;
}

// cuTensorMapEncodeTiled from the driver, through the runtime (no link to libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            f = nullptr;
        cudaGetLastError();
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor maps for the halo copies of the step kernel: phi as (nx, ny, nz) and
// each velocity buffer as (nx, ny, nz, D) floats, box = the halo tile of
// Tile<Q, V>; out[0] = phi, out[1 + k] = velocity buffer k.  Only for float
// fields whose rows are a multiple of 16 bytes (the strides TMA accepts);
// otherwise, or if the driver refuses, the kernel copies every halo element
// itself.
template <class Tl>
bool encode_halo_maps_tile(const lbm_domain* d, CUtensorMap out[3]) {
    const lbm_params& P = d->prm;
    if (d->fp64) return false;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const int D = Tl::D;
    const cuuint64_t dims[4] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, (cuuint64_t)P.nz, (cuuint64_t)D};
    const cuuint64_t strides[3] = {(cuuint64_t)d->lay.px * 4, (cuuint64_t)d->lay.px * P.ny * 4,
                                   (cuuint64_t)d->lay.plane * 4};
    const cuuint32_t box[4] = {(cuuint32_t)Tl::HX, (cuuint32_t)Tl::HY, (cuuint32_t)Tl::HZ, (cuuint32_t)D};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    auto one = [&](CUtensorMap* m, void* base, cuuint32_t rank) {
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return one(&out[0], d->phi(), 3) && one(&out[1], d->U(0), 4) && one(&out[2], d->U(1), 4);
}

template <int Q, int V>
bool encode_halo_maps(const lbm_domain* d, CUtensorMap out[3]) {
    return encode_halo_maps_tile<Tile<Q, V>>(d, out);
}

template <int Q>
bool make_pair_maps(lbm_domain* d) {
    CUtensorMap m[3];
    if (!encode_halo_maps_tile<PairTile<Q>>(d, m)) return false;
    d->tm2_phi = m[0];
    d->tm2_u[0] = m[1];
    d->tm2_u[1] = m[2];
    return true;
}

template <int Q>
bool make_halo_maps(lbm_domain* d) {
    CUtensorMap m[3];
    if (!encode_halo_maps<Q, 0>(d, m)) return false;
    d->tm_phi = m[0];
    d->tm_u[0] = m[1];
    d->tm_u[1] = m[2];
    return true;
}

// The maps of tile shape V for a domain of lattice Q (the batch's tables).
bool encode_halo_maps_any(const lbm_domain* d, int V, CUtensorMap out[3]) {
    if (d->prm.lattice == 9) {
        switch (V) {
        case 0: return encode_halo_maps<9, 0>(d, out);
        case 1: return encode_halo_maps<9, 1>(d, out);
        case 2: return encode_halo_maps<9, 2>(d, out);
        case 3: return encode_halo_maps<9, 3>(d, out);
        case 4: return encode_halo_maps<9, 4>(d, out);
        default: return encode_halo_maps<9, 5>(d, out);
        }
    }
    switch (V) {
    case 0: return encode_halo_maps<19, 0>(d, out);
    case 1: return encode_halo_maps<19, 1>(d, out);
    case 2: return encode_halo_maps<19, 2>(d, out);
    case 3: return encode_halo_maps<19, 3>(d, out);
    case 4: return encode_halo_maps<19, 4>(d, out);
    default: return encode_halo_maps<19, 5>(d, out);
    }
}

const char* const kPoisonedMsg =
    "a bounded halo-copy wait gave up earlier (LBM_ERR_TIMEOUT); the domain's state is not valid: destroy it";

lbm_status check_err_flag(lbm_domain* d) {
    int h = 0;
    CUDA_TRY(d, cudaMemcpyAsync(&h, d->errflag(), sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(d, cudaStreamSynchronize(d->stream));
    if (h & kErrCopyTimeout) {
        d->poisoned = true;
        return fail(d, LBM_ERR_TIMEOUT, "a halo copy of the step kernel did not complete");
    }
    if (h & kErrBounds)
        return fail(d, LBM_ERR_BOUNDS, "a step kernel computed an index outside its array (access skipped)");
    if (h) return fail(d, LBM_ERR_UNSTABLE, "a step produced a non-finite velocity");
    return LBM_OK;
}

// host double <-> device T conversions through a staging vector
// One whole field between a dense host array of doubles (nx * ny * nz values)
// and the device (field type, rows padded to px; the padding holds zeros).
template <typename V>
lbm_status upload_as(lbm_domain* d, void* dst, const double* src) {
    const Layout& L = d->lay;
    const int64_t nx = d->prm.nx, rows = L.nn_dense / nx;
    std::vector<V> tmp((size_t)L.nn, V(0));
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t x = 0; x < nx; ++x) tmp[(size_t)(r * L.px + x)] = (V)src[r * nx + x];
    CUDA_TRY(d, cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(V), cudaMemcpyHostToDevice, d->stream));
    CUDA_TRY(d, cudaStreamSynchronize(d->stream));
    return LBM_OK;
}

template <typename V>
lbm_status download_as(lbm_domain* d, double* dst, const void* src) {
    const Layout& L = d->lay;
    const int64_t nx = d->prm.nx, rows = L.nn_dense / nx;
    std::vector<V> tmp((size_t)L.nn);
    CUDA_TRY(d, cudaMemcpyAsync(tmp.data(), src, tmp.size() * sizeof(V), cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(d, cudaStreamSynchronize(d->stream));
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t x = 0; x < nx; ++x) dst[r * nx + x] = (double)tmp[(size_t)(r * L.px + x)];
    return LBM_OK;
}

// count must be the grid's node count: whole fields only
lbm_status upload(lbm_domain* d, void* dst, const double* src, size_t count) {
    if ((int64_t)count != d->lay.nn_dense) return fail(d, LBM_ERR_ARG, "field size mismatch");
    return d->fp64 ? upload_as<double>(d, dst, src) : upload_as<float>(d, dst, src);
}

lbm_status download(lbm_domain* d, double* dst, const void* src, size_t count) {
    if ((int64_t)count != d->lay.nn_dense) return fail(d, LBM_ERR_ARG, "field size mismatch");
    return d->fp64 ? download_as<double>(d, dst, src) : download_as<float>(d, dst, src);
}

lbm_status init_state(lbm_domain* d, int mode, const double ctr[3], double R0) {
    const double ghost_value = 0.5 * (1.0 + std::cos(d->prm.theta));
    d->cur = 0;
    d->step = 0;
    const Layout& L = d->lay;
    // What a step reads is set here: the populations of the fluid nodes
    // (init_pops) and the velocity of the first step's stencil, 0.  Population
    // slots of non-fluid nodes are never read (every pull of a fluid node reads
    // a fluid source or the node's own slots, as the diagnostics and state
    // transfer do), the second velocity buffer is written at every fluid node
    // by the first step, and the velocity of non-fluid nodes stays 0 from the
    // domain's creation (no kernel writes it but as 0).  So of the state only
    // the first velocity buffer and p (state read back as 0 before a step) are
    // cleared.
    CUDA_TRY(d, cudaMemsetAsync(d->errflag(), 0, sizeof(int), d->stream));
    CUDA_TRY(d, cudaMemsetAsync(d->U(0), 0, (size_t)L.D * L.plane * L.elem, d->stream));
    CUDA_TRY(d, cudaMemsetAsync(d->p(), 0, (size_t)L.plane * L.elem, d->stream));
    dispatch(d, [&](auto Lx) {
        decltype(Lx)::init_phi(d->cfg, d->cls(), d->phi(), mode, ctr, R0, ghost_value, d->stream);
        decltype(Lx)::init_pops(d->cfg, d->cls(), d->phi(), d->N(0), d->B(0), d->stream);
    });
    CUDA_TRY(d, cudaGetLastError());
    return LBM_OK;
}

// Solve the (n x n) system A z = b, n <= 4, by Gaussian elimination with partial pivoting.
bool solve_dense(int n, double A[4][4], double b[4], double z[4]) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return false;
        if (piv != c) {
            for (int j = 0; j < n; ++j) std::swap(A[c][j], A[piv][j]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int j = c; j < n; ++j) A[r][j] -= f * A[c][j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r][j] * z[j];
        z[r] = s / A[r][r];
    }
    return true;
}

}  // namespace

extern "C" {

size_t lbm_domain_bytes(const lbm_params* params, int64_t n_ghosts) {
    Layout L;
    std::string err;
    if (!make_layout(params, n_ghosts, L, err)) return 0;
    return L.total;
}

lbm_status lbm_create_domain(const lbm_params* params, const uint8_t* solid, const lbm_ghost* ghosts,
                             int64_t n_ghosts, void* dev_workspace, size_t ws_bytes, void* cuda_stream,
                             lbm_domain** out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    Layout L;
    std::string err;
    if (!make_layout(params, n_ghosts, L, err)) return fail(nullptr, LBM_ERR_ARG, err);
    const lbm_params& P = *params;
    if (!solid) return fail(nullptr, LBM_ERR_ARG, "solid mask is NULL");
    if (n_ghosts > 0 && !ghosts) return fail(nullptr, LBM_ERR_ARG, "ghost list is NULL");
    if (!(P.W >= 4.0)) return fail(nullptr, LBM_ERR_ARG, "W must be >= 4 lattice units");
    if (P.ghost_rule != LBM_GHOST_PRESENT && P.ghost_rule != LBM_GHOST_FAKHARI)
        return fail(nullptr, LBM_ERR_ARG, "ghost_rule must be LBM_GHOST_PRESENT or LBM_GHOST_FAKHARI");
    if (P.reserved != 0) return fail(nullptr, LBM_ERR_ARG, "reserved field of lbm_params must be 0");
    if (!(P.rho_l > 0 && P.rho_g > 0 && P.mu_l > 0 && P.mu_g > 0))
        return fail(nullptr, LBM_ERR_ARG, "densities and viscosities must be positive");
    if (!(P.sigma >= 0)) return fail(nullptr, LBM_ERR_ARG, "sigma must be >= 0");
    if (!std::isfinite(P.theta) || !std::isfinite(P.g[0]) || !std::isfinite(P.g[1]) || !std::isfinite(P.g[2]))
        return fail(nullptr, LBM_ERR_ARG, "theta and g must be finite");

    lbm_domain* d = new lbm_domain();
    d->prm = P;
    d->lay = L;
    d->fp64 = P.precision == LBM_FP64;
    d->contrast = P.rho_l != P.rho_g;
    d->ng = n_ghosts;
    d->stream = (cudaStream_t)cuda_stream;

    double alpha, c2chi;
    StepConfig& c = d->cfg;
    color_weights(P.lattice, P.M_phi, c.chi, alpha, c2chi);
    if (!(alpha > 0.0 && alpha < 1.0)) { delete d; return fail(nullptr, LBM_ERR_ARG, "M_phi gives alpha outside (0,1)"); }
    c.Q = P.lattice;
    c.contrast = d->contrast;
    c.d = Dims{P.nx, P.ny, P.nz, L.px, L.plane, P.periodic};
    c.rho_l = P.rho_l; c.rho_g = P.rho_g;
    c.nu_l = P.mu_l / P.rho_l; c.nu_g = P.mu_g / P.rho_g;
    c.sigma = P.sigma; c.W = P.W;
    for (int a = 0; a < 3; ++a) c.g[a] = (L.D == 2 && a == 2) ? 0.0 : P.g[a];
    c.c2chi = c2chi;
    c.eps = -(4.0 / P.W) * std::cos(P.theta);
    c.exp_eps = std::exp(c.eps);
    c.ghost_rule = P.ghost_rule;
    // Float arithmetic: the two-node step kernel (half the load/store and
    // address instructions per node of the one-node kernel; at 192^3 0.967
    // against 0.919 of the measured copy peak with FP32 storage, 0.667 against
    // 0.658 of its roofline with FP16 storage).  LBM_STEP_KERNEL=pair|single
    // overrides; both kernels give the same results to the bit.
    const char* step_kernel = std::getenv("LBM_STEP_KERNEL");
    c.pair = P.precision != LBM_FP64 && (step_kernel == nullptr || std::strcmp(step_kernel, "pair") == 0);

    // node classes, as row bit masks on the host (the device expands them)
    const int64_t nn = L.nn_dense;
    const int64_t nx = P.nx, ny = P.ny, nz = P.nz;
    d->row_words = (int)((nx + 63) / 64);
    int64_t n_cls_ghost = 0, n_solid = 0;
    classify_rows(P, solid, d->row_words, d->fluid_bits, d->ghost_bits, n_solid, n_cls_ghost);
    d->n_fluid = nn - n_solid;
    // a non-periodic axis needs solid end layers (the two layers of that axis only)
    for (int a = 0; a < L.D; ++a) {
        if (P.periodic & (1u << a)) continue;
        const int64_t ext[3] = {nx, ny, nz};
        bool fluid_end = false;
        for (int64_t z = 0; z < nz && !fluid_end; ++z)
            for (int64_t y = 0; y < ny && !fluid_end; ++y) {
                if (a == 0) {
                    fluid_end = !solid[nx * (y + ny * z)] || !solid[nx - 1 + nx * (y + ny * z)];
                } else if ((a == 1 && (y == 0 || y == ext[1] - 1)) || (a == 2 && (z == 0 || z == ext[2] - 1))) {
                    const uint8_t* row = solid + nx * (y + ny * z);
                    for (int64_t x = 0; x < nx; ++x)
                        if (!row[x]) { fluid_end = true; break; }
                }
            }
        if (fluid_end) {
            delete d;
            return fail(nullptr, LBM_ERR_ARG, "axis " + std::to_string(a) + " is not periodic but has fluid on an end layer");
        }
    }
    if (n_cls_ghost != n_ghosts) {
        delete d;
        return fail(nullptr, LBM_ERR_ARG, "ghost list has " + std::to_string(n_ghosts) + " entries, mask has " +
                                              std::to_string(n_cls_ghost) + " ghost nodes");
    }
    lbm_status st = prepare_ghosts(d, ghosts);
    if (st != LBM_OK) { delete d; return st; }

    // device memory
    if (dev_workspace) {
        if (ws_bytes < L.total) {
            delete d;
            return fail(nullptr, LBM_ERR_OOM, "workspace of " + std::to_string(ws_bytes) + " bytes, need " + std::to_string(L.total));
        }
        if (reinterpret_cast<uintptr_t>(dev_workspace) % ALIGN) {
            delete d;
            return fail(nullptr, LBM_ERR_ARG, "workspace must be 256-byte aligned");
        }
        d->ws = (char*)dev_workspace;
    } else {
        void* p = nullptr;
        cudaGetDevice(&d->device);
        cudaMemPool_t pool = workspace_pool(d->device);
        cudaError_t e = cudaErrorMemoryAllocation;
        if (pool) {
            e = cudaMallocFromPoolAsync(&p, L.total, pool, d->stream);
            if (e != cudaSuccess) {
                // the pool's cached blocks may not fit: give them back, try once more
                cudaGetLastError();
                cudaDeviceSynchronize();
                cudaMemPoolTrimTo(pool, 0);
                e = cudaMallocFromPoolAsync(&p, L.total, pool, d->stream);
            }
            d->pooled_ws = e == cudaSuccess;
        }
        if (e == cudaSuccess && reinterpret_cast<uintptr_t>(p) % ALIGN) {   // the layout's alignment
            cudaFreeAsync(p, d->stream);
            cudaStreamSynchronize(d->stream);
            d->pooled_ws = false;
            e = cudaErrorMemoryAllocation;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&p, L.total);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete d;
            return fail(nullptr, LBM_ERR_OOM, "allocation of " + std::to_string(L.total) + " bytes failed");
        }
        d->ws = (char*)p;
        d->own_ws = true;
    }
    auto bail = [&](const std::string& m) {
        std::string msg = m;
        lbm_destroy(d);
        return fail(nullptr, LBM_ERR_CUDA, msg);
    };
    if (cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking) != cudaSuccess) return bail("cudaStreamCreate failed");
    // LBM_HALO_COPY=elements: every tile copies its halo element by element
    // (the reference the tiled copies are tested against)
    const char* halo_copy = std::getenv("LBM_HALO_COPY");
    const bool elements_only = halo_copy && std::strcmp(halo_copy, "elements") == 0;
    d->tma = !elements_only && (P.lattice == 9 ? make_halo_maps<9>(d) : make_halo_maps<19>(d));
    d->tma2 = !elements_only && (P.lattice == 9 ? make_pair_maps<9>(d) : make_pair_maps<19>(d));
    // upload the row bit masks (into the staging planes, 2 W bytes per row
    // against their 8 px) and the ghost table; the node classes and the
    // bounce-back mask are built from them on the device, with the padded row
    // pitch of the device fields
    cudaStream_t s = d->stream;
    const size_t bits_bytes = d->fluid_bits.size() * sizeof(uint64_t);
    uint64_t* dF = d->at<uint64_t>(L.off_stage);
    uint64_t* dG = dF + d->fluid_bits.size();
    if (2 * bits_bytes > 2 * (size_t)L.plane * L.elem) return bail("row bit masks do not fit the staging planes");
    // zero the fields from phi on (u must stay 0 at non-fluid nodes); the
    // population buffers are left as they are: lbm_init_* writes every fluid
    // node's slots of the first ones, the first step those of the second ones,
    // and no pull of a fluid node reads a non-fluid node's slots (the step
    // kernels load them for non-fluid lanes, whose results are never stored
    // as state: u and p get 0 there, the populations values nothing reads)
    if (cudaMemsetAsync(d->ws + L.off_phi, 0, L.total - L.off_phi, s) != cudaSuccess)
        return bail("cudaMemset failed");
    if (cudaMemcpyAsync(dF, d->fluid_bits.data(), bits_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dG, d->ghost_bits.data(), bits_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail("upload of node classes failed");
    dispatch(d, [&](auto Lx) {
        decltype(Lx)::expand_classes(d->cfg, d->row_words, dF, dG, d->cls(), s);
        decltype(Lx)::build_mask(d->cfg, d->cls(), d->mask(), s);
    });
    if (cudaGetLastError() != cudaSuccess) return bail("launch of the class and mask kernels failed");
    const std::vector<int32_t>& gnode = d->h_pnode;
    const std::vector<int32_t>& pcorner = d->h_pcorner;
    if (n_ghosts > 0) {
        if (cudaMemcpyAsync(d->at<void>(L.off_gnode), gnode.data(), n_ghosts * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d->at<void>(L.off_gcorner), pcorner.data(), pcorner.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return bail("upload of the ghost table failed");
        if (d->fp64) {
            if (cudaMemcpyAsync(d->at<void>(L.off_gwt), d->h_wt.data(), d->h_wt.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return bail("upload of the ghost weights failed");
        } else {
            std::vector<float> wf(d->h_wt.begin(), d->h_wt.end());
            if (cudaMemcpyAsync(d->at<void>(L.off_gwt), wf.data(), wf.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return bail("upload of the ghost weights failed");
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail("synchronisation after upload failed");
    if (capture(d, 0, 1, &d->g1[0]) != LBM_OK || capture(d, 1, 1, &d->g1[1]) != LBM_OK ||
        capture(d, 0, GRAPH_STEPS, &d->g8) != LBM_OK)
        return bail("CUDA graph capture of the step failed: " + d->err);
    *out = d;
    return LBM_OK;
}

lbm_status lbm_init_droplet(lbm_domain* d, const double centre[3], double R0) {
    if (!d || !centre) return fail(d, LBM_ERR_ARG, "NULL argument");
    if (d->poisoned) return fail(d, LBM_ERR_TIMEOUT, kPoisonedMsg);
    if (!(R0 > 0) || !std::isfinite(centre[0]) || !std::isfinite(centre[1]) || !std::isfinite(centre[2]))
        return fail(d, LBM_ERR_ARG, "drop radius must be positive and the centre finite");
    return init_state(d, 0, centre, R0);
}

lbm_status lbm_init_phi(lbm_domain* d, const double* phi_host) {
    if (!d || !phi_host) return fail(d, LBM_ERR_ARG, "NULL argument");
    if (d->poisoned) return fail(d, LBM_ERR_TIMEOUT, kPoisonedMsg);
    lbm_status st = upload(d, d->phi(), phi_host, d->lay.nn_dense);
    if (st != LBM_OK) return st;
    const double zero[3] = {0, 0, 0};
    return init_state(d, 1, zero, 1.0);
}

lbm_status lbm_step(lbm_domain* d, int64_t n) {
    if (!d) return fail(d, LBM_ERR_ARG, "NULL domain");
    if (n < 0) return fail(d, LBM_ERR_ARG, "n must be >= 0");
    if (d->poisoned) return fail(d, LBM_ERR_TIMEOUT, kPoisonedMsg);
    while (n > 0) {
        if (d->cur == 0 && n >= GRAPH_STEPS) {
            CUDA_TRY(d, cudaGraphLaunch(d->g8, d->stream));
            n -= GRAPH_STEPS;
            d->step += GRAPH_STEPS;
        } else {
            CUDA_TRY(d, cudaGraphLaunch(d->g1[d->cur], d->stream));
            d->cur ^= 1;
            --n;
            d->step += 1;
        }
    }
    return LBM_OK;
}

lbm_status lbm_profile_steps(lbm_domain* d, int64_t n, double kernel_ms[3]) {
    if (!d || !kernel_ms) return fail(d, LBM_ERR_ARG, "NULL argument");
    if (n < 1) return fail(d, LBM_ERR_ARG, "n must be >= 1");
    if (d->poisoned) return fail(d, LBM_ERR_TIMEOUT, kPoisonedMsg);
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) CUDA_TRY(d, cudaEventCreate(&ev[k]));
    lbm_status st = LBM_OK;
    for (int64_t t = 0; t < n && st == LBM_OK; ++t) {
        launch_one_step(d, d->cur, d->stream, ev);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        if (e != cudaSuccess) { st = fail(d, LBM_ERR_CUDA, std::string("profiled step: ") + cudaGetErrorString(e)); break; }
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            kernel_ms[k] += ms;
        }
        d->cur ^= 1;
        d->step += 1;
    }
    for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
    return st;
}

lbm_status lbm_sync(lbm_domain* d) {
    if (!d) return fail(d, LBM_ERR_ARG, "NULL domain");
    CUDA_TRY(d, cudaStreamSynchronize(d->stream));
    return check_err_flag(d);
}

lbm_status lbm_diagnostics(lbm_domain* d, const lbm_probe* probe, lbm_diag* out) {
    if (!d || !out) return fail(d, LBM_ERR_ARG, "NULL argument");
    const Layout& L = d->lay;
    ProbeDev pr{};
    pr.kind = 0;
    if (probe) {
        if (probe->kind < 0 || probe->kind > 2) return fail(d, LBM_ERR_ARG, "probe kind must be 0, 1 or 2");
        pr.kind = probe->kind;
        for (int a = 0; a < 3; ++a) { pr.center[a] = probe->center[a]; pr.normal[a] = probe->normal[a]; }
        pr.radius = probe->radius;
        pr.exclude = probe->exclude;
    }
    double* partial = d->at<double>(L.off_partial);
    double* dout = d->at<double>(L.off_dout);
    dispatch(d, [&](auto Lx) {
        decltype(Lx)::diag(d->cfg, d->mask(), d->N(d->cur), d->phi(), d->U(d->cur), d->p(), pr, partial, dout,
                           d->stream);
    });
    CUDA_TRY(d, cudaGetLastError());
    double h[DG_REC];
    CUDA_TRY(d, cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, d->stream));
    CUDA_TRY(d, cudaStreamSynchronize(d->stream));
    std::memset(out, 0, sizeof(*out));
    const lbm_params& P = d->prm;
    out->phi_sum = h[DG_PHI];
    out->n_fluid = (int64_t)h[DG_NFLUID];
    out->mass_liquid = P.rho_l * h[DG_PHI];
    out->mass_gas = P.rho_g * (h[DG_NFLUID] - h[DG_PHI]);
    out->pop_sum = h[DG_POP];
    out->max_u = std::sqrt(h[DG_MAXU2]);
    out->n_in = (int64_t)h[DG_NIN];
    out->n_out = (int64_t)h[DG_NOUT];
    out->p_in = out->n_in ? h[DG_PIN] / h[DG_NIN] : 0.0;
    out->p_out = out->n_out ? h[DG_POUT] / h[DG_NOUT] : 0.0;
    out->n_iface = (int64_t)h[DG_NIFACE];
    out->n_fit = (int64_t)h[DG_NFIT];
    out->step = d->step;
    out->nan_flag = h[DG_NAN] > 0 ? 1 : 0;
    out->contact_angle = NAN;
    out->apex = NAN;
    if (pr.kind != 0) {
        out->apex = h[DG_APEX];
        const int D = L.D;
        double A[4][4], b[4], z[4] = {0, 0, 0, 0};
        for (int i = 0; i <= D; ++i) {
            for (int j = 0; j <= D; ++j) A[i][j] = h[DG_A + 4 * i + j];
            b[i] = h[DG_B + i];
        }
        if (out->n_fit >= D + 2 && solve_dense(D + 1, A, b, z)) {
            double c2 = 0.0, hn = 0.0;
            for (int k = 0; k < D; ++k) {
                const double ck = -z[k] / 2.0;
                out->fit_center[k] = ck + pr.center[k];
                c2 += ck * ck;
                hn += ck * pr.normal[k];
            }
            out->fit_radius = std::sqrt(c2 - z[D]);
            const double r = out->fit_radius;
            if (pr.kind == 1) {
                const double R = pr.radius;
                out->contact_angle = std::acos((R * R + r * r - c2) / (2.0 * R * r));
            } else {
                out->contact_angle = std::acos(-hn / r);
            }
        }
    }
    lbm_status st = check_err_flag(d);
    if (out->nan_flag && st == LBM_OK) return fail(d, LBM_ERR_UNSTABLE, "non-finite color or velocity in the state");
    return st;
}

lbm_status lbm_read_state(lbm_domain* d, int32_t field, double* host_out) {
    if (!d || !host_out) return fail(d, LBM_ERR_ARG, "NULL argument");
    const Layout& L = d->lay;
    const int64_t nn = L.nn_dense;
    std::vector<double> tmp;
    switch (field) {
    case LBM_FIELD_N:
    case LBM_FIELD_B: {
        const bool is_b = field == LBM_FIELD_B;
        void* st = is_b ? d->B(d->cur) : d->N(d->cur);
        void* stage = d->at<void>(L.off_stage);
        for (int i = 0; i < L.Q; ++i) {
            double base = 0.0;
            dispatch(d, [&](auto Lx) {
                decltype(Lx)::gather_dir(d->cfg, d->cls(), i, is_b, st, stage, d->stream);
                base = decltype(Lx)::storage_base(d->cfg, i, is_b);
            });
            CUDA_TRY(d, cudaGetLastError());
            double* out = host_out + (size_t)i * nn;
            lbm_status s = download(d, out, stage, nn);
            if (s != LBM_OK) return s;
            if (base != 0.0)                       // deviations from the storage reference -> values, in double
                for_fluid_nodes(d, [&](int64_t k) { out[k] += base; });
        }
        return LBM_OK;
    }
    case LBM_FIELD_PHI:
        return download(d, host_out, d->phi(), nn);
    case LBM_FIELD_U: {
        for (int a = 0; a < 3; ++a) {
            if (a < L.D) {
                lbm_status s = download(d, host_out + (size_t)a * nn, (const char*)d->U(d->cur) + (size_t)a * L.plane * L.elem, nn);
                if (s != LBM_OK) return s;
            } else {
                std::fill(host_out + (size_t)a * nn, host_out + (size_t)(a + 1) * nn, 0.0);
            }
        }
        return LBM_OK;
    }
    case LBM_FIELD_P:
        return download(d, host_out, d->p(), nn);
    }
    return fail(d, LBM_ERR_ARG, "unknown field");
}

lbm_status lbm_write_state(lbm_domain* d, int32_t field, const double* host_in) {
    if (!d || !host_in) return fail(d, LBM_ERR_ARG, "NULL argument");
    if (d->poisoned) return fail(d, LBM_ERR_TIMEOUT, kPoisonedMsg);
    const Layout& L = d->lay;
    const int64_t nn = L.nn_dense;
    switch (field) {
    case LBM_FIELD_N:
    case LBM_FIELD_B: {
        const bool is_b = field == LBM_FIELD_B;
        void* st = is_b ? d->B(d->cur) : d->N(d->cur);
        char* stage = d->at<char>(L.off_stage);
        std::vector<double> dev_i((size_t)nn), dev_o((size_t)nn);
        for (int i = 0; i < L.Q; ++i) {
            const int o = d->prm.lattice == 9 ? Lattice<9>::opp(i) : Lattice<19>::opp(i);
            double base = 0.0;                     // the same for i and its opposite (chi is even in c)
            dispatch(d, [&](auto Lx) { base = decltype(Lx)::storage_base(d->cfg, i, is_b); });
            // values -> deviations from the storage reference, in double
            for (int64_t k = 0; k < nn; ++k) {
                dev_i[k] = host_in[(size_t)i * nn + k] - base;
                dev_o[k] = host_in[(size_t)o * nn + k] - base;
            }
            lbm_status s = upload(d, stage, dev_i.data(), nn);
            if (s == LBM_OK) s = upload(d, stage + (size_t)L.plane * L.elem, dev_o.data(), nn);
            if (s != LBM_OK) return s;
            dispatch(d, [&](auto Lx) {
                decltype(Lx)::scatter_dir(d->cfg, d->cls(), i, is_b, stage, stage + (size_t)L.plane * L.elem, st,
                                          d->stream);
            });
            CUDA_TRY(d, cudaGetLastError());
        }
        CUDA_TRY(d, cudaStreamSynchronize(d->stream));
        return LBM_OK;
    }
    case LBM_FIELD_PHI:
        return upload(d, d->phi(), host_in, nn);
    case LBM_FIELD_U: {
        // the velocity of a non-fluid node is 0 whatever the caller passes: the
        // stencils read it there as the wall's velocity
        std::vector<double> ua((size_t)nn);
        for (int a = 0; a < L.D; ++a) {
            const double* src = host_in + (size_t)a * nn;
            std::fill(ua.begin(), ua.end(), 0.0);
            for_fluid_nodes(d, [&](int64_t k) { ua[k] = src[k]; });
            lbm_status s = upload(d, (char*)d->U(d->cur) + (size_t)a * L.plane * L.elem, ua.data(), nn);
            if (s != LBM_OK) return s;
        }
        return LBM_OK;
    }
    case LBM_FIELD_P:
        return upload(d, d->p(), host_in, nn);
    }
    return fail(d, LBM_ERR_ARG, "unknown field");
}

lbm_status lbm_ghost_table(lbm_domain* d, int64_t* corner, double* weight, int32_t* n_corner) {
    if (!d || !corner || !weight || !n_corner) return fail(d, LBM_ERR_ARG, "NULL argument");
    const int GK = d->lay.GK;
    for (int64_t g = 0; g < d->ng; ++g) {
        n_corner[g] = d->h_nc[g];
        for (int k = 0; k < GK; ++k) {
            corner[g * GK + k] = d->h_corner[(size_t)k * d->ng + g];
            weight[g * GK + k] = d->h_wt[(size_t)k * d->ng + g];
        }
    }
    return LBM_OK;
}

int64_t lbm_ghost_fallbacks(const lbm_domain* d) { return d ? d->n_fallback : 0; }

int32_t lbm_launches_per_step(const lbm_domain* d) { return d ? (d->ng > 0 ? 3 : 2) : 0; }

double lbm_bytes_per_fluid_node(const lbm_domain* d) {
    if (!d) return 0.0;
    const double s = (double)d->lay.elem;
    const double moving = (d->lay.Q - 1) * (double)d->lay.pop_elem;
    const double pop = (double)d->lay.rest_elem + moving;   // per node and array
    // k_step pulls N: the FP64 update follows the literal collision and reads the
    // rest population, the float updates take every moment from the moving ones
    const double pull = d->lay.elem == 8 ? pop : moving;
    const int D = d->lay.D;
    // N* and B* written, B* pulled by k_phi; phi written (k_phi) and read (k_step);
    // u written, and read when the density contrast makes F_visc active; p written; the 4-byte
    // bounce-back mask read by k_step and k_phi
    return pull + 3.0 * pop + 2.0 * s + (d->contrast ? 2.0 : 1.0) * D * s + s + 8.0;
}

int64_t lbm_fluid_nodes(const lbm_domain* d) { return d ? d->n_fluid : 0; }

const char* lbm_last_error(const lbm_domain* d) { return d ? d->err.c_str() : g_create_error.c_str(); }

void lbm_destroy(lbm_domain* d) {
    if (!d) return;
    if (d->g8) cudaGraphExecDestroy(d->g8);
    for (int k = 0; k < 2; ++k)
        if (d->g1[k]) cudaGraphExecDestroy(d->g1[k]);
    if (d->cap) cudaStreamDestroy(d->cap);
    if (d->own_ws && d->ws) {
        if (d->pooled_ws) {
            // as cudaFree: nothing on the device may still use the workspace
            // when it goes back to the pool (and to the next domain)
            int cur = 0;
            cudaGetDevice(&cur);
            if (cur != d->device) cudaSetDevice(d->device);
            cudaDeviceSynchronize();
            cudaFreeAsync(d->ws, d->stream);
            cudaStreamSynchronize(d->stream);
            if (cur != d->device) cudaSetDevice(cur);
        } else {
            cudaFree(d->ws);
        }
    }
    delete d;
}

lbm_status lbm_release_cached_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : g_pools) {
        cudaSetDevice(kv.first);
        if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(kv.second, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaSetDevice(cur);
            return LBM_ERR_CUDA;
        }
    }
    cudaSetDevice(cur);
    return LBM_OK;
}

}  // extern "C"

// ===========================================================================
// Batches: many domains advanced by one launch per phase.
// ===========================================================================
struct lbm_batch {
    std::vector<lbm_domain*> doms;
    int Q = 0, precision = 0, GK = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    std::vector<int> cur0;             // each domain's buffer parity when the batch was made
    int parity = 0;                    // steps taken by the batch, mod 2
    int variant = 0;
    // tiles of the color kernel, whatever shape the step kernels use (it has
    // no halo): row chunks of 128 nodes (kPhiRows), which leave only the
    // padding columns idle.  LBM_BATCH_PHI_SHAPE=step: the step's shape;
    // =0..5: that shape (shape 3, 32 x 2 x 2, ran a batch of 64 domains of 48^3 to 128^3 at 3.305 ms per
    // step against 3.331 on the step's 64-wide tiles).
    int phi_shape = kPhiRows;
    int4* phi_rows = nullptr;          // {slot, x0, y0, z} row chunks
    int nphi_rows = 0;
    int ntiles[kTileVariants] = {};
    int ncontrast[kTileVariants] = {};           // tiles of domains with density contrast come first
    int device = 0;
    std::vector<int> slots;            // each domain's slot of the constant table
    char* dev = nullptr;               // one allocation for every device table
    int4* tiles[kTileVariants] = {};             // {slot, x0, y0, z0}
    CUtensorMap* maps = nullptr;                 // [kTileVariants][kBatchSlots][3] halo maps by shape and slot
    void* ghost_tabs = nullptr;
    int64_t* ghost_begin = nullptr;
    int64_t total_ghosts = 0;
    cudaGraphExec_t g1[2] = {nullptr, nullptr};
    cudaGraphExec_t g8 = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
    if (b) b->err = m; else g_batch_error = m;
    return s;
}

// Slots of the constant tables (one table per precision and GPU).  A batch
// takes any n free slots (the tile list names each tile's slot, so they need
// not be contiguous); an empty vector means fewer than n are free.
std::mutex g_slot_mutex;
std::map<std::pair<int, int>, std::vector<char>> g_slots_used;

std::vector<int> reserve_slots(int device, int precision, int n) {
    std::lock_guard<std::mutex> lk(g_slot_mutex);
    std::vector<char>& used = g_slots_used[{device, precision}];
    used.resize(kBatchSlots, 0);
    std::vector<int> got;
    for (int k = 0; k < kBatchSlots && (int)got.size() < n; ++k)
        if (!used[k]) got.push_back(k);
    if ((int)got.size() < n) return {};
    for (int k : got) used[k] = 1;
    return got;
}

void release_slots(int device, int precision, const std::vector<int>& slots) {
    std::lock_guard<std::mutex> lk(g_slot_mutex);
    std::vector<char>& used = g_slots_used[{device, precision}];
    for (int k : slots)
        if (k >= 0 && k < (int)used.size()) used[k] = 0;
}

template <typename F>
void bdispatch(int precision, F&& f) {
    switch (precision) {
    case LBM_FP64: f(Launch<double, double>{}); break;
    case LBM_FP32: f(Launch<float, float>{}); break;
    default: f(Launch<float, __half>{}); break;
    }
}

// Appends the tiles {slot, x0, y0, z0} of a domain for tile shape V (the
// shapes of Tile<Q, V>).
void append_tiles(int Q, int V, const lbm_params& P, int i, std::vector<int4>& out) {
    const int TX = tile_extent(Q, V, 0), TY = tile_extent(Q, V, 1), TZ = tile_extent(Q, V, 2);
    for (int z = 0; z < P.nz; z += TZ)
        for (int y = 0; y < P.ny; y += TY)
            for (int x = 0; x < P.nx; x += TX) out.push_back(make_int4(i, x, y, z));
}

void batch_launch_step(lbm_batch* b, int parity, cudaStream_t s) {
    const int V = b->variant;
    bdispatch(b->precision, [&](auto Lx) {
        using L = decltype(Lx);
        L::ghost_batched(b->GK, b->ghost_tabs, b->ghost_begin, (int)b->doms.size(), b->total_ghosts, s);
        const int Vp = b->phi_shape < 0 ? V : b->phi_shape;
        const int4* pt = Vp == kPhiRows ? b->phi_rows : b->tiles[Vp];
        const int np = Vp == kPhiRows ? b->nphi_rows : b->ntiles[Vp];
        L::step_phi_batched(b->Q, V, b->tiles[V], b->maps + (size_t)V * kBatchSlots * 3, b->ntiles[V],
                            b->ncontrast[V], Vp, pt, np, parity, s);
    });
}

lbm_status batch_capture(lbm_batch* b) {
    for (auto* g : {&b->g1[0], &b->g1[1], &b->g8})
        if (*g) { cudaGraphExecDestroy(*g); *g = nullptr; }
    for (int k = 0; k < 3; ++k) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
        if (k < 2) batch_launch_step(b, k, b->cap);
        else for (int t = 0; t < 8; ++t) batch_launch_step(b, t & 1, b->cap);
        const cudaError_t le = cudaGetLastError();          // a launch the capture refused
        e = cudaStreamEndCapture(b->cap, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, LBM_ERR_CUDA, std::string("batch launch (tile shape ") + std::to_string(b->variant) +
                                              "): " + cudaGetErrorString(le));
        }
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t* dst = k == 0 ? &b->g1[0] : (k == 1 ? &b->g1[1] : &b->g8);
        e = cudaGraphInstantiate(dst, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_domain* const* doms, int32_t n, void* cuda_stream, lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!doms || n < 1) return bfail(nullptr, LBM_ERR_ARG, "a batch needs at least one domain");
    lbm_batch* b = new lbm_batch();
    b->Q = doms[0]->prm.lattice;
    b->precision = doms[0]->prm.precision;
    b->GK = doms[0]->lay.GK;
    for (int i = 0; i < n; ++i) {
        if (!doms[i]) { delete b; return bfail(nullptr, LBM_ERR_ARG, "NULL domain in the batch"); }
        if (doms[i]->prm.lattice != b->Q || doms[i]->prm.precision != b->precision) {
            delete b;
            return bfail(nullptr, LBM_ERR_ARG, "all domains of a batch need the same lattice and precision");
        }
        for (int j = 0; j < i; ++j)
            if (doms[j] == doms[i]) { delete b; return bfail(nullptr, LBM_ERR_ARG, "a domain appears twice"); }
        if (doms[i]->poisoned) {
            delete b;
            return bfail(nullptr, LBM_ERR_TIMEOUT, "domain " + std::to_string(i) + ": " + kPoisonedMsg);
        }
        b->doms.push_back(doms[i]);
        b->cur0.push_back(doms[i]->cur);
    }
    b->stream = (cudaStream_t)cuda_stream;
    const char* phi_shape = std::getenv("LBM_BATCH_PHI_SHAPE");
    if (phi_shape && std::strcmp(phi_shape, "step") == 0) b->phi_shape = -1;
    else if (phi_shape && std::strcmp(phi_shape, "rows") == 0) b->phi_shape = kPhiRows;
    else if (phi_shape && phi_shape[0] >= '0' && phi_shape[0] < '0' + kTileVariants && !phi_shape[1])
        b->phi_shape = phi_shape[0] - '0';
    if (n > kBatchSlots) {
        delete b;
        return bfail(nullptr, LBM_ERR_ARG, "a batch holds at most " + std::to_string(kBatchSlots) + " domains");
    }
    cudaGetDevice(&b->device);
    b->slots = reserve_slots(b->device, b->precision, n);
    if (b->slots.empty()) {
        delete b;
        return bfail(nullptr, LBM_ERR_OOM, "no " + std::to_string(n) + " free slots left in the constant table (" +
                                               std::to_string(kBatchSlots) + " per precision, shared by live batches)");
    }
    // host copies of the tables
    size_t esz = 0, gsz = 0;
    bdispatch(b->precision, [&](auto Lx) {
        using L = decltype(Lx);
        esz = L::entry_size(); gsz = L::ghost_table_size();
    });
    // halo maps by tile shape and slot: phi, then u_in of step parity 0 and 1
    // (u_in = U(cur0 ^ parity)), each with the box of that shape's halo tile
    std::vector<CUtensorMap> hm((size_t)kTileVariants * kBatchSlots * 3);
    std::vector<char> slot_tma(kBatchSlots, 0);
    for (int i = 0; i < n; ++i) {
        lbm_domain* d = b->doms[i];
        if (!d->tma) continue;
        const int sl = b->slots[i];
        bool ok = true;
        for (int V = 0; V < kTileVariants && ok; ++V) {
            CUtensorMap m[3];
            ok = encode_halo_maps_any(d, V, m);
            CUtensorMap* dst = &hm[((size_t)V * kBatchSlots + sl) * 3];
            dst[0] = m[0];
            dst[1] = m[1 + b->cur0[i]];
            dst[2] = m[1 + (b->cur0[i] ^ 1)];
        }
        slot_tma[sl] = ok;                       // a slot uses its maps only if every shape's encoded
    }
    std::vector<char> he(esz * n), hg(gsz * n);
    std::vector<int64_t> gbegin(n + 1, 0);
    std::vector<std::vector<int4>> tiles(kTileVariants);
    for (int i = 0; i < n; ++i) {
        lbm_domain* d = b->doms[i];
        const Layout& L = d->lay;
        bdispatch(b->precision, [&](auto Lx) {
            using LL = decltype(Lx);
            StepPtrs sp[2];
            for (int k = 0; k < 2; ++k) {
                const int c = b->cur0[i] ^ k;
                sp[k].Nin = d->N(c); sp[k].Bin = d->B(c); sp[k].Nout = d->N(1 - c); sp[k].Bout = d->B(1 - c);
                sp[k].phi = d->phi(); sp[k].u_in = d->U(c); sp[k].u_out = d->U(1 - c); sp[k].p = d->p();
                sp[k].mask = d->mask(); sp[k].err = d->errflag();
            }
            LL::fill_entry(&he[esz * i], d->cfg, sp, slot_tma[b->slots[i]] != 0);
            LL::fill_ghost_table(&hg[gsz * i], d->ng, d->at<int32_t>(L.off_gnode), d->at<int32_t>(L.off_gcorner),
                                 d->at<void>(L.off_gwt), d->cfg.exp_eps, d->cfg.eps, d->phi(), d->cfg.ghost_rule,
                                 L.plane, d->errflag());
        });
        gbegin[i + 1] = gbegin[i] + d->ng;
    }
    // tiles of the domains with density contrast first, then the others
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < n; ++i) {
            if (b->doms[i]->contrast != (pass == 0)) continue;
            for (int V = 0; V < kTileVariants; ++V) {
                append_tiles(b->Q, V, b->doms[i]->prm, b->slots[i], tiles[V]);
                if (pass == 0) b->ncontrast[V] = (int)tiles[V].size();
            }
        }
    // row chunks of the color kernel, domain by domain, plane by plane
    std::vector<int4> rows;
    for (int i = 0; i < n; ++i) {
        const lbm_params& P = b->doms[i]->prm;
        const int64_t px = b->doms[i]->lay.px, per_plane = px * P.ny;
        for (int z = 0; z < P.nz; ++z)
            for (int64_t o = 0; o < per_plane; o += kPhiChunk)
                rows.push_back(make_int4(b->slots[i], (int)(o % px), (int)(o / px), z));
    }
    b->total_ghosts = gbegin[n];
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off = round_up(off + bytes, 256); return r; };
    const size_t o_g = take(hg.size()), o_gb = take(gbegin.size() * 8);
    const size_t o_m = take(hm.size() * sizeof(CUtensorMap));
    size_t o_t[kTileVariants];
    for (int V = 0; V < kTileVariants; ++V) {
        if (tiles[V].size() > (size_t)INT32_MAX) {
            lbm_batch_destroy(b);
            return bfail(nullptr, LBM_ERR_ARG, "too many tiles");
        }
        o_t[V] = take(tiles[V].size() * sizeof(int4));
    }
    if (rows.size() > (size_t)INT32_MAX) {
        lbm_batch_destroy(b);
        return bfail(nullptr, LBM_ERR_ARG, "too many tiles");
    }
    const size_t o_r = take(rows.size() * sizeof(int4));
    if (cudaMalloc((void**)&b->dev, off) != cudaSuccess) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return bfail(nullptr, LBM_ERR_OOM, "cudaMalloc of the batch tables failed");
    }
    b->ghost_tabs = b->dev + o_g;
    b->ghost_begin = (int64_t*)(b->dev + o_gb);
    b->maps = (CUtensorMap*)(b->dev + o_m);
    cudaError_t e = cudaMemcpy(b->maps, hm.data(), hm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        bdispatch(b->precision, [&](auto Lx) { e = decltype(Lx)::upload_entries(b->slots[i], &he[esz * i], 1); });
    if (e == cudaSuccess) e = cudaMemcpy(b->ghost_tabs, hg.data(), hg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->ghost_begin, gbegin.data(), gbegin.size() * 8, cudaMemcpyHostToDevice);
    for (int V = 0; V < kTileVariants && e == cudaSuccess; ++V) {
        b->tiles[V] = (int4*)(b->dev + o_t[V]);
        b->ntiles[V] = (int)tiles[V].size();
        e = cudaMemcpy(b->tiles[V], tiles[V].data(), tiles[V].size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        b->phi_rows = (int4*)(b->dev + o_r);
        b->nphi_rows = (int)rows.size();
        e = cudaMemcpy(b->phi_rows, rows.data(), rows.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        std::string m = cudaGetErrorString(e);
        lbm_batch_destroy(b);
        return bfail(nullptr, LBM_ERR_CUDA, "batch set-up: " + m);
    }
    lbm_status st = batch_capture(b);
    if (st != LBM_OK) {
        std::string m = b->err;
        lbm_batch_destroy(b);
        return bfail(nullptr, st, m);
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
    if (!b) return bfail(b, LBM_ERR_ARG, "NULL batch");
    if (n < 0) return bfail(b, LBM_ERR_ARG, "n must be >= 0");
    for (size_t i = 0; i < b->doms.size(); ++i) {
        if (b->doms[i]->cur != (b->cur0[i] ^ b->parity))
            return bfail(b, LBM_ERR_ARG, "domain " + std::to_string(i) + " was stepped outside the batch; recreate it");
        if (b->doms[i]->poisoned)
            return bfail(b, LBM_ERR_TIMEOUT, "domain " + std::to_string(i) + ": " + kPoisonedMsg);
    }
    int64_t left = n;
    while (left > 0) {
        cudaError_t e;
        if (b->parity == 0 && left >= 8) { e = cudaGraphLaunch(b->g8, b->stream); left -= 8; }
        else { e = cudaGraphLaunch(b->g1[b->parity], b->stream); b->parity ^= 1; left -= 1; }
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
    }
    for (auto* d : b->doms) {
        d->step += n;
        if (n & 1) d->cur ^= 1;
    }
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b) {
    if (!b) return bfail(b, LBM_ERR_ARG, "NULL batch");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e));
    for (size_t i = 0; i < b->doms.size(); ++i) {
        lbm_status st = check_err_flag(b->doms[i]);
        if (st != LBM_OK) return bfail(b, st, "domain " + std::to_string(i) + ": " + b->doms[i]->err);
    }
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch* b, int32_t steps_per_trial, int32_t* chosen, double* ms_per_step) {
    if (!b || steps_per_trial < 1) return bfail(b, LBM_ERR_ARG, "bad arguments");
    for (size_t i = 0; i < b->doms.size(); ++i)
        if (b->doms[i]->poisoned)
            return bfail(b, LBM_ERR_TIMEOUT, "domain " + std::to_string(i) + ": " + kPoisonedMsg);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, LBM_ERR_CUDA, "cudaEventCreate failed");
    double best = 1e300;
    int best_v = 0;
    for (int V = 0; V < kTileVariants; ++V) {
        b->variant = V;
        batch_launch_step(b, b->parity, b->stream);        // warm-up step of this shape
        b->parity ^= 1;
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return bfail(b, LBM_ERR_CUDA, std::string("batch launch (tile shape ") + std::to_string(V) +
                                              "): " + cudaGetErrorString(le));
        }
        cudaEventRecord(e0, b->stream);
        for (int t = 0; t < steps_per_trial; ++t) {
            batch_launch_step(b, b->parity, b->stream);
            b->parity ^= 1;
        }
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return bfail(b, LBM_ERR_CUDA, cudaGetErrorString(e)); }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / steps_per_trial;
        if (ms_per_step) ms_per_step[V] = per;
        if (per < best) { best = per; best_v = V; }
        const int64_t taken = steps_per_trial + 1;
        for (auto* d : b->doms) { d->step += taken; if (taken & 1) d->cur ^= 1; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->variant = best_v;
    if (chosen) *chosen = best_v;
    return batch_capture(b);
}

int32_t lbm_batch_variant(const lbm_batch* b) { return b ? b->variant : -1; }

lbm_status lbm_batch_set_variant(lbm_batch* b, int32_t v) {
    if (!b || v < 0 || v >= kTileVariants) return bfail(b, LBM_ERR_ARG, "variant must be in 0.." + std::to_string(kTileVariants - 1));
    b->variant = v;
    return batch_capture(b);
}

int32_t lbm_batch_launches_per_step(const lbm_batch* b) {
    if (!b) return -1;
    const int V = b->variant;
    return (b->total_ghosts > 0) + (b->ncontrast[V] > 0) + (b->ntiles[V] > b->ncontrast[V]) + 1;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    // the slots may be handed to another batch: let this batch's launches finish first
    if (!b->slots.empty()) {
        cudaStreamSynchronize(b->stream);
        release_slots(b->device, b->precision, b->slots);
    }
    for (auto* g : {b->g1[0], b->g1[1], b->g8})
        if (g) cudaGraphExecDestroy(g);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->dev) cudaFree(b->dev);
    delete b;
}

}  // extern "C"
