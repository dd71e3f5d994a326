// mtpt.cu -- host side of the C ABI declared in include/mtpt.h.
//
// A handle owns the particle state of one realisation -- or of a batch of
// independent realisations -- on one device, in cell order, and runs one time
// step of Sec. 3 as a fixed sequence of kernels on the handle's stream:
//   walk_key -> scan (3 launches) -> scatter -> gather -> rowsum -> exchange
// A batch concatenates its realisations' particles and gives each
// realisation its own block of cells in one global cell list, so every phase
// is one launch over all particles of all realisations.  Multi-step calls
// replay a captured CUDA graph of two steps.  No step goes through the host:
// the only host<->device traffic is in mtpt_set_particles* / mtpt_get_*
// (the *_async pair copies on two streams of its own, ordered by events).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/mtpt.h"
#include "kernels.cuh"
#include "hostio.cuh"
#include "tiles.cuh"

using namespace mtpt;

namespace {

constexpr int kMaxDim = 3;
constexpr int64_t kGraphMinSteps = 4;   // multi-step calls from this size replay a graph
constexpr int kSettleBlocks = 152;      // grid-stride blocks of k_load_settle (one per SM)

// With MTPT_DEBUG set in the environment, a failing runtime call is named on
// stderr (the status code alone does not say which call failed).
void report_cuda_error(cudaError_t err, const char* expr, int line) {
    static const bool on = std::getenv("MTPT_DEBUG") != nullptr;
    if (on) std::fprintf(stderr, "mtpt: %s failed (line %d): %s\n", expr, line,
                         cudaGetErrorString(err));
}

#define MTPT_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t err_ = (expr);                            \
        if (err_ != cudaSuccess) {                            \
            report_cuda_error(err_, #expr, __LINE__);         \
            (void)cudaGetLastError();                         \
            return MTPT_ERR_CUDA;                             \
        }                                                     \
    } while (0)

#define MTPT_TRY(expr)                  \
    do {                                \
        int rc_ = (expr);               \
        if (rc_ != MTPT_OK) return rc_; \
    } while (0)

// Failure injection for the tests (mtpt_debug_fail_alloc): when positive,
// the countdown's allocation fails as if the device were out of memory.
std::atomic<int64_t> g_fail_alloc{0};

bool injected_alloc_failure() {
    int64_t v = g_fail_alloc.load();
    while (v > 0)
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

// Every device allocation of the library goes through here.
int device_alloc(void** out, size_t bytes) {
    *out = nullptr;
    if (injected_alloc_failure()) return MTPT_ERR_NO_MEMORY;
    if (cudaMalloc(out, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        *out = nullptr;
        return MTPT_ERR_NO_MEMORY;
    }
    return MTPT_OK;
}

// A device buffer that only grows.  A growth allocates before it releases,
// so a failed one leaves the old buffer (and its contents) in place.
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t count = 0;
    int ensure(size_t n) {
        if (n == 0 || (n <= count && p)) return MTPT_OK;
        void* q = nullptr;
        MTPT_TRY(device_alloc(&q, n * sizeof(T)));
        release();
        p = static_cast<T*>(q);
        count = n;
        return MTPT_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        count = 0;
    }
};

// Grows several buffers all or nothing: every new allocation is made before
// any old buffer is released, and after a failure nothing has changed.
struct GrowAll {
    struct Item { void** p; size_t* count; void* q; size_t n; };
    static constexpr int kMax = 48;
    Item items[kMax];
    int k = 0;
    int rc = MTPT_OK;
    template <typename T>
    void want(DevBuf<T>& b, size_t n) {
        if (rc != MTPT_OK || n == 0 || (n <= b.count && b.p)) return;
        if (k == kMax) {
            rc = MTPT_ERR_NO_MEMORY;
            return;
        }
        void* q = nullptr;
        rc = device_alloc(&q, n * sizeof(T));
        if (rc == MTPT_OK) items[k++] = {reinterpret_cast<void**>(&b.p), &b.count, q, n};
    }
    bool grows() const { return k > 0; }
    // Installs the new buffers; the old ones are freed, or, with keep_old,
    // kept (in `olds`) until release_old(), so their contents can be copied.
    void* olds[kMax];
    int nold = 0;
    int commit(bool keep_old = false) {
        if (rc != MTPT_OK) {
            for (int i = 0; i < k; ++i) cudaFree(items[i].q);
            k = 0;
            return rc;
        }
        for (int i = 0; i < k; ++i) {
            if (*items[i].p) {
                if (keep_old) olds[nold++] = *items[i].p;
                else cudaFree(*items[i].p);
            }
            *items[i].p = items[i].q;
            *items[i].count = items[i].n;
        }
        k = 0;
        return MTPT_OK;
    }
    void release_old() {
        for (int i = 0; i < nold; ++i) cudaFree(olds[i]);
        nold = 0;
    }
};

int grid_for(int64_t n) { return int((n + kBlock - 1) / kBlock); }

// Host-side data of one realisation.
struct RealHost {
    mtpt_params prm{};
    double D_RW = 0, D_MT = 0, h2 = 0, psi = 0, psi2 = 0, band_eta = 0;
    int64_t n = 0;
    int64_t n_cells = 0;
    int n_corners = 0;
    // one tile of a checkerboard (Secs. 4-5): the cell grid is the whole
    // box's grid for n_global particles, restricted to the tile and its pad
    bool tiled = false;
    int64_t n_global = 0;
    double tile_lo[3] = {0, 0, 0}, tile_hi[3] = {0, 0, 0}, pad = 0;
};

}  // namespace

struct mtpt_handle;
namespace {
cudaEvent_t take_event(mtpt_handle* h);
// Brackets one kernel launch with timing events when timing is enabled.
struct KernelTimer {
    mtpt_handle* h;
    const char* name;
    cudaEvent_t a = nullptr, b = nullptr;
    KernelTimer(mtpt_handle* hh, const char* nm);
    ~KernelTimer();
};
}  // namespace
#define MTPT_CAT_(a, b) a##b
#define MTPT_CAT(a, b) MTPT_CAT_(a, b)
#define MTPT_TIMED(h, name) KernelTimer MTPT_CAT(kernel_timer_, __LINE__)((h), (name))

struct mtpt_handle {
    int dim = 2, precision = MTPT_FP64;
    bool batch = false;               // created by mtpt_create_batch
    int nreal = 1;
    // realisations: inline storage for a single run (no host allocation on
    // that path), heap storage for a batch
    RealHost real_inline;
    RealParams params_inline{};
    std::vector<RealHost> real_heap;
    std::vector<RealParams> params_heap;
    RealHost* reals = &real_inline;
    RealParams* params = &params_inline;
    bool any_transfer = false, any_walk = false, any_advect = false;
    double cell_scale = 1.0;          // tuning: cell width = cell_scale x psi (>= 1)
    int pair_block = 256;             // tuning: block size of the binary32 pair passes
    cudaStream_t stream = nullptr;
    int64_t n = 0, cap = 0;
    int64_t n_cells = 0, n_cells_pad = 0;
    int n_corners = 0;
    uint64_t step = 0;                // host mirror of the device step counter
    bool have_row_sums = false;
    bool have_particles = false;
    // state, double-buffered (cur = index into the pair)
    DevBuf<double> pos[2], mass[2];
    DevBuf<uint32_t> id[2], rid[2];
    int cur = 0;
    // per-step scratch
    DevBuf<uint32_t> key, perm, cell, count, start;
    DevBuf<unsigned long long> scan_state;   // scan tiles' words + the ticket
    DevBuf<double2> sortkey;          // (x, id | cell << 32) per slot (k_scatter)
    DevBuf<double2> sortrec;          // payload records per slot (k_scatter_rec)
    bool fresh = false;               // state loaded in input order, not yet sorted
    // bimolecular reaction A + B -> 0: species B's masses (cell order, double
    // buffered like `mass`) and the rate constant of the concentration law
    bool reactive = false;
    double react_k = 0.0;
    DevBuf<double> massb[2];
    DevBuf<float2> exb;               // precision form: species B's mass split for pass 2
    DevBuf<float4> rec;
    DevBuf<float2> corners;
    DevBuf<int> corner_first;
    DevBuf<uint32_t> id_first;
    DevBuf<RealParams> params_dev;
    DevBuf<double> r64;
    DevBuf<float4> ex;                // precision form: {m_hi, m_lo, r, list length} per particle
    DevBuf<uint32_t> nb_j, nb_count;      // binary64 form neighbour lists
    DevBuf<double> nb_k;
    int nb_cap = 0;
    DevBuf<uint2> nb32_e;                 // precision form neighbour lists {j, K}
    int nb32_cap = 0;
    DevBuf<uint32_t> adj_nb_j, adj_nb_count;     // adjoint (K, dK) lists
    DevBuf<double2> adj_nb_k;
    int adj_cap = 0;
    DevBuf<double> out_tmp;
    // staging copy of host-loaded input and its check tables
    DevBuf<double> stage, chk_box;
    DevBuf<uint32_t> chk_first, chk_flag;
    DevBuf<double> exp_table;
    // pipelined host I/O: two staging slots each way, per-slot check flags,
    // copy streams and the events that order them against `stream`
    DevBuf<double> in_slot[2], out_slot[2];
    DevBuf<uint32_t> in_flag;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t in_ready[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr};
    cudaEvent_t out_ready[2] = {nullptr, nullptr}, out_free[2] = {nullptr, nullptr};
    int in_next = 0, out_next = 0;
    DevBuf<uint32_t> status;
    DevBuf<unsigned long long> pair_counter, step_dev;
    DevBuf<unsigned long long> emit_counter;
    DevBuf<uint32_t> emit_i, emit_j;
    // adjoint: position tangents dX/dD (double-buffered like pos), state
    // snapshots (checkpoints every `adj_every` steps, the tape of one segment
    // and the final state), adjoint vectors
    bool tangent_on = false;
    DevBuf<double> tan[2];
    DevBuf<unsigned char> snaps;
    size_t snap_bytes = 0;
    int64_t adj_steps = 0, adj_every = 0, adj_nck = 0;
    uint64_t adj_step0 = 0;
    bool adj_ready = false;
    DevBuf<double> dr64, lam_in, lam_s, lam_new, gD, partial, acc;
    // captured two-step graph (valid for `graph_cur`, `graph_flags` and the
    // mass buffer pair as it was: every step swaps the pair, so between loads
    // its order follows `cur`, but a pipelined load moves `cur` alone)
    cudaGraphExec_t graph = nullptr;
    int graph_cur = -1, graph_flags = -1;
    const double* graph_mass0 = nullptr;
    // one walk-ahead middle step, per current buffer (a call's last step
    // swaps the pairs, so consecutive calls alternate between the two)
    cudaGraphExec_t graph_mid[2] = {nullptr, nullptr};
    const double* graph_mid_mass0[2] = {nullptr, nullptr};
    // the next step's walk has been done (by the previous step's pass 2):
    // its positions, ids, keys and counts sit in buffer `cur`
    bool walked_ahead = false;
    cudaStream_t capture_stream = nullptr;
    // split domain: this handle's tile and its pack / keep buffers
    TileGeom tile{};
    int ntiles = 0;
    std::vector<long long> tile_tables;   // per axis: edge keys (f + 1), near_lo (f), near_hi (f)
    int tile_table_off[3] = {0, 0, 0};
    DevBuf<long long> tile_tables_dev;
    DevBuf<unsigned long long> tile_counts, tile_base, tile_cursor, tile_native;
    DevBuf<uint32_t> tile_flag;
    DevBuf<double> tile_keep, tile_stage;
    std::vector<unsigned long long> tile_host;
    int64_t keep_n = 0;
    bool keep_ready = false;
    // per-kernel timing
    bool timing = false;
    struct PendingEvent { const char* name; cudaEvent_t a, b; };
    std::vector<PendingEvent> pending;
    std::vector<cudaEvent_t> spare_events;
    struct Stat { const char* name; int64_t launches; double total_ms; };
    std::vector<Stat> stats;
};

namespace {

cudaEvent_t take_event(mtpt_handle* h) {
    if (!h->spare_events.empty()) {
        cudaEvent_t e = h->spare_events.back();
        h->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

KernelTimer::KernelTimer(mtpt_handle* hh, const char* nm) : h(hh), name(nm) {
    if (!h->timing) return;
    a = take_event(h);
    b = take_event(h);
    if (a && b) cudaEventRecord(a, h->stream);
}

KernelTimer::~KernelTimer() {
    if (!h->timing || !a || !b) return;
    cudaEventRecord(b, h->stream);
    h->pending.push_back({name, a, b});
}

int fold_timing(mtpt_handle* h) {
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (auto& pe : h->pending) {
        float ms = 0.0f;
        MTPT_CUDA_TRY(cudaEventElapsedTime(&ms, pe.a, pe.b));
        bool found = false;
        for (auto& st : h->stats) {
            if (std::strcmp(st.name, pe.name) == 0) {
                st.launches += 1;
                st.total_ms += ms;
                found = true;
                break;
            }
        }
        if (!found) h->stats.push_back({pe.name, 1, double(ms)});
        h->spare_events.push_back(pe.a);
        h->spare_events.push_back(pe.b);
    }
    h->pending.clear();
    return MTPT_OK;
}

void drop_graph(mtpt_handle* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_cur = -1;
    h->graph_flags = -1;
    h->graph_mass0 = nullptr;
    for (int k = 0; k < 2; ++k) {
        if (h->graph_mid[k]) cudaGraphExecDestroy(h->graph_mid[k]);
        h->graph_mid[k] = nullptr;
        h->graph_mid_mass0[k] = nullptr;
    }
}

int validate_params(const mtpt_params* p) {
    if (!p) return MTPT_ERR_INVALID_ARG;
    if (p->dim < 1 || p->dim > kMaxDim) return MTPT_ERR_INVALID_ARG;
    if (p->precision != MTPT_FP64 && p->precision != MTPT_FP32W) return MTPT_ERR_INVALID_ARG;
    if (!(p->D >= 0.0) || !std::isfinite(p->D)) return MTPT_ERR_INVALID_ARG;
    if (!(p->kappa >= 0.0 && p->kappa <= 1.0)) return MTPT_ERR_INVALID_ARG;
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return MTPT_ERR_INVALID_ARG;
    if (!(p->beta > 0.0) || !std::isfinite(p->beta)) return MTPT_ERR_INVALID_ARG;
    if (!(p->lambda > 0.0 && p->lambda <= 20.0)) return MTPT_ERR_INVALID_ARG;
    // kernel variance h^2 = 2 (1 - kappa) D dt / beta: 0 (no transfer) or at
    // least 1e-35, so a = 1 / (2 h^2) <= 5e34 stays within the range of the
    // binary64 kernel exponential
    const double h2 = 2.0 * (1.0 - p->kappa) * p->D * p->dt / p->beta;
    if (h2 > 0.0 && h2 < 1e-35) return MTPT_ERR_INVALID_ARG;
    for (int a = 0; a < p->dim; ++a) {
        if (!std::isfinite(p->lo[a]) || !std::isfinite(p->hi[a]) || !(p->lo[a] < p->hi[a]))
            return MTPT_ERR_INVALID_ARG;
        if (std::fabs(p->lo[a]) > 1e15 || std::fabs(p->hi[a]) > 1e15) return MTPT_ERR_INVALID_ARG;
        if (!std::isfinite(p->v[a]) || !(std::fabs(p->v[a] * p->dt) <= 1e15))
            return MTPT_ERR_INVALID_ARG;
    }
    return MTPT_OK;
}

// Host image of the kernels' order key (int64 order of binary64 values).
long long host_order_key(double x) {
    long long b;
    std::memcpy(&b, &x, sizeof(b));
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// Sec. 3: D_RW = kappa D, D_MT = (1 - kappa) D, walk scale sqrt(2 D_RW dt),
// h^2 = 2 D_MT dt / beta, psi = lambda sqrt(4 D_MT dt / beta).
void derive(RealHost& R, RealParams& P) {
    const mtpt_params& p = R.prm;
    R.D_RW = p.kappa * p.D;
    R.D_MT = (1.0 - p.kappa) * p.D;
    P.sigma = std::sqrt(2.0 * R.D_RW * p.dt);
    R.h2 = 2.0 * R.D_MT * p.dt / p.beta;
    R.psi = p.lambda * std::sqrt(4.0 * R.D_MT * p.dt / p.beta);
    R.psi2 = R.psi * R.psi;
    P.kernel_norm = R.h2 > 0.0 ? std::pow(2.0 * M_PI * R.h2, -0.5 * p.dim) : 0.0;
    P.transfer = R.h2 > 0.0 ? 1 : 0;
    P.advect = 0;
    for (int a = 0; a < 3; ++a) {
        P.vdt[a] = a < p.dim ? p.v[a] * p.dt : 0.0;
        if (a < p.dim && p.v[a] != 0.0) P.advect |= 1u << a;
    }
    P.walk = (P.sigma > 0.0 || P.advect) ? 1 : 0;
    P.h2 = R.h2;
    P.dsigma_dD = p.D > 0.0 ? P.sigma / (2.0 * p.D) : 0.0;
    P.inv_2D = p.D > 0.0 ? 1.0 / (2.0 * p.D) : 0.0;
    P.inv_h2 = R.h2 > 0.0 ? 1.0 / R.h2 : 0.0;
    P.seed = p.seed;
    for (int a = 0; a < 3; ++a) {
        P.box.lo[a] = a < p.dim ? p.lo[a] : 0.0;
        P.box.hi[a] = a < p.dim ? p.hi[a] : 0.0;
        P.box.lo_key[a] = host_order_key(P.box.lo[a]);
        P.box.hi_key[a] = host_order_key(P.box.hi[a]);
    }
}

// Cell grid of one realisation: width >= psi on every axis (slightly above,
// so a pair at distance psi never spans two cell boundaries under rounding),
// with the cell count capped near 4 n so sparse boxes do not allocate huge
// empty grids (cells then just get wider, which stays correct).  A
// realisation without mass transfer gets a single cell.
//
// The cell index of a walked particle is computed in binary32 when its error
// is small: with u = 2^-24, the binary32 evaluation of (x - lo) / w is within
// dc = 3 u (B + L) / psi cells of the exact one (B = max(|lo|, |hi|)), so
// cells of width w >= psi / (1 - 2 dc) keep every pair within psi in adjacent
// cells (at most 2 % wider).  Boxes where dc > 1e-2 (very many cells per
// axis) use binary64.
int setup_grid(RealHost& R, RealParams& P, int64_t cell_base, int corner_base, double scale) {
    const mtpt_params& p = R.prm;
    Grid& g = P.g;
    const double u = std::ldexp(1.0, -24);
    double dc = 0.0;
    for (int a = 0; a < p.dim && R.psi > 0.0; ++a) {
        const double B = std::max(std::fabs(p.lo[a]), std::fabs(p.hi[a]));
        dc = std::max(dc, 3.0 * u * (B + (p.hi[a] - p.lo[a])) / R.psi);
    }
    g.cell_f32 = (P.transfer && dc <= 1e-2) ? 1 : 0;
    // scale 1/2: cells half the cutoff wide, neighbours up to two cells away
    // (reach 2); a reach of R needs R w >= psi plus twice the cell index's
    // error, dc psi in length, on both sides: w >= psi (1 + 2 dc) / R
    g.reach = scale < 1.0 ? 2 : 1;
    const double widen = g.cell_f32 ? 1.0 / (1.0 - 2.0 * dc) : 1.0;
    const double psi_eff = R.psi * widen * (g.reach == 2 ? 0.5 : scale) * (1.0 + 1e-9);
    double ncell[3] = {1, 1, 1};
    for (int a = 0; a < p.dim; ++a) {
        const double L = p.hi[a] - p.lo[a];
        double k = P.transfer ? std::floor(L / psi_eff) : 1.0;
        ncell[a] = std::max(1.0, std::min(k, double(1 << 30)));
    }
    const double cap = std::max(4.0 * double(R.tiled ? R.n_global : R.n) + 64.0, 64.0);
    double total = ncell[0] * ncell[1] * ncell[2];
    for (int guard = 0; guard < 64 && total > cap; ++guard) {
        const double f = std::pow(cap / total, 1.0 / p.dim);
        for (int a = 0; a < p.dim; ++a) ncell[a] = std::max(1.0, std::floor(ncell[a] * f));
        total = ncell[0] * ncell[1] * ncell[2];
        if (total > cap) {
            int amax = 0;
            for (int a = 1; a < p.dim; ++a)
                if (ncell[a] > ncell[amax]) amax = a;
            ncell[amax] = std::max(1.0, ncell[amax] - 1.0);
            total = ncell[0] * ncell[1] * ncell[2];
        }
    }
    if (total > 2.0e9) return MTPT_ERR_INVALID_ARG;
    // a tile keeps the cells of the whole box's grid that cover it and its
    // pad (one cell of margin each side for the cell index's rounding), so
    // its cell corners, offsets and in-row orders are the undivided run's
    double nloc[3] = {ncell[0], ncell[1], ncell[2]}, first[3] = {0, 0, 0};
    if (R.tiled && P.transfer) {
        for (int a = 0; a < p.dim; ++a) {
            const double w = (p.hi[a] - p.lo[a]) / ncell[a];
            const double plo = std::max(p.lo[a], R.tile_lo[a] - R.pad);
            const double phi = std::min(p.hi[a], R.tile_hi[a] + R.pad);
            const double c0 = std::max(0.0, std::floor((plo - p.lo[a]) / w) - 1.0);
            const double c1 = std::min(ncell[a] - 1.0, std::floor((phi - p.lo[a]) / w) + 1.0);
            first[a] = c0;
            nloc[a] = std::max(1.0, c1 - c0 + 1.0);
        }
        total = nloc[0] * nloc[1] * nloc[2];
    }
    double sum_w = 0.0, sum_b = 0.0;
    int off = corner_base;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = int(nloc[a]);
        g.nglob[a] = int(ncell[a]);
        g.off[a] = int(first[a]);
        g.lo[a] = a < p.dim ? p.lo[a] : 0.0;
        g.w[a] = a < p.dim ? (p.hi[a] - p.lo[a]) / ncell[a] : 1.0;
        g.inv_w[a] = 1.0 / g.w[a];
        g.wf[a] = float(g.w[a]);
        g.lo_f[a] = float(g.lo[a]);
        g.inv_w_f[a] = float(g.inv_w[a]);
        g.corner_off[a] = off;
        off += (a < p.dim && P.transfer) ? g.n[a] : 0;
        if (a < p.dim && R.psi > 0.0) {
            sum_w += g.w[a] / R.psi;
            sum_b += (std::max(std::fabs(p.lo[a]), std::fabs(p.hi[a])) + g.w[a]) / R.psi;
        }
    }
    R.n_corners = off - corner_base;
    R.n_cells = int64_t(total);
    P.cell_base = uint32_t(cell_base);

    // Pair-test band.  Each binary32 cell offset is within 2u w (1 + dc) +
    // 2^-46 B of the exact offset; the binary32 difference
    // (off_j - off_i) + shift adds the rounding of both operations and of the
    // shift, so per axis |dx_f - dx| <= 7 u w (1 + dc) + 2^-44 B, and with the
    // roundings of the squares and sums
    //   |d2f - d2| <= psi^2 (u (3 + 14 (1 + dc) sum_a w_a / psi) + 2^-43 sum_a B_a / psi)
    // for every candidate within reach of the cutoff.  Twice that bound is the
    // band half-width eta.
    PairParams& pp = P.pp;
    // (with reach 2 the x difference can span three cells instead of two, one
    // more u w in its bound: 2 (6 + reach) in place of 14)
    const double kdx = 2.0 * (6.0 + g.reach);
    const double eta = 2.0 * (u * (3.0 + kdx * (1.0 + dc) * sum_w) + std::ldexp(sum_b, -43)) + 1e-14;
    R.band_eta = eta;
    pp.psi2 = R.psi2;
    pp.band_lo = std::nextafter(float(R.psi2 * (1.0 - eta)), 0.0f);
    pp.band_hi = std::nextafter(float(R.psi2 * (1.0 + eta)), INFINITY);
    // Candidate windows: reach2 bounds dx^2 + g^2 of every accepted candidate
    // with the binary32 roundings of d2f and of the window arithmetic
    // (2^-16 relative is far above them).  trim_eps covers the sqrt rounding,
    // two dx errors (7 u w (1 + dc) + 2^-44 B each) and the row's departure
    // from x order (a particle sits within dc cells of its cell, dc as above
    // for binary32 cell indices and 2^-29 of it for binary64 ones), with a
    // factor 2 to spare.
    pp.reach2 = std::nextafter(float(double(pp.band_hi) * (1.0 + std::ldexp(1.0, -16))), INFINITY);
    {
        const double dc_cells = g.cell_f32 ? dc : std::ldexp(dc, -29);
        double eps = 0.0;
        for (int a = 0; a < p.dim; ++a) {
            const double B = std::max(std::fabs(p.lo[a]), std::fabs(p.hi[a])) + g.w[a];
            // the cell index's error is dc_cells psi in length, whatever w is
            eps = std::max(eps, 2.0 * (2.0 * dc_cells * std::max(g.w[a], R.psi) +
                                       std::ldexp(g.w[a], -16) + std::ldexp(B, -40)));
        }
        pp.trim_eps = std::nextafter(float(eps), INFINITY);
    }
    pp.a = R.h2 > 0.0 ? 1.0 / (2.0 * R.h2) : 0.0;
    pp.a_log2e = float(pp.a * 1.4426950408889634);
    pp.beta = p.beta;
    // Constants of the binary64 kernel exponential exp(-a d2) (reduction step
    // c = ln 2 / (256 a), c_hi with 32 significant bits; Taylor coefficients
    // (-a)^m / m!), formed in long double.
    pp.ec = ExpNegConsts{};
    if (pp.a > 0.0) {
        const long double ln2 = std::log(2.0L), a = pp.a;
        const long double c = ln2 / (256.0L * a);
        int e = 0;
        const double m = std::frexp(double(c), &e);
        pp.ec.c_hi = std::ldexp(std::nearbyint(std::ldexp(m, 32)), e - 32);
        pp.ec.c_lo = double(c - (long double)pp.ec.c_hi);
        pp.ec.k_scale = float(256.0L * a / ln2);
        pp.ec.p1 = double(-a);
        pp.ec.p2 = double(a * a / 2.0L);
        pp.ec.p3 = double(-a * a * a / 6.0L);
        pp.ec.p4 = double(a * a * a * a / 24.0L);
    }
    return MTPT_OK;
}

// Grids of every realisation, laid out one after another in the global cell
// list and the corner table.
int setup_grids(mtpt_handle* h) {
    int64_t cell_base = 0;
    int corner_base = 0;
    h->any_transfer = false;
    h->any_walk = false;
    h->any_advect = false;
    for (int k = 0; k < h->nreal; ++k) {
        MTPT_TRY(setup_grid(h->reals[k], h->params[k], cell_base, corner_base, h->cell_scale));
        cell_base += h->reals[k].n_cells;
        corner_base += h->reals[k].n_corners;
        h->any_transfer |= h->params[k].transfer != 0;
        h->any_walk |= h->params[k].walk != 0;
        h->any_advect |= h->params[k].advect != 0;
    }
    if (cell_base > int64_t(0xffffffffLL) - kScanTile) return MTPT_ERR_INVALID_ARG;
    // binary64 neighbour-list slots: the expected neighbour count of the
    // densest realisation (density x volume of the cutoff ball) plus four
    // standard deviations of its Poisson spread plus 4, within [8, 64]
    double expect = 0.0;
    for (int k = 0; k < h->nreal; ++k) {
        const mtpt_params& p = h->reals[k].prm;
        double vol = 1.0;
        for (int a = 0; a < p.dim; ++a) vol *= p.hi[a] - p.lo[a];
        const double ball = p.dim == 1 ? 2.0 : (p.dim == 2 ? M_PI : 4.0 * M_PI / 3.0);
        const double nk = double(h->reals[k].tiled ? h->reals[k].n_global : h->reals[k].n);
        expect = std::max(expect, nk / vol * ball * std::pow(h->reals[k].psi, double(p.dim)));
    }
    const int list_cap =
        int(std::min(64.0, std::max(8.0, std::ceil(expect + 4.0 * std::sqrt(expect) + 4.0))));
    h->nb_cap = h->precision == MTPT_FP64 ? list_cap : 0;
    h->nb32_cap = h->precision == MTPT_FP32W ? list_cap : 0;
    h->adj_cap = list_cap;
    h->n_cells = cell_base;
    h->n_corners = corner_base;
    h->n_cells_pad = ((h->n_cells + 1 + kScanTile - 1) / kScanTile) * kScanTile;
    return MTPT_OK;
}

double* exp_table_host() {
    static double table[kExpTable];
    static std::once_flag once;
    std::call_once(once, []() {
        for (int j = 0; j < kExpTable; ++j)
            table[j] = double(exp2l(-static_cast<long double>(j) / static_cast<long double>(kExpTable)));
    });
    return table;
}

// Corner tables of every transferring realisation.
int build_corners(mtpt_handle* h, const RealParams* params_dev, const int* first_dev) {
    if (!h->any_transfer || h->n_corners == 0) return MTPT_OK;
    k_corners<<<grid_for(h->n_corners), kBlock, 0, h->stream>>>(h->n_corners, h->nreal, h->dim,
                                                               params_dev, first_dev,
                                                               h->corners.p);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// Payload-record chunks per particle of the record sort, tangents included
// (the adjoint's), so one allocation serves every record sort.
int64_t sort_rec_chunks(int dim) { return (2 + 2 * dim + 1) / 2; }

// State and per-step buffers for n particles, grown all or nothing (a failed
// growth leaves the handle's state and buffers as they were).  A growth
// carries the first `keep` particles of the current state half over into the
// new buffers, so a later failure of the same load can still go back to
// them.  The record sort's buffer of a single run is grown here too, so no
// step allocates.
int ensure_capacity(mtpt_handle* h, int64_t n, int64_t keep = 0) {
    const int d = h->dim;
    const int64_t cap = std::max<int64_t>(n, 1);
    const int c = h->cur;
    const int64_t old_cap = h->cap;
    const double* old_pos = h->pos[c].p;
    const double* old_mass = h->mass[c].p;
    const uint32_t* old_id = h->id[c].p;
    const uint32_t* old_rid = h->rid[c].p;
    const double* old_massb = h->massb[c].p;
    GrowAll g;
    if (cap > h->cap) {
        for (int b = 0; b < 2; ++b) {
            g.want(h->pos[b], size_t(d) * cap);
            g.want(h->mass[b], size_t(cap));
            if (h->reactive) g.want(h->massb[b], size_t(cap));
            if (h->reactive && b == 0 && h->precision == MTPT_FP32W) g.want(h->exb, size_t(cap));
            g.want(h->id[b], size_t(cap));
            if (h->batch) g.want(h->rid[b], size_t(cap));
        }
        g.want(h->key, size_t(cap));
        g.want(h->perm, size_t(cap));
        g.want(h->sortkey, size_t(cap));
        g.want(h->cell, size_t(cap));
        g.want(h->rec, size_t(cap));
        if (h->precision == MTPT_FP64) g.want(h->r64, size_t(cap));
        else g.want(h->ex, size_t(cap));
    }
    if (!h->batch) g.want(h->sortrec, size_t(sort_rec_chunks(d)) * size_t(std::max(cap, h->cap)));
    g.want(h->status, 1);
    g.want(h->pair_counter, 1);
    g.want(h->step_dev, 1);
    if (g.grows()) drop_graph(h);
    const bool carry = keep > 0 && cap > old_cap && old_pos;
    MTPT_TRY(g.commit(carry));
    if (carry) {
        const size_t row = size_t(keep) * sizeof(double);
        int rc = MTPT_OK;
        if (cudaMemcpy2DAsync(h->pos[c].p, size_t(cap) * sizeof(double), old_pos,
                              size_t(old_cap) * sizeof(double), row, size_t(d),
                              cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
            cudaMemcpyAsync(h->mass[c].p, old_mass, row, cudaMemcpyDeviceToDevice,
                            h->stream) != cudaSuccess ||
            cudaMemcpyAsync(h->id[c].p, old_id, size_t(keep) * 4, cudaMemcpyDeviceToDevice,
                            h->stream) != cudaSuccess ||
            (h->reactive && old_massb &&
             cudaMemcpyAsync(h->massb[c].p, old_massb, row, cudaMemcpyDeviceToDevice,
                             h->stream) != cudaSuccess) ||
            (h->batch && old_rid &&
             cudaMemcpyAsync(h->rid[c].p, old_rid, size_t(keep) * 4, cudaMemcpyDeviceToDevice,
                             h->stream) != cudaSuccess) ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            (void)cudaGetLastError();
            rc = MTPT_ERR_CUDA;
        }
        g.release_old();
        MTPT_TRY(rc);
    }
    if (cap > h->cap) h->cap = cap;
    return MTPT_OK;
}

// Zeroes the cell-count scan's tile words and ticket (a grid change moves
// the ticket's launch numbering).
int reset_scan(mtpt_handle* h, cudaStream_t st) {
    const size_t words = size_t(h->n_cells_pad / kScanTile) + 1;
    MTPT_CUDA_TRY(cudaMemsetAsync(h->scan_state.p, 0, words * sizeof(unsigned long long), st));
    return MTPT_OK;
}

// Test hook of mtpt_debug_scan_hold: the scan tile that never publishes (-1: none).
std::atomic<int> g_scan_hold{-1};

// Exclusive prefix sum of the cell counts into start (one launch).
int launch_scan(mtpt_handle* h, cudaStream_t st, bool advance) {
    const int ntiles = int(h->n_cells_pad / kScanTile);
    k_scan<<<ntiles, kScanThreads, 0, st>>>(reinterpret_cast<const uint4*>(h->count.p),
                                            reinterpret_cast<uint4*>(h->start.p),
                                            h->scan_state.p, ntiles, h->step_dev.p,
                                            advance ? 1 : 0, g_scan_hold.load());
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// The cell list's arrays for the current grid, grown all or nothing.
int ensure_cells(mtpt_handle* h) {
    const size_t padded = size_t(h->n_cells_pad);
    GrowAll g;
    g.want(h->count, padded);
    g.want(h->start, padded);
    g.want(h->scan_state, padded / kScanTile + 1);   // + the scan's ticket
    g.want(h->corners, size_t(std::max(h->n_corners, 1)));
    if (h->nb_cap > 0) {
        const size_t slots = size_t(h->nb_cap) * size_t(h->cap);
        g.want(h->nb_j, slots);
        g.want(h->nb_k, slots);
        g.want(h->nb_count, size_t(h->cap));
    }
    if (h->nb32_cap > 0) {
        g.want(h->nb32_e, size_t(h->nb32_cap) * size_t(h->cap));
    }
    if (g.grows()) drop_graph(h);
    MTPT_TRY(g.commit());
    // the scan's words for this grid's tiles
    MTPT_TRY(reset_scan(h, h->stream));
    // counts start (and, after each scatter, end) at zero
    MTPT_CUDA_TRY(cudaMemsetAsync(h->count.p, 0, padded * sizeof(uint32_t), h->stream));
    return MTPT_OK;
}

// Uploads the realisation table and the corner and particle offsets, and
// builds the corner tables.
int upload_tables(mtpt_handle* h) {
    const int nr = h->nreal;
    MTPT_TRY(h->params_dev.ensure(size_t(nr)));
    MTPT_CUDA_TRY(cudaMemcpyAsync(h->params_dev.p, h->params, size_t(nr) * sizeof(RealParams),
                                  cudaMemcpyHostToDevice, h->stream));
    std::vector<int> cf(size_t(nr) + 1);
    std::vector<uint32_t> idf(size_t(nr) + 1);
    for (int k = 0; k < nr; ++k) {
        cf[size_t(k)] = h->params[k].g.corner_off[0];
        idf[size_t(k)] = h->params[k].id_offset;
    }
    cf[size_t(nr)] = h->n_corners;
    idf[size_t(nr)] = uint32_t(h->n);
    MTPT_TRY(h->corner_first.ensure(size_t(nr) + 1));
    MTPT_TRY(h->id_first.ensure(size_t(nr) + 1));
    MTPT_CUDA_TRY(cudaMemcpyAsync(h->corner_first.p, cf.data(), cf.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, h->stream));
    MTPT_CUDA_TRY(cudaMemcpyAsync(h->id_first.p, idf.data(), idf.size() * sizeof(uint32_t),
                                  cudaMemcpyHostToDevice, h->stream));
    MTPT_TRY(build_corners(h, h->params_dev.p, h->corner_first.p));
    // the host vectors are pageable: wait before they go out of scope
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MTPT_OK;
}

// Status code of a status word read after the stream drained.  A rejected
// pipelined load is reported once: its bits are cleared here.  It kept the old
// step counter on the device, so the host mirror (reset when the load was
// enqueued) is read back.
int status_code(mtpt_handle* h, uint32_t st) {
    const uint32_t load_bits = st & (kStatusLoadPosition | kStatusLoadMass);
    if (load_bits) {
        const uint32_t rest = st & ~load_bits;
        MTPT_CUDA_TRY(cudaMemcpy(h->status.p, &rest, sizeof(rest), cudaMemcpyHostToDevice));
        unsigned long long step = 0;
        MTPT_CUDA_TRY(cudaMemcpy(&step, h->step_dev.p, sizeof(step), cudaMemcpyDeviceToHost));
        h->step = uint64_t(step);
    }
    if (st & (kStatusNonFinite | kStatusOutOfDomain | kStatusLoadPosition))
        return MTPT_ERR_OUT_OF_DOMAIN;
    if (st & kStatusLoadMass) return MTPT_ERR_INVALID_ARG;
    return MTPT_OK;
}

int read_status(mtpt_handle* h) {
    uint32_t st = 0;
    MTPT_CUDA_TRY(cudaMemcpyAsync(&st, h->status.p, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return status_code(h, st);
}

template <class View>
View make_view(const mtpt_handle* h, int input_buf, int sorted_buf);

template <>
SingleView make_view<SingleView>(const mtpt_handle* h, int, int) {
    SingleView v;
    v.p = h->params[0];
    return v;
}

template <>
BatchView make_view<BatchView>(const mtpt_handle* h, int input_buf, int sorted_buf) {
    BatchView v;
    v.tbl = h->params_dev.p;
    v.rid_input = h->rid[input_buf].p;
    v.rid_sorted = h->rid[sorted_buf].p;
    return v;
}

// Counting-sort scatter of buffer c's particles into slots (index and sort
// key), then the gather into buffer o in cell order (tangents too when on).
template <int DIM, class View, bool TANGENT>
int launch_sort_t(mtpt_handle* h, int c, int o, const View& vin) {
    const int n = int(h->n);
    const int blocks = grid_for(n);
    const int64_t stride = h->cap;
    uint32_t* rid_out = View::kBatch ? h->rid[o].p : nullptr;
    const double* tan_in = TANGENT ? h->tan[c].p : nullptr;
    double* tan_out = TANGENT ? h->tan[o].p : nullptr;
    {
        MTPT_TIMED(h, "scatter");
        k_scatter<<<blocks, kBlock, 0, h->stream>>>(n, h->key.p, h->start.p, h->count.p,
                                                    h->pos[c].p, h->id[c].p, h->perm.p,
                                                    h->sortkey.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    MTPT_TIMED(h, "gather");
    k_gather<DIM, View, TANGENT><<<blocks, kBlock, 0, h->stream>>>(
        n, stride, h->perm.p, h->sortkey.p, h->start.p, h->pos[c].p, h->mass[c].p, h->id[o].p,
        h->pos[o].p, h->mass[o].p, h->cell.p, h->rec.p, h->corners.p, rid_out, vin, tan_in,
        tan_out, h->reactive ? h->massb[c].p : nullptr, h->reactive ? h->massb[o].p : nullptr);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// The sort of a freshly loaded single run: payload records (see
// k_scatter_rec), then the gather from them.
template <int DIM, bool TANGENT>
int launch_sort_rec(mtpt_handle* h, int c, int o, const SingleView& vin) {
    const int n = int(h->n);
    const int blocks = grid_for(n);
    const int64_t stride = h->cap;
    MTPT_TRY(h->sortrec.ensure(size_t(SortRec<DIM, TANGENT>::kChunks) * size_t(h->cap)));
    {
        MTPT_TIMED(h, "scatter");
        k_scatter_rec<DIM, TANGENT><<<blocks, kBlock, 0, h->stream>>>(
            n, stride, h->key.p, h->start.p, h->count.p, h->pos[c].p, h->mass[c].p, h->id[c].p,
            TANGENT ? h->tan[c].p : nullptr, h->sortrec.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    MTPT_TIMED(h, "gather");
    double* tan_out = TANGENT ? h->tan[o].p : nullptr;
    k_gather_rec<DIM, TANGENT><<<blocks, kBlock, 0, h->stream>>>(
        n, stride, h->sortrec.p, h->start.p, h->id[o].p, h->pos[o].p, h->mass[o].p, h->cell.p,
        h->rec.p, h->corners.p, vin, tan_out);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// Sort of buffer c into buffer o: the record sort right after a host load of
// a single run (input order), the sort-key sort otherwise.  Both give the
// same cell order bit for bit.
template <int DIM, class View>
int launch_sort(mtpt_handle* h, int c, int o, const View& vin) {
    const bool fresh = h->fresh;
    h->fresh = false;
    if constexpr (!View::kBatch) {
        if (fresh && !h->reactive) {      // (the records carry one species)
            if (h->tangent_on) return launch_sort_rec<DIM, true>(h, c, o, vin);
            return launch_sort_rec<DIM, false>(h, c, o, vin);
        }
    }
    if (h->tangent_on) return launch_sort_t<DIM, View, true>(h, c, o, vin);
    return launch_sort_t<DIM, View, false>(h, c, o, vin);
}

// The reaction's particle rate kp = k N / V (C = N M / V, V the run's box)
// and the step dt.
void reaction_rate(const mtpt_handle* h, double* kp, double* dt) {
    const mtpt_params& p = h->reals[0].prm;
    double vol = 1.0;
    for (int a = 0; a < h->dim; ++a) vol *= p.hi[a] - p.lo[a];
    *kp = h->react_k * double(h->n) / vol;
    *dt = p.dt;
}

template <int DIM, class View, int BLOCK>
int launch_pairs_f32(mtpt_handle* h, int n, int64_t stride, const double* pos_s, const View& vs,
                     int o, int c, bool walk_ahead) {
    const int blocks = int((n + BLOCK - 1) / BLOCK);
    const NbList32 nb{h->nb32_e.p, h->nb32_e.p ? h->nb32_cap : 0};
    {
        MTPT_TIMED(h, "rowsum_f32");
        k_rowsum_f32<DIM, View, BLOCK><<<blocks, BLOCK, 0, h->stream>>>(
            n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->mass[o].p, h->ex.p,
            h->pair_counter.p,
            h->ntiles > 0 ? h->id[o].p : nullptr, nb);
    }
    if (h->reactive) {
        // species B's split, then one pass 2 for both species and the reaction
        // (a reaction runs on a plain handle only: batches refuse it)
        k_split_mass<<<grid_for(n), kBlock, 0, h->stream>>>(n, h->massb[o].p, h->exb.p);
        double kp, dt;
        reaction_rate(h, &kp, &dt);
        if constexpr (!View::kBatch) {
            if (walk_ahead) {
                // and the next step's walk into buffer c (see WalkAhead)
                const WalkAhead wa{h->id[o].p, h->pos[c].p, h->id[c].p, h->key.p, h->count.p,
                                   h->status.p, h->step_dev.p};
                MTPT_TIMED(h, "exchange_walk_f32");
                if (h->any_advect)
                    k_exchange_f32<DIM, View, BLOCK, true, 2><<<blocks, BLOCK, 0, h->stream>>>(
                        n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->ex.p,
                        h->mass[o].p, h->mass[c].p, nb, h->exb.p, h->massb[o].p, h->massb[c].p,
                        kp, dt, float(kp * dt), wa);
                else
                    k_exchange_f32<DIM, View, BLOCK, true, 1><<<blocks, BLOCK, 0, h->stream>>>(
                        n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->ex.p,
                        h->mass[o].p, h->mass[c].p, nb, h->exb.p, h->massb[o].p, h->massb[c].p,
                        kp, dt, float(kp * dt), wa);
                MTPT_CUDA_TRY(cudaGetLastError());
                return MTPT_OK;
            }
        }
        MTPT_TIMED(h, "exchange_f32");
        k_exchange_f32<DIM, View, BLOCK, true><<<blocks, BLOCK, 0, h->stream>>>(
            n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->ex.p, h->mass[o].p,
            h->mass[c].p, nb, h->exb.p, h->massb[o].p, h->massb[c].p, kp, dt, float(kp * dt));
        MTPT_CUDA_TRY(cudaGetLastError());
        return MTPT_OK;
    }
    if (walk_ahead) {
        // pass 2 plus the next step's walk into buffer c (see WalkAhead)
        WalkAhead wa{h->id[o].p, h->pos[c].p, h->id[c].p, h->key.p, h->count.p,
                     h->status.p, h->step_dev.p};
        if (View::kBatch) {
            wa.rid_in = h->rid[o].p;
            wa.rid_next = h->rid[c].p;
        }
        MTPT_TIMED(h, "exchange_walk_f32");
        if (h->any_advect)
            k_exchange_f32<DIM, View, BLOCK, false, 2><<<blocks, BLOCK, 0, h->stream>>>(
                n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->ex.p, h->mass[o].p,
                h->mass[c].p, nb, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0f, wa);
        else
            k_exchange_f32<DIM, View, BLOCK, false, 1><<<blocks, BLOCK, 0, h->stream>>>(
                n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->ex.p, h->mass[o].p,
                h->mass[c].p, nb, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0f, wa);
        MTPT_CUDA_TRY(cudaGetLastError());
        return MTPT_OK;
    }
    MTPT_TIMED(h, "exchange_f32");
    k_exchange_f32<DIM, View, BLOCK><<<blocks, BLOCK, 0, h->stream>>>(
        n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, vs, h->ex.p, h->mass[o].p,
        h->mass[c].p, nb);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// Species B of a binary64 reaction run: its transfer with the weights of
// this step (the row sums and neighbour lists of species A's passes), then
// the reaction on every particle (k_react).  B's masses move from buffer o
// to c like A's.  (The precision form does both species and the reaction in
// one pass 2: launch_pairs_f32.)
template <int DIM, class View>
int launch_species_b(mtpt_handle* h, int n, int64_t stride, const double* pos_s, const View& vs,
                     int o, int c) {
    if (h->precision == MTPT_FP32W) return MTPT_OK;
    const int blocks = grid_for(n);
    cudaStream_t st = h->stream;
    {
        MTPT_TIMED(h, "exchange_f64");
        k_exchange_f64<DIM, View><<<blocks, kBlock, 0, st>>>(
            n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, vs, h->r64.p,
            h->massb[o].p, h->massb[c].p, NbList64{h->nb_j.p, h->nb_k.p, h->nb_count.p, h->nb_cap});
    }
    MTPT_CUDA_TRY(cudaGetLastError());
    double kp, dt;
    reaction_rate(h, &kp, &dt);
    {
        MTPT_TIMED(h, "react");
        k_react<true><<<blocks, kBlock, 0, st>>>(n, h->mass[c].p, h->massb[c].p, kp, dt,
                                                 float(kp * dt));
    }
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// Enqueues one time step (or part of it, per `flags`).  The step counter
// lives on the device and advances inside the step, so the same launches can
// be captured once and replayed.
template <int DIM, class View>
int launch_step(mtpt_handle* h, int flags, bool walk_ahead) {
    // a reaction walks ahead in the precision form, whose pass 2 does both
    // species and the reaction (the binary64 form runs species B after it)
    walk_ahead = walk_ahead && (!h->reactive || (h->precision == MTPT_FP32W && !View::kBatch));
    const int n = int(h->n);
    if (n == 0) {
        // an empty handle (e.g. a tile without particles) keeps its walk's
        // step counter in line with the host mirror
        if ((flags & MTPT_DO_WALK) && h->step_dev.p) {
            k_advance_step<<<1, 1, 0, h->stream>>>(h->step_dev.p);
            MTPT_CUDA_TRY(cudaGetLastError());
        }
        return MTPT_OK;
    }
    const int64_t stride = h->cap;
    const int blocks = grid_for(n);
    cudaStream_t st = h->stream;
    const bool walk = (flags & MTPT_DO_WALK) && h->any_walk;
    const bool transfer = (flags & MTPT_DO_TRANSFER) && h->any_transfer;
    const int c = h->cur, o = 1 - h->cur;
    const View vin = make_view<View>(h, c, c);
    if ((walk || transfer) && !h->walked_ahead) {
        MTPT_TIMED(h, "walk_key");
        if (h->tangent_on) {
            if (h->any_advect)
                k_walk_key<DIM, View, true, true><<<blocks, kBlock, 0, st>>>(
                    n, stride, h->pos[c].p, h->id[c].p, h->step_dev.p, walk ? 1 : 0,
                    transfer ? 1 : 0, vin, h->key.p, h->count.p, h->status.p, h->tan[c].p);
            else
                k_walk_key<DIM, View, true><<<blocks, kBlock, 0, st>>>(
                    n, stride, h->pos[c].p, h->id[c].p, h->step_dev.p, walk ? 1 : 0,
                    transfer ? 1 : 0, vin, h->key.p, h->count.p, h->status.p, h->tan[c].p);
        } else if (h->any_advect) {
            k_walk_key<DIM, View, false, true><<<blocks, kBlock, 0, st>>>(
                n, stride, h->pos[c].p, h->id[c].p, h->step_dev.p, walk ? 1 : 0,
                transfer ? 1 : 0, vin, h->key.p, h->count.p, h->status.p);
        } else {
            k_walk_key<DIM, View><<<blocks, kBlock, 0, st>>>(
                n, stride, h->pos[c].p, h->id[c].p, h->step_dev.p, walk ? 1 : 0,
                transfer ? 1 : 0, vin, h->key.p, h->count.p, h->status.p);
        }
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    const bool advance = (flags & MTPT_DO_WALK) != 0;
    if (!transfer) {
        if (advance) {
            k_advance_step<<<1, 1, 0, st>>>(h->step_dev.p);
            MTPT_CUDA_TRY(cudaGetLastError());
        }
        return MTPT_OK;
    }

    {
        MTPT_TIMED(h, "scan");
        MTPT_TRY(launch_scan(h, st, advance));
    }
    const bool split = h->precision == MTPT_FP32W;
    MTPT_TRY((launch_sort<DIM, View>(h, c, o, vin)));
    // state now lives in buffer o (cell order); masses are updated into c
    const View vs = make_view<View>(h, o, o);
    const double* pos_s = h->pos[o].p;
    if (!split) {
        {
            MTPT_TIMED(h, "rowsum_f64");
            k_rowsum_f64<DIM, View><<<blocks, kBlock, 0, st>>>(
                n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, vs, h->r64.p,
                h->pair_counter.p, NbList64{h->nb_j.p, h->nb_k.p, h->nb_count.p, h->nb_cap},
                h->ntiles > 0 ? h->id[o].p : nullptr);
        }
        const NbList64 nb64{h->nb_j.p, h->nb_k.p, h->nb_count.p, h->nb_cap};
        if (walk_ahead) {
            // pass 2 plus the next step's walk into buffer c (see WalkAhead)
            WalkAhead wa{h->id[o].p, h->pos[c].p, h->id[c].p, h->key.p, h->count.p,
                         h->status.p, h->step_dev.p};
            if (View::kBatch) {
                wa.rid_in = h->rid[o].p;
                wa.rid_next = h->rid[c].p;
            }
            MTPT_TIMED(h, "exchange_walk_f64");
            if (h->any_advect)
                k_exchange_f64<DIM, View, 2><<<blocks, kBlock, 0, st>>>(
                    n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, vs,
                    h->r64.p, h->mass[o].p, h->mass[c].p, nb64, wa);
            else
                k_exchange_f64<DIM, View, 1><<<blocks, kBlock, 0, st>>>(
                    n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, vs,
                    h->r64.p, h->mass[o].p, h->mass[c].p, nb64, wa);
        } else {
            MTPT_TIMED(h, "exchange_f64");
            k_exchange_f64<DIM, View><<<blocks, kBlock, 0, st>>>(
                n, stride, pos_s, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, vs, h->r64.p,
                h->mass[o].p, h->mass[c].p, nb64);
        }
    } else {
        if (h->pair_block == 128) {
            MTPT_TRY((launch_pairs_f32<DIM, View, 128>(h, n, stride, pos_s, vs, o, c, walk_ahead)));
        } else {
            MTPT_TRY((launch_pairs_f32<DIM, View, 256>(h, n, stride, pos_s, vs, o, c, walk_ahead)));
        }
    }
    MTPT_CUDA_TRY(cudaGetLastError());
    h->have_row_sums = true;
    if (walk_ahead) {
        // pass 2 wrote the masses and the next step's walked positions, ids,
        // keys and counts into buffer c, which stays current
        h->walked_ahead = true;
        return MTPT_OK;
    }
    h->walked_ahead = false;
    if (h->reactive) MTPT_TRY((launch_species_b<DIM, View>(h, n, stride, pos_s, vs, o, c)));
    // positions and ids live in o; the updated masses were written into c's
    // buffer: swap the mass pair so both sit at index o, then make o current.
    std::swap(h->mass[c], h->mass[o]);
    if (h->reactive) std::swap(h->massb[c], h->massb[o]);
    h->cur = o;
    return MTPT_OK;
}

int dispatch_step(mtpt_handle* h, int flags, bool walk_ahead = false) {
    if (h->batch) {
        switch (h->dim) {
            case 1: return launch_step<1, BatchView>(h, flags, walk_ahead);
            case 2: return launch_step<2, BatchView>(h, flags, walk_ahead);
            default: return launch_step<3, BatchView>(h, flags, walk_ahead);
        }
    }
    switch (h->dim) {
        case 1: return launch_step<1, SingleView>(h, flags, walk_ahead);
        case 2: return launch_step<2, SingleView>(h, flags, walk_ahead);
        default: return launch_step<3, SingleView>(h, flags, walk_ahead);
    }
}

// Captures steps into an executable graph: two consecutive plain steps (the
// buffer pairs swap every step, so two steps return them to the starting
// arrangement), or, with walk_ahead, one middle step of a walk-ahead run
// (entered with the walk done, it leaves it done for the next step and swaps
// nothing).
int capture_steps(mtpt_handle* h, int flags, bool walk_ahead) {
    if (walk_ahead) {
        cudaGraphExec_t& old = h->graph_mid[h->cur];
        if (old) cudaGraphExecDestroy(old);
        old = nullptr;
    } else {
        if (h->graph) cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (!h->capture_stream)
        MTPT_CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    const cudaStream_t user = h->stream;
    const int cur0 = h->cur;
    const bool rows0 = h->have_row_sums, fresh0 = h->fresh, ahead0 = h->walked_ahead;
    DevBuf<double> mass0 = h->mass[0], mass1 = h->mass[1];
    DevBuf<double> massb0 = h->massb[0], massb1 = h->massb[1];
    h->stream = h->capture_stream;
    MTPT_CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = dispatch_step(h, flags, walk_ahead);
    if (rc == MTPT_OK && !walk_ahead) rc = dispatch_step(h, flags);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
    // capture only recorded the launches: restore the host bookkeeping
    h->stream = user;
    h->cur = cur0;
    h->have_row_sums = rows0;
    h->fresh = fresh0;
    h->walked_ahead = ahead0;
    h->mass[0] = mass0;
    h->mass[1] = mass1;
    h->massb[0] = massb0;
    h->massb[1] = massb1;
    if (ec != cudaSuccess || rc != MTPT_OK || !graph) {
        (void)cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return rc != MTPT_OK ? rc : MTPT_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        (void)cudaGetLastError();
        return MTPT_ERR_CUDA;
    }
    if (walk_ahead) {
        h->graph_mid[cur0] = exec;
        h->graph_mid_mass0[cur0] = h->mass[0].p;
        return MTPT_OK;
    }
    h->graph = exec;
    h->graph_cur = cur0;
    h->graph_flags = flags;
    h->graph_mass0 = h->mass[0].p;
    return MTPT_OK;
}

// Whether a call's steps can run with walk-ahead (all but the last step's
// pass 2 also walk the particles for the step after): a plain handle or a
// batch (not a tile, a binary64 reaction or the adjoint's tangent run)
// stepping with both the walk and the transfer.
bool walk_ahead_ok(const mtpt_handle* h, int flags) {
    return h->ntiles == 0 && (!h->reactive || h->precision == MTPT_FP32W) && !h->tangent_on &&
           h->any_walk && h->any_transfer && h->n > 0 &&
           flags == (MTPT_DO_WALK | MTPT_DO_TRANSFER);
}

int run_steps(mtpt_handle* h, int64_t nsteps, int flags) {
    const bool use_graph = nsteps >= kGraphMinSteps && !h->timing && !h->tangent_on && h->n > 0;
    if (nsteps >= 2 && walk_ahead_ok(h, flags)) {
        // first step (walk, and the record sort after a host load), the middle
        // steps (replayed from a one-step graph), a last step without walk-ahead
        MTPT_TRY(dispatch_step(h, flags, true));
        int64_t middle = nsteps - 2;
        if (use_graph && middle > 0) {
            // (walk-ahead runs only with both flags, so the flags need no key)
            const int k = h->cur;
            if (!h->graph_mid[k] || h->graph_mid_mass0[k] != h->mass[0].p)
                MTPT_TRY(capture_steps(h, flags, true));
            for (; middle > 0; --middle) MTPT_CUDA_TRY(cudaGraphLaunch(h->graph_mid[k], h->stream));
        }
        for (; middle > 0; --middle) MTPT_TRY(dispatch_step(h, flags, true));
        MTPT_TRY(dispatch_step(h, flags, false));
        h->step += uint64_t(nsteps);
        return MTPT_OK;
    }
    int64_t done = 0;
    if (use_graph && h->fresh) {          // the record sort stays out of the graph
        MTPT_TRY(dispatch_step(h, flags));
        done = 1;
    }
    if (use_graph) {
        if (!h->graph || h->graph_cur != h->cur || h->graph_flags != flags ||
            h->graph_mass0 != h->mass[0].p)
            MTPT_TRY(capture_steps(h, flags, false));
        for (; done + 2 <= nsteps; done += 2) MTPT_CUDA_TRY(cudaGraphLaunch(h->graph, h->stream));
        // an even number of steps leaves the buffers where they started; a
        // transfer step leaves row sums behind
        const bool transfer = (flags & MTPT_DO_TRANSFER) && h->any_transfer;
        if (transfer && done > 0) h->have_row_sums = true;
    }
    for (; done < nsteps; ++done) MTPT_TRY(dispatch_step(h, flags));
    if (flags & MTPT_DO_WALK) h->step += uint64_t(nsteps);
    return MTPT_OK;
}

int ensure_out_tmp(mtpt_handle* h) {
    return h->out_tmp.ensure(size_t(h->dim) * std::max<int64_t>(h->n, 1));
}

// Copy `naxes` arrays of the current state (stride cap, cell order) into
// `out_dev` (stride n, input order).
int unpermute_to(mtpt_handle* h, const double* src, int naxes, double* out_dev) {
    if (h->n == 0) return MTPT_OK;
    if (h->ntiles > 0) {            // a tile's particles come and go: its own order
        MTPT_CUDA_TRY(cudaMemcpy2DAsync(out_dev, size_t(h->n) * sizeof(double), src,
                                        size_t(h->cap) * sizeof(double),
                                        size_t(h->n) * sizeof(double), size_t(naxes),
                                        cudaMemcpyDeviceToDevice, h->stream));
        return MTPT_OK;
    }
    k_unpermute<double><<<grid_for(h->n), kBlock, 0, h->stream>>>(
        int(h->n), h->cap, naxes, h->id[h->cur].p, src, 1, 1.0, out_dev);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

int copy_out_host(mtpt_handle* h, int naxes, double* out) {
    const size_t bytes = size_t(naxes) * size_t(h->n) * sizeof(double);
    if (bytes) MTPT_CUDA_TRY(cudaMemcpyAsync(out, h->out_tmp.p, bytes, cudaMemcpyDeviceToHost, h->stream));
    uint32_t st = 0;
    MTPT_CUDA_TRY(cudaMemcpyAsync(&st, h->status.p, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return status_code(h, st);
}

int set_step_dev(mtpt_handle* h, uint64_t step) {
    k_set_step<<<1, 1, 0, h->stream>>>(h->step_dev.p, (unsigned long long)step);
    MTPT_CUDA_TRY(cudaGetLastError());
    h->step = step;
    return MTPT_OK;
}

// Host-side bookkeeping of a handle's particles and grid, saved before a load
// or a retuning and put back when that fails part of the way (the device
// buffers grow all or nothing and never lose the state they hold).
struct HostSnapshot {
    std::vector<RealHost> reals;
    std::vector<RealParams> params;
    int64_t n = 0, n_cells = 0, n_cells_pad = 0;
    int n_corners = 0, nb_cap = 0, nb32_cap = 0, adj_cap = 0, cur = 0, pair_block = 256;
    bool any_transfer = false, any_walk = false, any_advect = false, fresh = false;
    bool have_row_sums = false, have_particles = false, adj_ready = false;
    uint64_t step = 0;
    double cell_scale = 1.0;

    bool take(const mtpt_handle* h) {
        try {
            reals.assign(h->reals, h->reals + h->nreal);
            params.assign(h->params, h->params + h->nreal);
        } catch (...) {
            return false;
        }
        n = h->n; n_cells = h->n_cells; n_cells_pad = h->n_cells_pad;
        n_corners = h->n_corners; nb_cap = h->nb_cap; nb32_cap = h->nb32_cap;
        adj_cap = h->adj_cap; cur = h->cur; pair_block = h->pair_block;
        any_transfer = h->any_transfer; any_walk = h->any_walk; any_advect = h->any_advect;
        fresh = h->fresh; have_row_sums = h->have_row_sums; have_particles = h->have_particles;
        adj_ready = h->adj_ready; step = h->step; cell_scale = h->cell_scale;
        return true;
    }
    void put(mtpt_handle* h) const {
        std::copy(reals.begin(), reals.end(), h->reals);
        std::copy(params.begin(), params.end(), h->params);
        h->n = n; h->n_cells = n_cells; h->n_cells_pad = n_cells_pad;
        h->n_corners = n_corners; h->nb_cap = nb_cap; h->nb32_cap = nb32_cap;
        h->adj_cap = adj_cap; h->cur = cur; h->pair_block = pair_block;
        h->any_transfer = any_transfer; h->any_walk = any_walk; h->any_advect = any_advect;
        h->fresh = fresh; h->have_row_sums = have_row_sums; h->have_particles = have_particles;
        h->adj_ready = adj_ready; h->step = step; h->cell_scale = cell_scale;
    }
};

// Puts a snapshot back and rebuilds the device tables of its grid (cell
// counts at zero, corner tables, realisation table): the arrays only grew,
// so this allocates nothing.
int restore_snapshot(mtpt_handle* h, const HostSnapshot& snap) {
    snap.put(h);
    drop_graph(h);
    if (!h->have_particles) return MTPT_OK;
    if (h->any_transfer) MTPT_TRY(ensure_cells(h));
    return upload_tables(h);
}

int load_particles_body(mtpt_handle* h, const int64_t* counts, const double* pos,
                        const double* mass, cudaMemcpyKind kind, int in_place);

// Loads particles (counts[k] per realisation, concatenated) from host or
// device buffers.  A load that fails before the new particles are in place
// (an allocation, a grid too large) leaves the old state as it was.
int load_particles(mtpt_handle* h, const int64_t* counts, const double* pos, const double* mass,
                   cudaMemcpyKind kind, int in_place = -1) {
    HostSnapshot snap;
    const bool saved = h->have_particles && snap.take(h);
    const int rc = load_particles_body(h, counts, pos, mass, kind, in_place);
    if (rc != MTPT_OK && saved && restore_snapshot(h, snap) != MTPT_OK) {
        h->have_particles = false;   // the old grid's tables could not be rebuilt
        h->n = 0;
    }
    return rc;
}

int load_particles_body(mtpt_handle* h, const int64_t* counts, const double* pos,
                        const double* mass, cudaMemcpyKind kind, int in_place) {
    const int d = h->dim;
    const int64_t held = h->have_particles ? h->n : 0;   // carried over if buffers grow
    int64_t n = 0;
    for (int k = 0; k < h->nreal; ++k) {
        if (counts[k] < 0) return MTPT_ERR_INVALID_ARG;
        n += counts[k];
    }
    if (n > int64_t(0x7fffffff) - kBlock) return MTPT_ERR_INVALID_ARG;
    if (n > 0 && (!pos || !mass)) return MTPT_ERR_INVALID_ARG;
    int64_t off = 0;
    for (int k = 0; k < h->nreal; ++k) {
        h->reals[k].n = counts[k];
        h->params[k].id_offset = uint32_t(off);
        off += counts[k];
    }
    h->n = n;
    MTPT_TRY(ensure_capacity(h, n, held));
    MTPT_TRY(setup_grids(h));
    if (h->any_transfer) MTPT_TRY(ensure_cells(h));
    drop_graph(h);
    if (!h->exp_table.p) {
        MTPT_TRY(h->exp_table.ensure(kExpTable));
        MTPT_CUDA_TRY(cudaMemcpyAsync(h->exp_table.p, exp_table_host(), kExpTable * sizeof(double),
                                      cudaMemcpyHostToDevice, h->stream));
    }
    MTPT_TRY(upload_tables(h));
    // the particles already sit in buffer in_place (positions, masses, ids)
    // when the host load wrote them there
    h->cur = in_place >= 0 ? in_place : 0;
    const int b = h->cur;
    if (n > 0) {
        if (in_place < 0) {
            MTPT_CUDA_TRY(cudaMemcpy2DAsync(h->pos[b].p, size_t(h->cap) * sizeof(double), pos,
                                            size_t(n) * sizeof(double), size_t(n) * sizeof(double),
                                            d, kind, h->stream));
            MTPT_CUDA_TRY(cudaMemcpyAsync(h->mass[b].p, mass, size_t(n) * sizeof(double), kind,
                                          h->stream));
            k_iota<<<grid_for(n), kBlock, 0, h->stream>>>(int(n), h->id[b].p);
            MTPT_CUDA_TRY(cudaGetLastError());
        }
        if (h->batch) {
            k_fill_rid<<<grid_for(n), kBlock, 0, h->stream>>>(int(n), h->nreal, h->id_first.p,
                                                             h->rid[b].p);
            MTPT_CUDA_TRY(cudaGetLastError());
        }
    }
    MTPT_CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(uint32_t), h->stream));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->pair_counter.p, 0, sizeof(unsigned long long), h->stream));
    MTPT_TRY(set_step_dev(h, 0));
    h->have_row_sums = false;
    h->walked_ahead = false;
    h->have_particles = true;
    h->adj_ready = false;
    h->fresh = true;
    // species B starts at zero on newly loaded particles
    if (h->reactive && n > 0)
        MTPT_CUDA_TRY(cudaMemsetAsync(h->massb[b].p, 0, size_t(n) * sizeof(double), h->stream));
    return MTPT_OK;
}

// Host loads are copied to the device and checked there (k_check_input:
// positions inside their realisation's box, masses finite and, in the
// precision form, at most 1e30 in magnitude) before the handle's state is
// touched, so a rejected load leaves the old state in place.  When the
// handle's capacity already holds n particles the copy goes straight into the
// free half of the state double buffer (which becomes current on success,
// *in_place set to its index, ids written by the check); otherwise into a
// staging area, and *pos_dev / *mass_dev point at it (positions dim x n).
int stage_host_particles(mtpt_handle* h, const int64_t* counts, const double* pos,
                         const double* mass, const double** pos_dev, const double** mass_dev,
                         int* in_place) {
    int64_t n = 0;
    for (int k = 0; k < h->nreal; ++k) {
        if (counts[k] < 0) return MTPT_ERR_INVALID_ARG;
        n += counts[k];
    }
    if (n > int64_t(0x7fffffff) - kBlock) return MTPT_ERR_INVALID_ARG;
    if (n > 0 && (!pos || !mass)) return MTPT_ERR_INVALID_ARG;
    *pos_dev = nullptr;
    *mass_dev = nullptr;
    *in_place = -1;
    if (n == 0) return MTPT_OK;
    const int d = h->dim;
    MTPT_TRY(h->chk_flag.ensure(1));
    if (!h->chk_box.p) {
        std::vector<double> box(size_t(6) * size_t(h->nreal), 0.0);
        for (int k = 0; k < h->nreal; ++k)
            for (int a = 0; a < d; ++a) {
                box[size_t(6) * k + a] = h->reals[k].prm.lo[a];
                box[size_t(6) * k + 3 + a] = h->reals[k].prm.hi[a];
            }
        MTPT_TRY(h->chk_box.ensure(box.size()));
        MTPT_CUDA_TRY(cudaMemcpyAsync(h->chk_box.p, box.data(), box.size() * sizeof(double),
                                      cudaMemcpyHostToDevice, h->stream));
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    if (h->nreal > 1) {
        std::vector<uint32_t> first(size_t(h->nreal) + 1, 0u);
        for (int k = 0; k < h->nreal; ++k) first[k + 1] = first[k] + uint32_t(counts[k]);
        MTPT_TRY(h->chk_first.ensure(first.size()));
        MTPT_CUDA_TRY(cudaMemcpyAsync(h->chk_first.p, first.data(), first.size() * sizeof(uint32_t),
                                      cudaMemcpyHostToDevice, h->stream));
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));   // `first` is a local
    }
    const int f = 1 - h->cur;
    const bool direct = n <= h->cap && h->pos[f].p && h->mass[f].p && h->id[f].p;
    double* sp;
    double* sm;
    int64_t stride;
    if (direct) {
        sp = h->pos[f].p;
        sm = h->mass[f].p;
        stride = h->cap;
        MTPT_CUDA_TRY(cudaMemcpy2DAsync(sp, size_t(stride) * sizeof(double), pos,
                                        size_t(n) * sizeof(double), size_t(n) * sizeof(double), d,
                                        cudaMemcpyHostToDevice, h->stream));
    } else {
        MTPT_TRY(h->stage.ensure(size_t(d + 1) * size_t(n)));
        sp = h->stage.p;
        sm = h->stage.p + size_t(d) * size_t(n);
        stride = n;
        MTPT_CUDA_TRY(cudaMemcpyAsync(sp, pos, size_t(d) * size_t(n) * sizeof(double),
                                      cudaMemcpyHostToDevice, h->stream));
    }
    MTPT_CUDA_TRY(cudaMemcpyAsync(sm, mass, size_t(n) * sizeof(double), cudaMemcpyHostToDevice,
                                  h->stream));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->chk_flag.p, 0, sizeof(uint32_t), h->stream));
    const double mass_limit = h->precision == MTPT_FP32W ? 1e30 : HUGE_VAL;
    uint32_t* ids = direct ? h->id[f].p : nullptr;
    switch (d) {
        case 1: k_check_input<1><<<grid_for(n), kBlock, 0, h->stream>>>(
                    int(n), stride, h->nreal, sp, sm, h->chk_box.p, h->chk_first.p, mass_limit,
                    h->chk_flag.p, ids);
                break;
        case 2: k_check_input<2><<<grid_for(n), kBlock, 0, h->stream>>>(
                    int(n), stride, h->nreal, sp, sm, h->chk_box.p, h->chk_first.p, mass_limit,
                    h->chk_flag.p, ids);
                break;
        default: k_check_input<3><<<grid_for(n), kBlock, 0, h->stream>>>(
                    int(n), stride, h->nreal, sp, sm, h->chk_box.p, h->chk_first.p, mass_limit,
                    h->chk_flag.p, ids);
                break;
    }
    MTPT_CUDA_TRY(cudaGetLastError());
    uint32_t flag = 0;
    MTPT_CUDA_TRY(cudaMemcpyAsync(&flag, h->chk_flag.p, sizeof(flag), cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (flag & 1u) return MTPT_ERR_OUT_OF_DOMAIN;
    if (flag & 2u) return MTPT_ERR_INVALID_ARG;
    *pos_dev = sp;
    *mass_dev = sm;
    if (direct) *in_place = f;
    return MTPT_OK;
}

// Streams, events and staging slots of the pipelined host I/O, made on first
// use and grown with n.  Growing a slot waits for every copy in flight first
// (a copy may still read or write the old allocation).
int ensure_async(mtpt_handle* h) {
    if (!h->h2d) MTPT_CUDA_TRY(cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking));
    if (!h->d2h) MTPT_CUDA_TRY(cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking));
    for (int s = 0; s < 2; ++s) {
        cudaEvent_t* evs[4] = {&h->in_ready[s], &h->in_free[s], &h->out_ready[s], &h->out_free[s]};
        for (cudaEvent_t* e : evs)
            if (!*e) MTPT_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    const size_t n = size_t(std::max<int64_t>(h->n, 1));
    const size_t in_need = size_t(h->dim + 1) * n;
    if (h->in_slot[0].count < in_need || h->in_slot[1].count < in_need ||
        h->out_slot[0].count < n || h->out_slot[1].count < n) {
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->h2d));
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->d2h));
        for (int s = 0; s < 2; ++s) {
            MTPT_TRY(h->in_slot[s].ensure(in_need));
            MTPT_TRY(h->out_slot[s].ensure(n));
        }
    }
    MTPT_TRY(h->in_flag.ensure(2));
    if (!h->chk_box.p) {
        double box[6] = {0, 0, 0, 0, 0, 0};
        for (int a = 0; a < h->dim; ++a) {
            box[a] = h->reals[0].prm.lo[a];
            box[3 + a] = h->reals[0].prm.hi[a];
        }
        MTPT_TRY(h->chk_box.ensure(6));
        MTPT_CUDA_TRY(cudaMemcpyAsync(h->chk_box.p, box, sizeof(box), cudaMemcpyHostToDevice,
                                      h->stream));
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));   // `box` is a local
    }
    return MTPT_OK;
}

void release_async(mtpt_handle* h) {
    if (h->h2d) cudaStreamSynchronize(h->h2d);
    if (h->d2h) cudaStreamSynchronize(h->d2h);
    for (int s = 0; s < 2; ++s) {
        cudaEvent_t* evs[4] = {&h->in_ready[s], &h->in_free[s], &h->out_ready[s], &h->out_free[s]};
        for (cudaEvent_t* e : evs) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
        h->in_slot[s].release();
        h->out_slot[s].release();
    }
    h->in_flag.release();
    if (h->h2d) cudaStreamDestroy(h->h2d);
    if (h->d2h) cudaStreamDestroy(h->d2h);
    h->h2d = h->d2h = nullptr;
}

template <int DIM>
int launch_load_async(mtpt_handle* h, int slot, int f) {
    const int n = int(h->n);
    const int c = h->cur;
    const double mass_limit = h->precision == MTPT_FP32W ? 1e30 : HUGE_VAL;
    uint32_t* flag = h->in_flag.p + slot;
    MTPT_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(uint32_t), h->stream));
    {
        MTPT_TIMED(h, "load_input");
        k_load_input<DIM><<<grid_for(n), kBlock, 0, h->stream>>>(
            n, h->in_slot[slot].p, h->chk_box.p, mass_limit, flag, h->cap, h->pos[f].p,
            h->mass[f].p, h->id[f].p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    {
        MTPT_TIMED(h, "load_settle");
        k_load_settle<DIM><<<std::min(grid_for(n), kSettleBlocks), kBlock, 0, h->stream>>>(
            n, h->cap, flag, h->pos[c].p, h->mass[c].p, h->id[c].p, h->pos[f].p, h->mass[f].p,
            h->id[f].p, h->status.p, h->step_dev.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    if (h->batch) {
        // one realisation: every rid is 0, whichever state the settle kept
        k_fill_rid<<<grid_for(n), kBlock, 0, h->stream>>>(n, h->nreal, h->id_first.p,
                                                         h->rid[f].p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    return MTPT_OK;
}

int create_common(const mtpt_params* params, int count, bool batch, mtpt_handle** out) {
    if (!out) return MTPT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || count < 1 || count > (1 << 20)) return MTPT_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k) {
        MTPT_TRY(validate_params(params + k));
        if (params[k].dim != params[0].dim || params[k].precision != params[0].precision)
            return MTPT_ERR_INVALID_ARG;
    }
    mtpt_handle* h = new (std::nothrow) mtpt_handle();
    if (!h) return MTPT_ERR_NO_MEMORY;
    h->dim = params[0].dim;
    h->precision = params[0].precision;
    h->batch = batch;
    h->nreal = count;
    if (count > 1) {
        try {
            h->real_heap.resize(size_t(count));
            h->params_heap.resize(size_t(count));
        } catch (...) {
            delete h;
            return MTPT_ERR_NO_MEMORY;
        }
        h->reals = h->real_heap.data();
        h->params = h->params_heap.data();
    }
    for (int k = 0; k < count; ++k) {
        h->reals[k].prm = params[k];
        derive(h->reals[k], h->params[k]);
    }
    *out = h;
    return MTPT_OK;
}

void fill_info(const mtpt_handle* h, int k, mtpt_info* out) {
    const RealHost& R = h->reals[k];
    const RealParams& P = h->params[k];
    out->D_RW = R.D_RW;
    out->D_MT = R.D_MT;
    out->sigma = P.sigma;
    out->h2 = R.h2;
    out->psi = R.psi;
    out->psi2 = R.psi2;
    out->kernel_norm = P.kernel_norm;
    for (int a = 0; a < 3; ++a) {
        out->cells[a] = P.g.n[a] ? P.g.n[a] : 1;
        out->cell_width[a] = P.g.w[a];
    }
}

template <int DIM, class View>
int launch_emit(mtpt_handle* h, int64_t cap) {
    const int n = int(h->n);
    const int blocks = grid_for(n);
    const int64_t stride = h->cap;
    const int c = h->cur, o = 1 - h->cur;
    const View vin = make_view<View>(h, c, c);
    k_walk_key<DIM, View><<<blocks, kBlock, 0, h->stream>>>(n, stride, h->pos[c].p, h->id[c].p,
                                                            h->step_dev.p, 0, 1, vin, h->key.p,
                                                            h->count.p, h->status.p);
    MTPT_TRY(launch_scan(h, h->stream, false));
    MTPT_TRY((launch_sort<DIM, View>(h, c, o, vin)));
    const View vs = make_view<View>(h, o, o);
    k_emit_pairs<DIM, View><<<blocks, kBlock, 0, h->stream>>>(
        n, stride, h->pos[o].p, h->rec.p, h->cell.p, h->start.p, h->id[o].p, vs,
        (unsigned long long)cap, h->emit_counter.p, h->emit_i.p, h->emit_j.p);
    MTPT_CUDA_TRY(cudaGetLastError());
    // the gathered copy in o is the same state in cell order: make it current
    h->cur = o;
    h->have_row_sums = false;
    h->walked_ahead = false;
    return MTPT_OK;
}

int dispatch_emit(mtpt_handle* h, int64_t cap) {
    if (h->batch) {
        switch (h->dim) {
            case 1: return launch_emit<1, BatchView>(h, cap);
            case 2: return launch_emit<2, BatchView>(h, cap);
            default: return launch_emit<3, BatchView>(h, cap);
        }
    }
    switch (h->dim) {
        case 1: return launch_emit<1, SingleView>(h, cap);
        case 2: return launch_emit<2, SingleView>(h, cap);
        default: return launch_emit<3, SingleView>(h, cap);
    }
}

template <class View, class T>
int launch_row_sums_out(mtpt_handle* h, const T* src, int src_step) {
    const View v = make_view<View>(h, h->cur, h->cur);
    k_row_sums_out<T, View><<<grid_for(h->n), kBlock, 0, h->stream>>>(
        int(h->n), h->id[h->cur].p, src, src_step, v, h->out_tmp.p);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

template <int DIM, class View>
int launch_check_domain(mtpt_handle* h) {
    const View v = make_view<View>(h, 0, 0);
    k_check_domain<DIM, View><<<grid_for(h->n), kBlock, 0, h->stream>>>(int(h->n), h->cap,
                                                                      h->pos[0].p, v,
                                                                      h->status.p);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}

// --- adjoint -----------------------------------------------------------------

size_t snap_size(const mtpt_handle* h) {
    const size_t n = size_t(h->n), d = size_t(h->dim);
    return 2 * d * n * sizeof(double) + n * sizeof(double) + n * sizeof(uint32_t) + 64;
}

// Copies the current state (positions, tangents, masses, ids of buffer cur)
// into snapshot slot k, or back into buffer 0 (then current).
int snapshot(mtpt_handle* h, int64_t k, bool save) {
    const size_t n = size_t(h->n), d = size_t(h->dim);
    if (n == 0) return MTPT_OK;
    unsigned char* base = h->snaps.p + size_t(k) * h->snap_bytes;
    double* spos = reinterpret_cast<double*>(base);
    double* stan = spos + d * n;
    double* smass = stan + d * n;
    uint32_t* sid = reinterpret_cast<uint32_t*>(smass + n);
    const size_t pitch = size_t(h->cap) * sizeof(double), row = n * sizeof(double);
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    if (save) {
        const int c = h->cur;
        MTPT_CUDA_TRY(cudaMemcpy2DAsync(spos, row, h->pos[c].p, pitch, row, d, dd, h->stream));
        MTPT_CUDA_TRY(cudaMemcpy2DAsync(stan, row, h->tan[c].p, pitch, row, d, dd, h->stream));
        MTPT_CUDA_TRY(cudaMemcpyAsync(smass, h->mass[c].p, row, dd, h->stream));
        MTPT_CUDA_TRY(cudaMemcpyAsync(sid, h->id[c].p, n * sizeof(uint32_t), dd, h->stream));
    } else {
        h->cur = 0;
        MTPT_CUDA_TRY(cudaMemcpy2DAsync(h->pos[0].p, pitch, spos, row, row, d, dd, h->stream));
        MTPT_CUDA_TRY(cudaMemcpy2DAsync(h->tan[0].p, pitch, stan, row, row, d, dd, h->stream));
        MTPT_CUDA_TRY(cudaMemcpyAsync(h->mass[0].p, smass, row, dd, h->stream));
        MTPT_CUDA_TRY(cudaMemcpyAsync(h->id[0].p, sid, n * sizeof(uint32_t), dd, h->stream));
    }
    return MTPT_OK;
}

// One backward step: walk (with tangents) and sort exactly as forward step t
// did, then the adjoint passes, lambda kept in input order between steps.
template <int DIM>
int launch_adjoint_step(mtpt_handle* h) {
    const int n = int(h->n);
    const int64_t stride = h->cap;
    const int blocks = grid_for(n);
    cudaStream_t st = h->stream;
    const int c = h->cur, o = 1 - h->cur;
    const SingleView v = make_view<SingleView>(h, c, c);
    if (h->any_advect)
        k_walk_key<DIM, SingleView, true, true><<<blocks, kBlock, 0, st>>>(
            n, stride, h->pos[c].p, h->id[c].p, h->step_dev.p, h->any_walk ? 1 : 0, 1, v,
            h->key.p, h->count.p, h->status.p, h->tan[c].p);
    else
        k_walk_key<DIM, SingleView, true><<<blocks, kBlock, 0, st>>>(
            n, stride, h->pos[c].p, h->id[c].p, h->step_dev.p, h->any_walk ? 1 : 0, 1, v,
            h->key.p, h->count.p, h->status.p, h->tan[c].p);
    MTPT_TRY(launch_scan(h, st, true));
    MTPT_TRY((launch_sort<DIM, SingleView>(h, c, o, v)));
    k_take_by_id<<<blocks, kBlock, 0, st>>>(n, h->id[o].p, h->lam_in.p, h->lam_s.p);
    const NbList<double2> adj_nb{h->adj_nb_j.p, h->adj_nb_k.p, h->adj_nb_count.p,
                                 h->adj_nb_k.p ? h->adj_cap : 0};
    k_adj_rowsum<DIM, SingleView><<<blocks, kBlock, 0, st>>>(
        n, stride, h->pos[o].p, h->tan[o].p, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, v,
        h->r64.p, h->dr64.p, adj_nb);
    k_adj_exchange<DIM, SingleView><<<blocks, kBlock, 0, st>>>(
        n, stride, h->pos[o].p, h->tan[o].p, h->rec.p, h->cell.p, h->start.p, h->exp_table.p, v,
        h->r64.p, h->dr64.p, h->mass[o].p, h->lam_s.p, h->lam_new.p, h->gD.p, adj_nb);
    k_put_by_id<<<blocks, kBlock, 0, st>>>(n, h->id[o].p, h->lam_new.p, h->lam_in.p);
    const int nparts = (n + kReduceThreads - 1) / kReduceThreads;
    k_block_sums<<<nparts, kReduceThreads, 0, st>>>(n, h->gD.p, h->partial.p);
    k_sum_into<<<1, kReduceThreads, 0, st>>>(nparts, h->partial.p, h->acc.p);
    MTPT_CUDA_TRY(cudaGetLastError());
    h->cur = o;
    return MTPT_OK;
}

int dispatch_adjoint_step(mtpt_handle* h) {
    switch (h->dim) {
        case 1: return launch_adjoint_step<1>(h);
        case 2: return launch_adjoint_step<2>(h);
        default: return launch_adjoint_step<3>(h);
    }
}

}  // namespace

extern "C" {

int mtpt_adjoint_forward(mtpt_handle* h, int64_t nsteps, int64_t checkpoint_every) {
    if (!h || nsteps < 1 || checkpoint_every < 1) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles || h->ntiles > 0 || h->reactive) return MTPT_ERR_STATE;
    if (h->nreal != 1 || !h->any_transfer || !(h->reals[0].prm.D > 0.0)) return MTPT_ERR_INVALID_ARG;
    const int64_t n = h->n;
    const size_t cap = size_t(std::max<int64_t>(h->cap, 1));
    for (int b = 0; b < 2; ++b) MTPT_TRY(h->tan[b].ensure(size_t(h->dim) * cap));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->tan[h->cur].p, 0, size_t(h->dim) * cap * sizeof(double), h->stream));
    const int64_t nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
    const int64_t seg = std::min(checkpoint_every, nsteps);
    h->snap_bytes = (snap_size(h) + 255) & ~size_t(255);
    MTPT_TRY(h->snaps.ensure(size_t(nck + seg + 1) * h->snap_bytes));
    for (auto* b : {&h->dr64, &h->lam_in, &h->lam_s, &h->lam_new, &h->gD})
        MTPT_TRY(b->ensure(cap));
    MTPT_TRY(h->r64.ensure(cap));
    if (h->adj_cap > 0) {
        MTPT_TRY(h->adj_nb_j.ensure(size_t(h->adj_cap) * cap));
        MTPT_TRY(h->adj_nb_k.ensure(size_t(h->adj_cap) * cap));
        MTPT_TRY(h->adj_nb_count.ensure(cap));
    }
    MTPT_TRY(h->partial.ensure(size_t((n + kReduceThreads - 1) / kReduceThreads + 1)));
    MTPT_TRY(h->acc.ensure(1));
    h->tangent_on = true;
    h->adj_step0 = h->step;
    int rc = MTPT_OK;
    for (int64_t t = 0; t < nsteps && rc == MTPT_OK; ++t) {
        if (t % checkpoint_every == 0) rc = snapshot(h, t / checkpoint_every, true);
        if (rc == MTPT_OK) rc = dispatch_step(h, MTPT_DO_WALK | MTPT_DO_TRANSFER);
    }
    if (rc == MTPT_OK) rc = snapshot(h, nck + seg, true);   // final state
    h->tangent_on = false;
    if (rc != MTPT_OK) return rc;
    h->step += uint64_t(nsteps);
    h->adj_steps = nsteps;
    h->adj_every = checkpoint_every;
    h->adj_nck = nck;
    h->adj_ready = true;
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MTPT_OK;
}

int mtpt_adjoint_backward(mtpt_handle* h, const double* gmass_dev, double* gmass0_dev,
                          double* dldD) {
    if (!h || (h->n > 0 && (!gmass_dev || !gmass0_dev)) || !dldD) return MTPT_ERR_INVALID_ARG;
    if (!h->adj_ready) return MTPT_ERR_STATE;
    const int64_t n = h->n, K = h->adj_every, T = h->adj_steps, nck = h->adj_nck;
    const int64_t seg = std::min(K, T);
    const int64_t final_slot = nck + seg;
    MTPT_CUDA_TRY(cudaMemcpyAsync(h->lam_in.p, gmass_dev, size_t(n) * sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->stream));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->acc.p, 0, sizeof(double), h->stream));
    drop_graph(h);
    h->tangent_on = true;
    int rc = MTPT_OK;
    for (int64_t k = nck - 1; k >= 0 && rc == MTPT_OK; --k) {
        const int64_t t0 = k * K, t1 = std::min(t0 + K, T);
        // forward over the segment from its checkpoint, recording the state
        // before every step on the tape
        rc = snapshot(h, k, false);
        if (rc == MTPT_OK) rc = set_step_dev(h, h->adj_step0 + uint64_t(t0));
        for (int64_t t = t0; t < t1 && rc == MTPT_OK; ++t) {
            rc = snapshot(h, nck + (t - t0), true);
            if (rc == MTPT_OK && t + 1 < t1) rc = dispatch_step(h, MTPT_DO_WALK | MTPT_DO_TRANSFER);
        }
        // backward through the tape
        for (int64_t t = t1 - 1; t >= t0 && rc == MTPT_OK; --t) {
            rc = snapshot(h, nck + (t - t0), false);
            if (rc == MTPT_OK) rc = set_step_dev(h, h->adj_step0 + uint64_t(t));
            if (rc == MTPT_OK) rc = dispatch_adjoint_step(h);
        }
    }
    h->tangent_on = false;
    // leave the handle in its final forward state
    if (rc == MTPT_OK) rc = snapshot(h, final_slot, false);
    if (rc == MTPT_OK) rc = set_step_dev(h, h->adj_step0 + uint64_t(T));
    h->have_row_sums = false;
    h->walked_ahead = false;
    if (rc != MTPT_OK) return rc;
    MTPT_CUDA_TRY(cudaMemcpyAsync(gmass0_dev, h->lam_in.p, size_t(n) * sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->stream));
    MTPT_CUDA_TRY(cudaMemcpyAsync(dldD, h->acc.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return read_status(h);
}

int mtpt_check_word(uint32_t* out, int32_t reset) {
    if (!out) return MTPT_ERR_INVALID_ARG;
    *out = 0;
#ifdef MTPT_CHECKED
    MTPT_CUDA_TRY(cudaDeviceSynchronize());
    MTPT_CUDA_TRY(cudaMemcpyFromSymbol(out, g_check_word, sizeof(uint32_t)));
    if (reset) {
        const uint32_t zero = 0;
        MTPT_CUDA_TRY(cudaMemcpyToSymbol(g_check_word, &zero, sizeof(uint32_t)));
    }
    return MTPT_OK;
#else
    (void)reset;
    return MTPT_ERR_STATE;
#endif
}

int mtpt_create(const mtpt_params* params, mtpt_handle** out) {
    return create_common(params, 1, false, out);
}

int mtpt_create_batch(const mtpt_params* params, int32_t count, mtpt_handle** out) {
    return create_common(params, count, true, out);
}

int mtpt_destroy(mtpt_handle* h) {
    if (!h) return MTPT_OK;
    cudaStreamSynchronize(h->stream);
    release_async(h);
    drop_graph(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (int b = 0; b < 2; ++b) {
        h->pos[b].release();
        h->mass[b].release();
        h->id[b].release();
        h->rid[b].release();
    }
    h->key.release(); h->perm.release(); h->sortkey.release(); h->sortrec.release(); h->cell.release(); h->count.release();
    h->start.release(); h->scan_state.release(); h->rec.release(); h->corners.release();
    h->corner_first.release(); h->id_first.release(); h->params_dev.release();
    h->r64.release(); h->ex.release(); h->out_tmp.release();
    h->exp_table.release();
    h->stage.release(); h->chk_box.release(); h->chk_first.release(); h->chk_flag.release();
    h->status.release(); h->pair_counter.release(); h->step_dev.release();
    h->emit_counter.release(); h->emit_i.release(); h->emit_j.release();
    h->tan[0].release(); h->tan[1].release(); h->snaps.release(); h->dr64.release();
    h->lam_in.release(); h->lam_s.release(); h->lam_new.release(); h->gD.release();
    h->partial.release(); h->acc.release();
    h->nb_j.release(); h->nb_k.release(); h->nb_count.release();
    h->nb32_e.release();
    h->massb[0].release(); h->massb[1].release(); h->exb.release();
    h->adj_nb_j.release(); h->adj_nb_k.release(); h->adj_nb_count.release();
    h->tile_counts.release(); h->tile_base.release(); h->tile_cursor.release();
    h->tile_native.release(); h->tile_flag.release(); h->tile_keep.release();
    h->tile_stage.release(); h->tile_tables_dev.release();
    for (auto& pe : h->pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (auto e : h->spare_events) cudaEventDestroy(e);
    delete h;
    return MTPT_OK;
}

int mtpt_set_stream(mtpt_handle* h, void* stream) {
    if (!h) return MTPT_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return MTPT_OK;
}

int mtpt_set_particles(mtpt_handle* h, int64_t n, const double* pos, const double* mass) {
    if (!h || h->nreal != 1) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles > 0) return MTPT_ERR_STATE;
    if (n < 0) return MTPT_ERR_INVALID_ARG;
    const double *pd = nullptr, *md = nullptr;
    int in_place = -1;
    MTPT_TRY(stage_host_particles(h, &n, pos, mass, &pd, &md, &in_place));
    return load_particles(h, &n, pd, md, cudaMemcpyDeviceToDevice, in_place);
}

int mtpt_set_particles_batch(mtpt_handle* h, const int64_t* counts, const double* pos,
                             const double* mass) {
    if (!h || !counts) return MTPT_ERR_INVALID_ARG;
    const double *pd = nullptr, *md = nullptr;
    int in_place = -1;
    MTPT_TRY(stage_host_particles(h, counts, pos, mass, &pd, &md, &in_place));
    return load_particles(h, counts, pd, md, cudaMemcpyDeviceToDevice, in_place);
}

int mtpt_set_particles_device(mtpt_handle* h, int64_t n, const double* pos_dev,
                              const double* mass_dev) {
    if (!h || h->nreal != 1 || n < 0) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles > 0) return MTPT_ERR_STATE;
    MTPT_TRY(load_particles(h, &n, pos_dev, mass_dev, cudaMemcpyDeviceToDevice));
    if (n > 0) {
        if (h->batch) {
            switch (h->dim) {
                case 1: MTPT_TRY((launch_check_domain<1, BatchView>(h))); break;
                case 2: MTPT_TRY((launch_check_domain<2, BatchView>(h))); break;
                default: MTPT_TRY((launch_check_domain<3, BatchView>(h))); break;
            }
        } else {
            switch (h->dim) {
                case 1: MTPT_TRY((launch_check_domain<1, SingleView>(h))); break;
                case 2: MTPT_TRY((launch_check_domain<2, SingleView>(h))); break;
                default: MTPT_TRY((launch_check_domain<3, SingleView>(h))); break;
            }
        }
    }
    return MTPT_OK;
}

int mtpt_step_ex(mtpt_handle* h, int64_t nsteps, int32_t flags) {
    if (!h || nsteps < 0) return MTPT_ERR_INVALID_ARG;
    if (flags & ~(MTPT_DO_WALK | MTPT_DO_TRANSFER)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    // a tile's transfer needs its ghosts: mtpt_tile_pack / mtpt_tile_transfer
    if (h->ntiles > 0 && (flags & MTPT_DO_TRANSFER)) return MTPT_ERR_STATE;
    if (h->ntiles > 0) h->keep_ready = false;
    return run_steps(h, nsteps, flags);
}

int mtpt_step(mtpt_handle* h, int64_t nsteps) {
    return mtpt_step_ex(h, nsteps, MTPT_DO_WALK | MTPT_DO_TRANSFER);
}

int mtpt_get_masses_device(mtpt_handle* h, double* out_dev) {
    if (!h || (!out_dev && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    return unpermute_to(h, h->mass[h->cur].p, 1, out_dev);
}

int mtpt_get_masses(mtpt_handle* h, double* out) {
    if (!h || (!out && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    MTPT_TRY(ensure_out_tmp(h));
    MTPT_TRY(unpermute_to(h, h->mass[h->cur].p, 1, h->out_tmp.p));
    return copy_out_host(h, 1, out);
}

int mtpt_set_particles_async(mtpt_handle* h, int64_t n, const double* pos, const double* mass) {
    if (!h || h->nreal != 1) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles > 0) return MTPT_ERR_STATE;
    if (!h->have_particles) return MTPT_ERR_STATE;
    if (n != h->n || (n > 0 && (!pos || !mass))) return MTPT_ERR_INVALID_ARG;
    if (n == 0) return MTPT_OK;
    MTPT_TRY(ensure_async(h));
    const int slot = h->in_next;
    const int d = h->dim;
    double* dst = h->in_slot[slot].p;
    // the slot is free once the load that used it last has been checked
    MTPT_CUDA_TRY(cudaStreamWaitEvent(h->h2d, h->in_free[slot], 0));
    MTPT_CUDA_TRY(cudaMemcpyAsync(dst, pos, size_t(d) * size_t(n) * sizeof(double),
                                  cudaMemcpyHostToDevice, h->h2d));
    MTPT_CUDA_TRY(cudaMemcpyAsync(dst + size_t(d) * size_t(n), mass, size_t(n) * sizeof(double),
                                  cudaMemcpyHostToDevice, h->h2d));
    MTPT_CUDA_TRY(cudaEventRecord(h->in_ready[slot], h->h2d));
    MTPT_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->in_ready[slot], 0));
    const int f = 1 - h->cur;
    switch (d) {
        case 1: MTPT_TRY(launch_load_async<1>(h, slot, f)); break;
        case 2: MTPT_TRY(launch_load_async<2>(h, slot, f)); break;
        default: MTPT_TRY(launch_load_async<3>(h, slot, f)); break;
    }
    MTPT_CUDA_TRY(cudaEventRecord(h->in_free[slot], h->stream));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->pair_counter.p, 0, sizeof(unsigned long long), h->stream));
    if (h->reactive)                  // species B starts at zero on the new particles
        MTPT_CUDA_TRY(cudaMemsetAsync(h->massb[f].p, 0, size_t(n) * sizeof(double), h->stream));
    h->in_next = 1 - slot;
    h->cur = f;
    h->step = 0;
    h->have_row_sums = false;
    h->walked_ahead = false;
    h->adj_ready = false;
    h->fresh = true;
    return MTPT_OK;
}

int mtpt_get_masses_async(mtpt_handle* h, double* out) {
    if (!h || (!out && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    if (h->n == 0) return MTPT_OK;
    MTPT_TRY(ensure_async(h));
    const int slot = h->out_next;
    // the slot is free once the copy that read it last has finished
    MTPT_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->out_free[slot], 0));
    MTPT_TRY(unpermute_to(h, h->mass[h->cur].p, 1, h->out_slot[slot].p));
    MTPT_CUDA_TRY(cudaEventRecord(h->out_ready[slot], h->stream));
    MTPT_CUDA_TRY(cudaStreamWaitEvent(h->d2h, h->out_ready[slot], 0));
    MTPT_CUDA_TRY(cudaMemcpyAsync(out, h->out_slot[slot].p, size_t(h->n) * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->d2h));
    MTPT_CUDA_TRY(cudaEventRecord(h->out_free[slot], h->d2h));
    h->out_next = 1 - slot;
    return MTPT_OK;
}

int mtpt_get_positions_device(mtpt_handle* h, double* out_dev) {
    if (!h || (!out_dev && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    return unpermute_to(h, h->pos[h->cur].p, h->dim, out_dev);
}

int mtpt_get_positions(mtpt_handle* h, double* out) {
    if (!h || (!out && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    MTPT_TRY(ensure_out_tmp(h));
    MTPT_TRY(unpermute_to(h, h->pos[h->cur].p, h->dim, h->out_tmp.p));
    return copy_out_host(h, h->dim, out);
}

int mtpt_get_row_sums(mtpt_handle* h, double* out) {
    if (!h || (!out && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles || !h->have_row_sums) return MTPT_ERR_STATE;
    MTPT_TRY(ensure_out_tmp(h));
    if (h->n > 0) {
        if (h->precision == MTPT_FP64) {
            if (h->batch) MTPT_TRY((launch_row_sums_out<BatchView, double>(h, h->r64.p, 1)));
            else MTPT_TRY((launch_row_sums_out<SingleView, double>(h, h->r64.p, 1)));
        } else {
            const float* r = reinterpret_cast<const float*>(h->ex.p) + 2;   // ex[s].z
            if (h->batch) MTPT_TRY((launch_row_sums_out<BatchView, float>(h, r, 4)));
            else MTPT_TRY((launch_row_sums_out<SingleView, float>(h, r, 4)));
        }
    }
    return copy_out_host(h, 1, out);
}

int mtpt_get_pairs(mtpt_handle* h, int64_t cap, int64_t* count, uint32_t* pair_i,
                   uint32_t* pair_j) {
    if (!h || !count || cap < 0 || (cap > 0 && (!pair_i || !pair_j))) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles || h->ntiles > 0) return MTPT_ERR_STATE;
    *count = 0;
    if (h->n == 0 || !h->any_transfer) return read_status(h);
    MTPT_TRY(h->emit_counter.ensure(1));
    const size_t ecap = size_t(std::max<int64_t>(cap, 1));
    MTPT_TRY(h->emit_i.ensure(ecap));
    MTPT_TRY(h->emit_j.ensure(ecap));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->emit_counter.p, 0, sizeof(unsigned long long), h->stream));
    // Re-sort the current positions (no walk, no transfer) so the cell list
    // describes them, then emit every accepted pair.
    MTPT_TRY(dispatch_emit(h, cap));
    unsigned long long total = 0;
    MTPT_CUDA_TRY(cudaMemcpyAsync(&total, h->emit_counter.p, sizeof(total), cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    *count = int64_t(total);
    const int64_t ncopy = std::min<int64_t>(int64_t(total), cap);
    if (ncopy > 0) {
        MTPT_CUDA_TRY(cudaMemcpy(pair_i, h->emit_i.p, size_t(ncopy) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        MTPT_CUDA_TRY(cudaMemcpy(pair_j, h->emit_j.p, size_t(ncopy) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    }
    MTPT_TRY(read_status(h));
    return int64_t(total) > cap ? MTPT_ERR_CAPACITY : MTPT_OK;
}

int mtpt_get_info(mtpt_handle* h, mtpt_info* out) {
    if (!h || !out) return MTPT_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->step = h->step;
    if (h->pair_counter.p) {
        unsigned long long pc = 0;
        MTPT_CUDA_TRY(cudaMemcpyAsync(&pc, h->pair_counter.p, sizeof(pc), cudaMemcpyDeviceToHost, h->stream));
        MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
        out->pair_count = pc;
    }
    fill_info(h, 0, out);
    return h->status.p ? read_status(h) : MTPT_OK;
}

int mtpt_get_realisation_info(mtpt_handle* h, int32_t k, mtpt_info* out) {
    if (!h || !out || k < 0 || k >= h->nreal) return MTPT_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = h->reals[k].n;
    out->step = h->step;
    fill_info(h, k, out);
    return MTPT_OK;
}

int mtpt_set_step(mtpt_handle* h, uint64_t step) {
    if (!h) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) {
        h->step = step;
        return MTPT_OK;
    }
    return set_step_dev(h, step);
}

int mtpt_sync(mtpt_handle* h) {
    if (!h) return MTPT_ERR_INVALID_ARG;
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->h2d) MTPT_CUDA_TRY(cudaStreamSynchronize(h->h2d));
    if (h->d2h) MTPT_CUDA_TRY(cudaStreamSynchronize(h->d2h));
    return h->status.p ? read_status(h) : MTPT_OK;
}

int mtpt_timing_enable(mtpt_handle* h, int32_t on) {
    if (!h) return MTPT_ERR_INVALID_ARG;
    h->timing = on != 0;
    return MTPT_OK;
}

int mtpt_timing_read(mtpt_handle* h, int32_t cap, mtpt_kernel_stat* out, int32_t* count) {
    if (!h || !count || cap < 0 || (cap > 0 && !out)) return MTPT_ERR_INVALID_ARG;
    MTPT_TRY(fold_timing(h));
    *count = int32_t(h->stats.size());
    for (int32_t k = 0; k < cap && k < *count; ++k) {
        std::memset(&out[k], 0, sizeof(out[k]));
        std::strncpy(out[k].name, h->stats[k].name, sizeof(out[k].name) - 1);
        out[k].launches = h->stats[k].launches;
        out[k].total_ms = h->stats[k].total_ms;
    }
    return MTPT_OK;
}

int mtpt_timing_reset(mtpt_handle* h) {
    if (!h) return MTPT_ERR_INVALID_ARG;
    MTPT_TRY(fold_timing(h));
    h->stats.clear();
    return MTPT_OK;
}

int mtpt_set_tuning(mtpt_handle* h, const mtpt_tuning* t) {
    if (!h || !t) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles > 0) return MTPT_ERR_STATE;   // a tile's grid is the whole box's
    if (!(t->cell_scale == 0.5 || (t->cell_scale >= 1.0 && t->cell_scale <= 8.0)))
        return MTPT_ERR_INVALID_ARG;
    if (t->pair_block != 128 && t->pair_block != 256) return MTPT_ERR_INVALID_ARG;
    const bool regrid = t->cell_scale != h->cell_scale;
    HostSnapshot snap;
    const bool saved = regrid && h->have_particles && snap.take(h);
    if (regrid && h->have_particles && !saved) return MTPT_ERR_NO_MEMORY;
    h->cell_scale = t->cell_scale;
    h->pair_block = t->pair_block;
    drop_graph(h);
    if (regrid && h->have_particles) {
        int rc = setup_grids(h);
        if (rc == MTPT_OK && h->any_transfer) rc = ensure_cells(h);
        if (rc == MTPT_OK) rc = upload_tables(h);
        if (rc != MTPT_OK) {
            // back to the old grid (its arrays are all still there)
            if (restore_snapshot(h, snap) != MTPT_OK) {
                h->have_particles = false;
                h->n = 0;
            }
            return rc;
        }
        h->have_row_sums = false;
        h->walked_ahead = false;
    }
    return MTPT_OK;
}

int mtpt_get_tuning(mtpt_handle* h, mtpt_tuning* out) {
    if (!h || !out) return MTPT_ERR_INVALID_ARG;
    out->cell_scale = h->cell_scale;
    out->pair_block = h->pair_block;
    out->pad = 0;
    return MTPT_OK;
}

int mtpt_autotune(mtpt_handle* h, int32_t trial_steps, mtpt_tuning* chosen) {
    if (!h || trial_steps < 1) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles || h->ntiles > 0) return MTPT_ERR_STATE;
    // snapshot of the current state (the trials step it)
    const int64_t n = h->n;
    const int d = h->dim;
    DevBuf<double> spos, smass, smassb;
    DevBuf<uint32_t> sid, srid;
    auto free_snapshot = [&]() {
        spos.release();
        smass.release();
        smassb.release();
        sid.release();
        srid.release();
    };
    {
        GrowAll g;
        g.want(spos, size_t(d) * size_t(std::max<int64_t>(n, 1)));
        g.want(smass, size_t(std::max<int64_t>(n, 1)));
        if (h->reactive) g.want(smassb, size_t(std::max<int64_t>(n, 1)));
        g.want(sid, size_t(std::max<int64_t>(n, 1)));
        if (h->batch) g.want(srid, size_t(std::max<int64_t>(n, 1)));
        MTPT_TRY(g.commit());
    }
    const bool timing0 = h->timing;
    h->timing = false;
    const mtpt_tuning start_tuning{h->cell_scale, h->pair_block, 0};
    const int c0 = h->cur;
    const bool fresh0 = h->fresh;         // every trial starts from the same state
    auto copy_state = [&](bool save) -> int {
        const size_t pitch = size_t(h->cap) * sizeof(double), row = size_t(n) * sizeof(double);
        if (n == 0) return MTPT_OK;
        if (save) {
            MTPT_CUDA_TRY(cudaMemcpy2DAsync(spos.p, row, h->pos[c0].p, pitch, row, d,
                                            cudaMemcpyDeviceToDevice, h->stream));
            MTPT_CUDA_TRY(cudaMemcpyAsync(smass.p, h->mass[c0].p, row, cudaMemcpyDeviceToDevice, h->stream));
            if (h->reactive)
                MTPT_CUDA_TRY(cudaMemcpyAsync(smassb.p, h->massb[c0].p, row, cudaMemcpyDeviceToDevice,
                                              h->stream));
            MTPT_CUDA_TRY(cudaMemcpyAsync(sid.p, h->id[c0].p, size_t(n) * 4, cudaMemcpyDeviceToDevice, h->stream));
            if (h->batch)
                MTPT_CUDA_TRY(cudaMemcpyAsync(srid.p, h->rid[c0].p, size_t(n) * 4, cudaMemcpyDeviceToDevice, h->stream));
        } else {
            h->cur = c0;
            h->fresh = fresh0;
            MTPT_CUDA_TRY(cudaMemcpy2DAsync(h->pos[c0].p, pitch, spos.p, row, row, d,
                                            cudaMemcpyDeviceToDevice, h->stream));
            MTPT_CUDA_TRY(cudaMemcpyAsync(h->mass[c0].p, smass.p, row, cudaMemcpyDeviceToDevice, h->stream));
            if (h->reactive)
                MTPT_CUDA_TRY(cudaMemcpyAsync(h->massb[c0].p, smassb.p, row, cudaMemcpyDeviceToDevice,
                                              h->stream));
            MTPT_CUDA_TRY(cudaMemcpyAsync(h->id[c0].p, sid.p, size_t(n) * 4, cudaMemcpyDeviceToDevice, h->stream));
            if (h->batch)
                MTPT_CUDA_TRY(cudaMemcpyAsync(h->rid[c0].p, srid.p, size_t(n) * 4, cudaMemcpyDeviceToDevice, h->stream));
        }
        return MTPT_OK;
    };
    const uint64_t step0 = h->step;
    unsigned long long pairs0 = 0;
    int rc = MTPT_OK;
    if (cudaMemcpyAsync(&pairs0, h->pair_counter.p, sizeof(pairs0), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
        rc = MTPT_ERR_CUDA;
    if (rc == MTPT_OK) rc = copy_state(true);
    if (rc == MTPT_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = MTPT_ERR_CUDA;
    if (rc != MTPT_OK) {
        (void)cudaGetLastError();
        h->timing = timing0;
        free_snapshot();
        return rc;
    }
    const double scales[] = {0.5, 1.0, 1.25, 1.5, 2.0};
    const int blocks[] = {128, 256};
    mtpt_tuning best{1.0, 256, 0};
    float best_ms = INFINITY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = MTPT_ERR_CUDA;
    for (double sc : scales) {
        if (rc != MTPT_OK) break;
        for (int bl : blocks) {
            mtpt_tuning t{sc, bl, 0};
            rc = mtpt_set_tuning(h, &t);
            if (rc == MTPT_OK) rc = run_steps(h, 1, MTPT_DO_WALK | MTPT_DO_TRANSFER);   // warm-up
            if (rc == MTPT_OK && cudaEventRecord(e0, h->stream) != cudaSuccess) rc = MTPT_ERR_CUDA;
            if (rc == MTPT_OK) rc = run_steps(h, trial_steps, MTPT_DO_WALK | MTPT_DO_TRANSFER);
            if (rc == MTPT_OK && cudaEventRecord(e1, h->stream) != cudaSuccess) rc = MTPT_ERR_CUDA;
            if (rc == MTPT_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = MTPT_ERR_CUDA;
            float ms = 0.0f;
            if (rc == MTPT_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = MTPT_ERR_CUDA;
            if (rc == MTPT_OK) rc = copy_state(false);
            if (rc != MTPT_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        if (rc != MTPT_OK) break;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    (void)cudaGetLastError();
    // the pick (or, after a failed trial, the starting tuning) with the state
    // of before the call; the starting grid's arrays exist, so this allocates
    // nothing when the trials failed
    const mtpt_tuning keep = rc == MTPT_OK ? best : start_tuning;
    int rc2 = mtpt_set_tuning(h, &keep);
    if (rc2 != MTPT_OK && rc != MTPT_OK) rc2 = mtpt_set_tuning(h, &start_tuning);
    if (rc2 == MTPT_OK) rc2 = copy_state(false);
    if (rc2 == MTPT_OK) rc2 = set_step_dev(h, step0);
    if (rc2 == MTPT_OK) {
        if (cudaMemcpyAsync(h->pair_counter.p, &pairs0, sizeof(pairs0), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            rc2 = MTPT_ERR_CUDA;
    }
    h->have_row_sums = false;
    h->walked_ahead = false;
    h->timing = timing0;
    free_snapshot();
    if (rc == MTPT_OK) rc = rc2;
    if (rc == MTPT_OK && chosen) *chosen = best;
    return rc;
}

// --- split domain (Secs. 4-5) ------------------------------------------------
}  // extern "C"

namespace {

// The tile's particle set from n_keep kept records and n_recv received ones
// (records of dim + 2 binary64 values), natives first classified by the
// tile that owns them; *flags receives the assembly's error bits.
template <int DIM>
int tile_install_t(mtpt_handle* h, int64_t n_keep, const double* keep, int64_t n_recv,
                   const double* recv, bool strict, double mass_limit) {
    const int64_t n = n_keep + n_recv;
    if (n > int64_t(0x7fffffff) - kBlock) return MTPT_ERR_INVALID_ARG;
    const bool first = !h->have_particles;
    const int64_t cap0 = h->cap;
    h->n = n;
    h->reals[0].n = n;
    // headroom: a tile's particle count drifts from step to step
    MTPT_TRY(ensure_capacity(h, n > h->cap ? n + n / 8 : n));
    // the grid and its cell arrays (ensure_cells allocates the corner tables
    // that upload_tables fills), as the plain load does them
    if (first) MTPT_TRY(setup_grids(h));
    if ((first || h->cap != cap0) && h->any_transfer) MTPT_TRY(ensure_cells(h));
    if (first) {
        // the tile geometry's edge tables (device copies, pointers into them)
        const size_t nt = std::max<size_t>(h->tile_tables.size(), 1);
        MTPT_TRY(h->tile_tables_dev.ensure(nt));
        if (!h->tile_tables.empty())
            MTPT_CUDA_TRY(cudaMemcpyAsync(h->tile_tables_dev.p, h->tile_tables.data(),
                                          h->tile_tables.size() * sizeof(long long),
                                          cudaMemcpyHostToDevice, h->stream));
        for (int a = 0; a < 3; ++a) {
            const int aa = a < h->dim ? a : 0;
            const int f = h->tile.f[aa];
            const long long* base = h->tile_tables_dev.p + h->tile_table_off[aa];
            h->tile.edge[a] = base;
            h->tile.near_lo[a] = base + f + 1;
            h->tile.near_hi[a] = base + 2 * f + 1;
        }
        if (!h->exp_table.p) {
            MTPT_TRY(h->exp_table.ensure(kExpTable));
            MTPT_CUDA_TRY(cudaMemcpyAsync(h->exp_table.p, exp_table_host(),
                                          kExpTable * sizeof(double), cudaMemcpyHostToDevice,
                                          h->stream));
        }
        MTPT_TRY(upload_tables(h));
    }
    MTPT_TRY(h->tile_flag.ensure(1));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->tile_flag.p, 0, sizeof(uint32_t), h->stream));
    drop_graph(h);
    h->cur = 0;
    if (n > 0) {
        MTPT_TIMED(h, "tile_assemble");
        k_tile_assemble<DIM><<<grid_for(n), kBlock, 0, h->stream>>>(
            int(n_keep), keep, int(n_recv), recv, h->tile, strict ? 1 : 0, mass_limit, h->cap,
            h->pos[0].p, h->mass[0].p, h->id[0].p, h->tile_flag.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    h->fresh = true;
    h->have_particles = true;
    h->have_row_sums = false;
    h->walked_ahead = false;
    return MTPT_OK;
}

template <int DIM>
int tile_pack_t(mtpt_handle* h, int64_t cap, double* send, int64_t* counts) {
    const int P = h->ntiles;
    const int n = int(h->n);
    constexpr int K = DIM + 2;
    MTPT_TRY(h->tile_counts.ensure(size_t(2 * P)));
    MTPT_TRY(h->tile_base.ensure(size_t(2 * P)));
    MTPT_TRY(h->tile_cursor.ensure(size_t(2 * P)));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->tile_counts.p, 0, size_t(2 * P) * 8, h->stream));
    if (n > 0) {
        MTPT_TIMED(h, "tile_count");
        k_tile_count<DIM><<<grid_for(n), kBlock, 0, h->stream>>>(n, h->cap, h->pos[h->cur].p,
                                                                 h->tile, h->tile_counts.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    h->tile_host.assign(size_t(4 * P), 0ull);
    unsigned long long* cnt = h->tile_host.data();
    unsigned long long* base = cnt + 2 * P;
    MTPT_CUDA_TRY(cudaMemcpyAsync(cnt, h->tile_counts.p, size_t(2 * P) * 8,
                                  cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    const int self = h->tile.self;
    unsigned long long total = 0;
    for (int t = 0; t < P; ++t) {
        counts[2 * t] = int64_t(cnt[2 * t]);
        counts[2 * t + 1] = int64_t(cnt[2 * t + 1]);
        if (t == self) continue;
        base[2 * t] = total;
        total += cnt[2 * t];
        base[2 * t + 1] = total;
        total += cnt[2 * t + 1];
    }
    base[2 * self] = 0;
    base[2 * self + 1] = cnt[2 * self];
    h->keep_ready = false;
    if (int64_t(total) > cap) return MTPT_ERR_CAPACITY;
    if (total > 0 && !send) return MTPT_ERR_INVALID_ARG;
    const int64_t kept = int64_t(cnt[2 * self] + cnt[2 * self + 1]);
    MTPT_TRY(h->tile_keep.ensure(size_t(K) * size_t(std::max<int64_t>(kept, 1))));
    MTPT_CUDA_TRY(cudaMemcpyAsync(h->tile_base.p, base, size_t(2 * P) * 8,
                                  cudaMemcpyHostToDevice, h->stream));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->tile_cursor.p, 0, size_t(2 * P) * 8, h->stream));
    if (n > 0) {
        MTPT_TIMED(h, "tile_scatter");
        k_tile_scatter<DIM><<<grid_for(n), kBlock, 0, h->stream>>>(
            n, h->cap, h->pos[h->cur].p, h->mass[h->cur].p, h->id[h->cur].p, h->tile,
            h->tile_base.p, h->tile_cursor.p, send, h->tile_keep.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    h->keep_n = kept;
    h->keep_ready = true;
    return MTPT_OK;
}

template <int DIM>
int tile_transfer_t(mtpt_handle* h, int64_t n_recv, const double* recv) {
    MTPT_TRY(tile_install_t<DIM>(h, h->keep_n, h->tile_keep.p, n_recv, recv, false, HUGE_VAL));
    h->keep_ready = false;
    MTPT_TRY(dispatch_step(h, MTPT_DO_TRANSFER));
    // keep the natives
    MTPT_TRY(h->tile_native.ensure(1));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->tile_native.p, 0, 8, h->stream));
    const int c = h->cur, o = 1 - h->cur;
    if (h->n > 0) {
        MTPT_TIMED(h, "tile_compact");
        k_tile_compact<DIM><<<grid_for(h->n), kBlock, 0, h->stream>>>(
            int(h->n), h->cap, h->pos[c].p, h->mass[c].p, h->id[c].p, h->pos[o].p,
            h->mass[o].p, h->id[o].p, h->tile_native.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long natives = 0;
    uint32_t flag = 0, st = 0;
    MTPT_CUDA_TRY(cudaMemcpyAsync(&natives, h->tile_native.p, 8, cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaMemcpyAsync(&flag, h->tile_flag.p, 4, cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaMemcpyAsync(&st, h->status.p, 4, cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->cur = o;
    h->n = int64_t(natives);
    h->reals[0].n = h->n;
    h->have_row_sums = false;
    h->walked_ahead = false;
    if (flag) return MTPT_ERR_INVALID_ARG;
    return status_code(h, st);
}

template <int DIM>
int tile_load_t(mtpt_handle* h, int64_t n, const double* pos, const double* mass,
                const uint32_t* ids) {
    constexpr int K = DIM + 2;
    const size_t nn = size_t(std::max<int64_t>(n, 1));
    MTPT_TRY(h->tile_stage.ensure(size_t(DIM + 1) * nn + (nn + 1) / 2));
    MTPT_TRY(h->tile_keep.ensure(size_t(K) * nn));
    double* sp = h->tile_stage.p;
    double* sm = sp + size_t(DIM) * nn;
    uint32_t* si = reinterpret_cast<uint32_t*>(sm + nn);
    if (n > 0) {
        MTPT_CUDA_TRY(cudaMemcpyAsync(sp, pos, size_t(DIM) * size_t(n) * 8,
                                      cudaMemcpyHostToDevice, h->stream));
        MTPT_CUDA_TRY(cudaMemcpyAsync(sm, mass, size_t(n) * 8, cudaMemcpyHostToDevice, h->stream));
        MTPT_CUDA_TRY(cudaMemcpyAsync(si, ids, size_t(n) * 4, cudaMemcpyHostToDevice, h->stream));
        // the positions' SoA stride is n in the staging copy
        k_tile_records<DIM><<<grid_for(n), kBlock, 0, h->stream>>>(int(n), sp, sm, si,
                                                                  h->tile_keep.p);
        MTPT_CUDA_TRY(cudaGetLastError());
    }
    h->have_particles = false;
    const double mass_limit = h->precision == MTPT_FP32W ? 1e30 : HUGE_VAL;
    MTPT_TRY(tile_install_t<DIM>(h, n, h->tile_keep.p, 0, nullptr, true, mass_limit));
    uint32_t flag = 0;
    MTPT_CUDA_TRY(cudaMemcpyAsync(&flag, h->tile_flag.p, 4, cudaMemcpyDeviceToHost, h->stream));
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (flag) {
        h->have_particles = false;
        h->n = 0;
        h->reals[0].n = 0;
        if (flag & kTileErrForeign) return MTPT_ERR_OUT_OF_DOMAIN;
        return MTPT_ERR_INVALID_ARG;
    }
    MTPT_CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(uint32_t), h->stream));
    MTPT_CUDA_TRY(cudaMemsetAsync(h->pair_counter.p, 0, sizeof(unsigned long long), h->stream));
    MTPT_TRY(set_step_dev(h, 0));
    h->keep_ready = false;
    return MTPT_OK;
}

}  // namespace

extern "C" {

int mtpt_tiling_factors(int32_t dim, const double* lo, const double* hi, int32_t ntiles,
                        int32_t* factors) {
    if (!lo || !hi || !factors || dim < 1 || dim > kMaxDim || ntiles < 1 || ntiles > (1 << 20))
        return MTPT_ERR_INVALID_ARG;
    double L[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        if (!(hi[a] > lo[a]) || !std::isfinite(hi[a] - lo[a])) return MTPT_ERR_INVALID_ARG;
        L[a] = hi[a] - lo[a];
    }
    factors[0] = ntiles;
    factors[1] = factors[2] = 1;
    if (dim == 2) {
        // Eq. "minimization": f1 <= f2, f1 f2 = N, |f2 / f1 - A| least for the
        // aspect ratio A >= 1; the longer side takes f2 tiles
        const int wide = L[0] >= L[1] ? 0 : 1;
        const double A = L[wide] / L[1 - wide];
        int best1 = 1;
        double best = INFINITY;
        for (int f1 = 1; int64_t(f1) * f1 <= ntiles; ++f1) {
            if (ntiles % f1) continue;
            const double e = std::fabs(double(ntiles / f1) / double(f1) - A);
            if (e < best) {
                best = e;
                best1 = f1;
            }
        }
        factors[wide] = ntiles / best1;
        factors[1 - wide] = best1;
    } else if (dim == 3) {
        // the 3-d counterpart (the paper asks for tiles closest to cubes):
        // the factor triple whose largest tile edge over its smallest is least
        double best = INFINITY;
        for (int f0 = 1; f0 <= ntiles; ++f0) {
            if (ntiles % f0) continue;
            const int rest = ntiles / f0;
            for (int f1 = 1; f1 <= rest; ++f1) {
                if (rest % f1) continue;
                const int f2 = rest / f1;
                const double e[3] = {L[0] / f0, L[1] / f1, L[2] / f2};
                const double r = std::max({e[0], e[1], e[2]}) / std::min({e[0], e[1], e[2]});
                if (r < best) {
                    best = r;
                    factors[0] = f0;
                    factors[1] = f1;
                    factors[2] = f2;
                }
            }
        }
    }
    return MTPT_OK;
}

int mtpt_set_tiling(mtpt_handle* h, const mtpt_tiling* t) {
    if (!h || !t) return MTPT_ERR_INVALID_ARG;
    if (h->nreal != 1 || h->batch || h->have_particles || h->reactive) return MTPT_ERR_STATE;
    RealHost& R = h->reals[0];
    const mtpt_params& p = R.prm;
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        if (t->tiles[a] < 1 || (a >= p.dim && t->tiles[a] != 1)) return MTPT_ERR_INVALID_ARG;
        total *= t->tiles[a];
    }
    if (total > (1 << 20) || t->tile < 0 || t->tile >= total) return MTPT_ERR_INVALID_ARG;
    if (t->n_global < 0 || t->n_global > int64_t(0x7fffffff) - kBlock) return MTPT_ERR_INVALID_ARG;
    const double pad = R.psi > 0.0 ? 2.0 * R.psi * (1.0 + 1e-6) : 0.0;
    TileGeom g{};
    int at[3] = {t->tile % t->tiles[0], (t->tile / t->tiles[0]) % t->tiles[1],
                 t->tile / (t->tiles[0] * t->tiles[1])};
    // edge tables: e_t = lo + t width, e_t + pad, e_(t+1) - pad as order keys
    std::vector<long long> tables;
    int table_off[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        const int f = t->tiles[a];
        g.f[a] = f;
        table_off[a] = int(tables.size());
        if (a >= p.dim) {
            g.lo_f[a] = 0.0f;
            g.inv_w_f[a] = 1.0f;
            R.tile_lo[a] = R.tile_hi[a] = 0.0;
            continue;
        }
        const double width = (p.hi[a] - p.lo[a]) / double(f);
        // every tile at least a pad wide, so a pad reaches the next tile only
        if (f > 1 && !(width >= pad)) return MTPT_ERR_INVALID_ARG;
        g.lo_f[a] = float(p.lo[a]);
        g.inv_w_f[a] = float(1.0 / width);
        std::vector<double> e(size_t(f) + 1);
        for (int k = 0; k <= f; ++k) e[size_t(k)] = p.lo[a] + double(k) * width;
        for (int k = 0; k <= f; ++k) tables.push_back(host_order_key(e[size_t(k)]));
        for (int k = 0; k < f; ++k) tables.push_back(host_order_key(e[size_t(k)] + pad));
        for (int k = 0; k < f; ++k) tables.push_back(host_order_key(e[size_t(k) + 1] - pad));
        R.tile_lo[a] = e[size_t(at[a])];
        R.tile_hi[a] = e[size_t(at[a]) + 1];
    }
    g.self = t->tile;
    R.tiled = true;
    R.n_global = t->n_global;
    R.pad = pad;
    h->tile = g;
    h->tile_tables = std::move(tables);
    for (int a = 0; a < 3; ++a) h->tile_table_off[a] = table_off[a];
    h->ntiles = int(total);
    return MTPT_OK;
}

int mtpt_set_particles_tile(mtpt_handle* h, int64_t n, const double* pos, const double* mass,
                            const uint32_t* ids) {
    if (!h || n < 0 || (n > 0 && (!pos || !mass || !ids))) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles == 0) return MTPT_ERR_STATE;
    switch (h->dim) {
        case 1: return tile_load_t<1>(h, n, pos, mass, ids);
        case 2: return tile_load_t<2>(h, n, pos, mass, ids);
        default: return tile_load_t<3>(h, n, pos, mass, ids);
    }
}

int mtpt_tile_pack(mtpt_handle* h, int64_t cap, double* send_dev, int64_t* counts) {
    if (!h || !counts || cap < 0) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles == 0 || !h->have_particles) return MTPT_ERR_STATE;
    switch (h->dim) {
        case 1: return tile_pack_t<1>(h, cap, send_dev, counts);
        case 2: return tile_pack_t<2>(h, cap, send_dev, counts);
        default: return tile_pack_t<3>(h, cap, send_dev, counts);
    }
}

int mtpt_tile_transfer(mtpt_handle* h, int64_t n_recv, const double* recv_dev) {
    if (!h || n_recv < 0 || (n_recv > 0 && !recv_dev)) return MTPT_ERR_INVALID_ARG;
    if (h->ntiles == 0 || !h->have_particles || !h->keep_ready) return MTPT_ERR_STATE;
    switch (h->dim) {
        case 1: return tile_transfer_t<1>(h, n_recv, recv_dev);
        case 2: return tile_transfer_t<2>(h, n_recv, recv_dev);
        default: return tile_transfer_t<3>(h, n_recv, recv_dev);
    }
}

int mtpt_get_ids(mtpt_handle* h, uint32_t* out) {
    if (!h || (!out && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->have_particles) return MTPT_ERR_STATE;
    if (h->n == 0) return MTPT_OK;
    if (h->ntiles == 0) {
        for (int64_t i = 0; i < h->n; ++i) out[i] = uint32_t(i);
        return MTPT_OK;
    }
    MTPT_CUDA_TRY(cudaMemcpyAsync(out, h->id[h->cur].p, size_t(h->n) * 4, cudaMemcpyDeviceToHost,
                                  h->stream));
    return read_status(h);
}

int mtpt_set_reaction(mtpt_handle* h, double k) {
    if (!h) return MTPT_ERR_INVALID_ARG;
    if (h->batch || h->nreal != 1 || h->ntiles > 0) return MTPT_ERR_STATE;
    if (!(k >= 0.0) || !std::isfinite(k)) return MTPT_ERR_INVALID_ARG;
    if (!h->reactive && h->cap > 0) {
        GrowAll g;
        for (int b = 0; b < 2; ++b) g.want(h->massb[b], size_t(h->cap));
        if (h->precision == MTPT_FP32W) g.want(h->exb, size_t(h->cap));
        MTPT_TRY(g.commit());
        if (h->have_particles && h->n > 0)
            MTPT_CUDA_TRY(cudaMemsetAsync(h->massb[h->cur].p, 0, size_t(h->n) * sizeof(double),
                                          h->stream));
    }
    drop_graph(h);
    h->reactive = true;
    h->react_k = k;
    h->adj_ready = false;
    return MTPT_OK;
}

int mtpt_set_masses_b(mtpt_handle* h, const double* mass_b) {
    if (!h || (!mass_b && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->reactive || !h->have_particles) return MTPT_ERR_STATE;
    const int64_t n = h->n;
    if (n == 0) return MTPT_OK;
    for (int64_t i = 0; i < n; ++i)
        if (!(mass_b[i] >= 0.0) || !std::isfinite(mass_b[i]) ||
            (h->precision == MTPT_FP32W && mass_b[i] > 1e30))
            return MTPT_ERR_INVALID_ARG;
    MTPT_TRY(ensure_out_tmp(h));
    MTPT_CUDA_TRY(cudaMemcpyAsync(h->out_tmp.p, mass_b, size_t(n) * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream));
    // to the current order: slot s holds the particle of input index id[s]
    k_take_by_id<<<grid_for(n), kBlock, 0, h->stream>>>(int(n), h->id[h->cur].p, h->out_tmp.p,
                                                        h->massb[h->cur].p);
    MTPT_CUDA_TRY(cudaGetLastError());
    MTPT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return MTPT_OK;
}

int mtpt_get_masses_b(mtpt_handle* h, double* out) {
    if (!h || (!out && h->n > 0)) return MTPT_ERR_INVALID_ARG;
    if (!h->reactive || !h->have_particles) return MTPT_ERR_STATE;
    if (h->n == 0) return MTPT_OK;
    MTPT_TRY(ensure_out_tmp(h));
    MTPT_TRY(unpermute_to(h, h->massb[h->cur].p, 1, h->out_tmp.p));
    return copy_out_host(h, 1, out);
}

int mtpt_debug_fail_alloc(int64_t nth, int64_t* remaining) {
    if (nth < 0) return MTPT_ERR_INVALID_ARG;
    const int64_t before = g_fail_alloc.exchange(nth);
    if (remaining) *remaining = before;
    return MTPT_OK;
}

int mtpt_debug_scan_hold(int32_t tile, uint64_t* gave_up) {
    if (tile < -1) return MTPT_ERR_INVALID_ARG;
    g_scan_hold.store(tile);
    if (gave_up) {
        unsigned long long v = 0;
        MTPT_CUDA_TRY(cudaDeviceSynchronize());
        MTPT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_scan_waits_given_up, sizeof(v)));
        *gave_up = uint64_t(v);
    }
    return MTPT_OK;
}

const char* mtpt_status_string(int status) {
    switch (status) {
        case MTPT_OK: return "ok";
        case MTPT_ERR_INVALID_ARG: return "invalid argument";
        case MTPT_ERR_OUT_OF_DOMAIN: return "particle outside the box or not finite";
        case MTPT_ERR_CUDA: return "CUDA runtime error";
        case MTPT_ERR_NO_MEMORY: return "allocation failed";
        case MTPT_ERR_STATE: return "call not valid in the handle's state";
        case MTPT_ERR_CAPACITY: return "output buffer too small";
        case MTPT_ERR_TOO_LARGE: return "problem larger than the fixed no-allocation scratch";
        default: return "unknown status";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mtpt_step_noalloc: one time step with all working memory in a fixed
// file-scope device array instead of cudaMalloc'ed buffers, for callers that
// must not allocate.  It runs the same kernels as mtpt_step through a handle
// that lives on the host stack (inline realisation storage, no host
// allocation) and whose buffers point into the array.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MTPT_NOALLOC_SCRATCH_BYTES];

// Head of the array, at fixed offsets whatever n is: the binary64 kernel
// exponential's table (written once per device at set-up) and the per-call
// words that the init kernel writes.
struct NoallocHead {
    double exp_table[kExpTable];
    RealParams params;
    int corner_first[2];
    uint32_t status;
    unsigned long long pair_counter;
    unsigned long long step;
};
constexpr size_t kNoallocHeadBytes = (sizeof(NoallocHead) + 255) & ~size_t(255);

// Worst case of the per-call pieces carved after the head, at n =
// MTPT_NOALLOC_MAX_PARTICLES: 3-d binary32 form, 108 bytes per particle
// (mass copy 8, sorted positions 24 and mass 8, two id arrays 8, key 4,
// permutation 4, sort key 16, cell 4, rec 16, mass split and row sum 16); the
// cell grid capped at 4 n + 64 cells (setup_grid), so count and start hold at
// most that many plus one cells padded to a scan tile, and the corner tables
// at most the sum of the per-axis cell counts (<= their product + 2); each
// piece rounded up to 256 bytes.
constexpr size_t kNoallocMaxCells = 4 * size_t(MTPT_NOALLOC_MAX_PARTICLES) + 64;
constexpr size_t kNoallocMaxCellsPad = (kNoallocMaxCells + 1 + kScanTile - 1) / kScanTile * kScanTile;
constexpr size_t kNoallocWorstBytes =
    kNoallocHeadBytes + 108 * size_t(MTPT_NOALLOC_MAX_PARTICLES) +
    2 * sizeof(uint32_t) * kNoallocMaxCellsPad +
    sizeof(unsigned long long) * (kNoallocMaxCellsPad / kScanTile + 1) +
    sizeof(float2) * (kNoallocMaxCells + 2) + 16 * 256;
static_assert(kNoallocWorstBytes <= size_t(MTPT_NOALLOC_SCRATCH_BYTES),
              "the no-allocation scratch must hold the largest layout n allows");

constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_addr[kNoallocMaxDevices] = {};
std::once_flag g_noalloc_once[kNoallocMaxDevices];
cudaError_t g_noalloc_err[kNoallocMaxDevices] = {};

// The array's device address on the current device, looked up once per
// device (with its exponential table written there at the same time).  In
// host code `g_noalloc_scratch` names a host-side stand-in, never a device
// address, so kernels only ever receive the looked-up pointer.
int noalloc_scratch(void** out) {
    int dev = -1;
    MTPT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return MTPT_ERR_CUDA;
    std::call_once(g_noalloc_once[dev], [dev]() {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess)
            e = cudaMemcpy(static_cast<NoallocHead*>(p)->exp_table, exp_table_host(),
                           kExpTable * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) (void)cudaGetLastError();
        g_noalloc_err[dev] = e;
        g_noalloc_addr[dev] = (e == cudaSuccess) ? p : nullptr;
    });
    if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_addr[dev]) return MTPT_ERR_CUDA;
    *out = g_noalloc_addr[dev];
    return MTPT_OK;
}

// The per-call words of the head, from kernel arguments (taken by value at
// launch, so nothing on the host is read after the call returns).
__global__ void k_noalloc_init(RealParams p, int n_corners, unsigned long long step,
                               NoallocHead* head) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    head->params = p;
    head->corner_first[0] = 0;
    head->corner_first[1] = n_corners;
    head->status = 0u;
    head->pair_counter = 0ull;
    head->step = step;
}

// Bump carving of the rest of the array into 256-byte-aligned pieces.
struct Carver {
    unsigned char* base;
    size_t used = kNoallocHeadBytes;
    bool overflow = false;
    template <typename T>
    T* take(size_t count) {
        const size_t off = (used + 255) & ~size_t(255);
        const size_t bytes = count * sizeof(T);
        if (off + bytes > size_t(MTPT_NOALLOC_SCRATCH_BYTES)) {
            overflow = true;
            return nullptr;
        }
        used = off + bytes;
        return reinterpret_cast<T*>(base + off);
    }
};

}  // namespace

extern "C" int mtpt_step_noalloc(const mtpt_params* params, int64_t n, uint64_t step,
                                 double* pos_dev, double* mass_dev, void* stream) {
    MTPT_TRY(validate_params(params));
    if (n < 0 || (n > 0 && (!pos_dev || !mass_dev))) return MTPT_ERR_INVALID_ARG;
    if (n > MTPT_NOALLOC_MAX_PARTICLES) return MTPT_ERR_TOO_LARGE;
    void* scratch = nullptr;
    MTPT_TRY(noalloc_scratch(&scratch));
    if (n == 0) return MTPT_OK;

    mtpt_handle h;                       // host-side bookkeeping only
    h.dim = params->dim;
    h.precision = params->precision;
    h.reals[0].prm = *params;
    derive(h.reals[0], h.params[0]);
    h.stream = static_cast<cudaStream_t>(stream);
    h.n = n;
    h.cap = n;
    h.reals[0].n = n;
    h.params[0].id_offset = 0;
    MTPT_TRY(setup_grids(&h));
    h.nb_cap = 0;                        // no neighbour lists: pass 2 searches
    h.nb32_cap = 0;
    const int d = h.dim;
    const size_t cells_pad = size_t(h.n_cells_pad);

    NoallocHead* head = static_cast<NoallocHead*>(scratch);
    h.exp_table.p = head->exp_table;
    h.status.p = &head->status;
    h.pair_counter.p = &head->pair_counter;
    h.step_dev.p = &head->step;
    Carver cv{static_cast<unsigned char*>(scratch)};
    double* mass_in = cv.take<double>(size_t(n));
    double* pos_sorted = cv.take<double>(size_t(d) * size_t(n));
    double* mass_sorted = cv.take<double>(size_t(n));
    uint32_t* id_in = cv.take<uint32_t>(size_t(n));
    uint32_t* id_sorted = cv.take<uint32_t>(size_t(n));
    h.key.p = cv.take<uint32_t>(size_t(n));
    h.perm.p = cv.take<uint32_t>(size_t(n));
    h.sortkey.p = cv.take<double2>(size_t(n));
    h.cell.p = cv.take<uint32_t>(size_t(n));
    h.rec.p = cv.take<float4>(size_t(n));
    if (h.precision == MTPT_FP64) {
        h.r64.p = cv.take<double>(size_t(n));
    } else {
        h.ex.p = cv.take<float4>(size_t(n));
    }
    h.corners.p = cv.take<float2>(size_t(std::max(h.n_corners, 1)));
    h.count.p = cv.take<uint32_t>(cells_pad);
    h.start.p = cv.take<uint32_t>(cells_pad);
    h.scan_state.p = cv.take<unsigned long long>(cells_pad / kScanTile + 1);   // + the ticket
    if (cv.overflow) return MTPT_ERR_TOO_LARGE;

    // The handle's buffer pairs: index 0 is the caller's state (positions are
    // walked in place; masses are read from a scratch copy), index 1 the
    // cell-ordered copy.  None of these pointers is owned by `h`.
    h.pos[0].p = pos_dev;
    h.pos[1].p = pos_sorted;
    h.mass[0].p = mass_in;
    h.mass[1].p = mass_sorted;
    h.id[0].p = id_in;
    h.id[1].p = id_sorted;
    h.cur = 0;
    h.have_particles = true;

    cudaStream_t st = h.stream;
    // what must start at zero (cell counts, status word, pair counter) and the
    // call's parameters, step and corner offsets, all from device-side work
    if (h.any_transfer) {
        MTPT_CUDA_TRY(cudaMemsetAsync(h.count.p, 0, cells_pad * sizeof(uint32_t), st));
        MTPT_TRY(reset_scan(&h, st));
    }
    k_noalloc_init<<<1, 32, 0, st>>>(h.params[0], h.n_corners, (unsigned long long)step, head);
    MTPT_CUDA_TRY(cudaGetLastError());
    MTPT_CUDA_TRY(cudaMemcpyAsync(mass_in, mass_dev, size_t(n) * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
    k_iota<<<grid_for(n), kBlock, 0, st>>>(int(n), id_in);
    MTPT_CUDA_TRY(cudaGetLastError());
    MTPT_TRY(build_corners(&h, &head->params, head->corner_first));
    MTPT_TRY(dispatch_step(&h, MTPT_DO_WALK | MTPT_DO_TRANSFER));
    // masses back to the caller's order; positions are already there
    k_unpermute<double><<<grid_for(n), kBlock, 0, st>>>(int(n), h.cap, 1, h.id[h.cur].p,
                                                        h.mass[h.cur].p, 1, 1.0, mass_dev);
    MTPT_CUDA_TRY(cudaGetLastError());
    return MTPT_OK;
}
