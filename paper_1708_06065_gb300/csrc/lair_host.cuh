// lair_host.cuh -- host-side internals shared by lair_api.cu (set-up orchestration, C ABI) and
// lair_solve.cu (the outer FP64 loops): the hierarchy and handle structures, the stream-ordered
// allocation arenas, kernel timers, exclusive scans and status read-backs.
#pragma once

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <atomic>
#include <type_traits>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "setup_kernels.cuh"

namespace lair {

void plus_one(int n, const int *a, int *b, cudaStream_t s);
void count_flags(int n, const uint8_t *f, int *out, cudaStream_t s);
void normalize_cf(int n, int8_t *cf, cudaStream_t s);



// ---------------------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------------------
struct Level {
    DCsr A;
    int8_t *cf = nullptr;
    uint8_t *strong = nullptr;
    int nc = 0;
    int *cidx = nullptr;
    DCsr R, P;
    uint8_t *lsR = nullptr, *lsP = nullptr;
    double *dinv = nullptr;
    float *dinv32 = nullptr;
    double *b64 = nullptr, *x64[2] = {nullptr, nullptr};
    float *b32 = nullptr, *x32[2] = {nullptr, nullptr};
    int xfinal = 0;         // which x buffer holds the cycle's result on this level
    bool coarsest = false;
    double *Ainv = nullptr;
    long long nF = 0, nnzF = 0, nC = 0, nnzC = 0;   // rows and entries by kind (for byte counts)
    std::vector<int> seg_h;   // batched systems: first row of every system on this level, nseg + 1 entries
    int *seg_d = nullptr;
    // cycle storage: sliced-ELL views of the F rows and C rows of A, of R and of P (cycle precision)
    int *frows = nullptr, *crows = nullptr;
    SellView AF, AC, Rv, Pv;
    SellView A64;             // level 0: all rows of A in FP64 for the outer iteration
    int *p1col = nullptr;     // one-point P (every entry 1): the coarse column of each row's entry, -1 without one
    int *blk_sys = nullptr;   // batched systems: the system of every 32-row block of the level (-1: several)
    // nodal hierarchy (k x k blocks): block Jacobi as point Jacobi on Ahat = D^{-1} A (diagonal blocks
    // inverted, diagonal exactly 1) with right-hand side D^{-1} b; binv holds the k x k inverses
    DCsr Ahat;
    double *binv = nullptr, *dinv_hat = nullptr, *bh64 = nullptr;
    float *binv32 = nullptr, *dinv_hat32 = nullptr, *bh32 = nullptr;
};

struct Hier {
    std::vector<Level> lev;
    int bs = 0;
    double *blk_inv = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_nodes = 0;
    long long singular_R = 0, singular_P = 0;
    double setup_ms = 0.0;
    // the sliced-ELL fill descriptors of all views (device), kept so that a refresh refills the views in place
    SellDesc *sell_desc = nullptr;
    // the bottom of the cycle in one CTA: levels bottom_first .. coarsest (-1: a kernel per phase everywhere);
    // bottom_desc holds their BottomLevel descriptors in the cycle's precision
    int bottom_first = -1;
    void *bottom_desc = nullptr;
    int sell_gp[3] = {0, 0, 0}, sell_glin[3] = {0, 0, 0};
};

}  // namespace lair

struct lair_handle {
    lair_options o;
    cudaStream_t s = nullptr;
    cudaStream_t own = nullptr;   // created when the caller gives no stream
    lair::DCsr A_in;              // the caller's matrix on the device (unscaled, unlumped)
    lair::Hier H;
    lair::Hier *HT = nullptr;     // adjoint hierarchy, built on demand
    int *status = nullptr;        // device status word
    int *h_int = nullptr;         // pinned host scratch
    double *h_dbl = nullptr;
    void *scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    std::vector<void *> allocs;   // everything owned by the handle
    int *prod_nnz = nullptr;      // device: entry counts of the timed level-0 products (timing only)
    bool prod_fused = false;      // level 0 formed R A P in one pass
    // bump arenas over large device chunks (owned through allocs): set-up temporaries (stack
    // discipline, see Temps) and small long-lived arrays; each allocation is 256-byte aligned
    struct Chunk { char *p; size_t size; size_t used; };
    std::vector<Chunk> tmp_chunks;
    int tmp_cur = -1, tmp_depth = 0;
    Chunk keep_chunk{nullptr, 0, 0};
    // outer-iteration work (FP64)
    double *wb = nullptr, *wx = nullptr, *wr = nullptr, *part = nullptr, *dsc = nullptr;
    double *V = nullptr, *Z = nullptr;
    int fg_m = 0;
    std::string err;
    long long launches = 0;
    // kernel timing (options.timing)
    struct Timer { std::string name; long long launches = 0; double ms = 0.0; double bytes = 0.0; };
    struct Pending { int slot; cudaEvent_t a, b; bool closed; int id; };
    int next_timer_id = 0;
    std::vector<Timer> timers;
    std::vector<Pending> pending;        // events recorded by direct launches, read at the next sync
    std::vector<Pending> graph_events;   // events inside the captured cycle graph
    std::vector<cudaEvent_t> ev_pool;
    bool graph_pending = false;
    // batched systems (block-diagonal input)
    int nseg = 0;
    // batched systems: per-system run flags read by the cycle's kernels (slices and blocks of systems that have
    // stopped are skipped); all 1 outside the batched outer loops, which steer them
    uint8_t *sys_run = nullptr;
    std::vector<int> seg0;
    double *h_seg = nullptr;      // pinned, nseg doubles
    uint8_t *h_act = nullptr;     // pinned, nseg bytes
    double *h_bat = nullptr;      // pinned, nseg * 32 doubles (per-system Hessenberg columns)
    double *d_bat = nullptr;      // device, nseg * (3 * 32 + 1) doubles: sums, pass values, y, norms
    int *d_batcnt = nullptr;      // device, nseg ints
    int *h_batcnt = nullptr;      // pinned, nseg ints
    lair::SegTiles segt;          // row tiles of the systems (level 0), built at the first batched solve
    // device-side control of the batched outer loops, and a ring of running-system counts read back late
    lair::BatchCtl bctl;
    int bctl_m = -1;
    static constexpr int RING = 8, LAG = 2;
    int *d_ring = nullptr;        // device, RING ints
    int *h_ring = nullptr;        // pinned, RING ints
    cudaEvent_t ring_ev[RING] = {};
};

namespace lair {

static inline lair_status fail(lair_handle *h, lair_status st, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

#define CU(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            if (e_ == cudaErrorMemoryAllocation) return fail(h, LAIR_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_)); \
            return fail(h, LAIR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                   \
        }                                                                                              \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        lair_status st_ = (expr);          \
        if (st_ != LAIR_OK) return st_;    \
    } while (0)

constexpr size_t ARENA_ALIGN = 256;
constexpr size_t KEEP_CHUNK = (size_t)32 << 20;      // long-lived arrays up to KEEP_CHUNK / 8 share chunks
constexpr size_t TMP_CHUNK_MIN = (size_t)64 << 20;

static inline size_t arena_round(size_t bytes) { return (bytes + ARENA_ALIGN - 1) & ~(ARENA_ALIGN - 1); }

// The library's own stream-ordered pool per device: memory freed by one handle stays reserved
// (up to POOL_KEEP bytes) for the next one instead of going back to the driver at every
// synchronisation, and the device's default pool is left as the caller configured it.
constexpr unsigned long long POOL_KEEP = 16ull << 30;
constexpr int POOL_DEVICES = 64;

cudaError_t lair_pool(cudaMemPool_t *out);   // the library's device memory pool (lair_api.cu)

// pinned host scratch of HOST_BLOCK bytes per handle, recycled between handles
constexpr size_t HOST_BLOCK = 1024;
// pinned host blocks of HOST_BLOCK bytes, recycled between handles (lair_api.cu)
cudaError_t host_block_get(void **p);
void host_block_put(void *p);

static inline lair_status raw_alloc(lair_handle *h, void **p, size_t bytes) {
    cudaMemPool_t pool;
    cudaError_t e = lair_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, h->s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LAIR_ERR_OOM, "device allocation of %zu bytes failed", bytes);
    }
    return LAIR_OK;
}

// keep = true: owned by the handle until lair_free (small arrays share chunks);
// keep = false: plain stream-ordered allocation, released with dfree
template <class T>
static inline lair_status dalloc(lair_handle *h, T **p, size_t n, bool keep = true) {
    *p = nullptr;
    if (n == 0) n = 1;
    const size_t bytes = arena_round(n * sizeof(T));
    void *q = nullptr;
    if (keep && bytes <= KEEP_CHUNK / 8) {
        auto &c = h->keep_chunk;
        if (!c.p || c.used + bytes > c.size) {
            void *np = nullptr;
            TRY(raw_alloc(h, &np, KEEP_CHUNK));
            h->allocs.push_back(np);
            c = lair_handle::Chunk{static_cast<char *>(np), KEEP_CHUNK, 0};
        }
        q = c.p + c.used;
        c.used += bytes;
    } else {
        TRY(raw_alloc(h, &q, bytes));
        if (keep) h->allocs.push_back(q);
    }
    *p = static_cast<T *>(q);
    return LAIR_OK;
}

static inline void dfree(lair_handle *h, void *p) {
    if (p) cudaFreeAsync(p, h->s);
}

// Set-up temporaries. The innermost live Temps bumps through the handle's temporary chunks and
// gives everything back at once when it goes out of scope; memory is reused only by work issued
// later on the same stream. A Temps that is not the innermost one allocates plainly instead.
struct Temps {
    lair_handle *h;
    int depth, mark_cur;
    size_t mark_used;
    std::vector<void *> raw;
    explicit Temps(lair_handle *hh) : h(hh) {
        depth = ++h->tmp_depth;
        mark_cur = h->tmp_cur;
        mark_used = h->tmp_cur >= 0 ? h->tmp_chunks[h->tmp_cur].used : 0;
    }
    template <class T> lair_status get(T **p, size_t n) {
        if (n == 0) n = 1;
        const size_t bytes = arena_round(n * sizeof(T));
        if (depth != h->tmp_depth) {
            void *q = nullptr;
            TRY(raw_alloc(h, &q, bytes));
            raw.push_back(q);
            *p = static_cast<T *>(q);
            return LAIR_OK;
        }
        auto &ch = h->tmp_chunks;
        if (h->tmp_cur < 0 || ch[h->tmp_cur].used + bytes > ch[h->tmp_cur].size) {
            // the next chunk if it is large enough, else a new one in its place
            const int nx = h->tmp_cur + 1;
            if (nx < (int)ch.size() && ch[nx].size >= bytes) {
                ch[nx].used = 0;
            } else {
                size_t sz = TMP_CHUNK_MIN;
                if (2 * bytes > sz) sz = 2 * bytes;
                void *np = nullptr;
                TRY(raw_alloc(h, &np, sz));
                h->allocs.push_back(np);
                ch.insert(ch.begin() + nx, lair_handle::Chunk{static_cast<char *>(np), sz, 0});
            }
            h->tmp_cur = nx;
        }
        auto &c = ch[h->tmp_cur];
        *p = reinterpret_cast<T *>(c.p + c.used);
        c.used += bytes;
        return LAIR_OK;
    }
    ~Temps() {
        for (void *q : raw) dfree(h, q);
        if (depth == h->tmp_depth) {
            h->tmp_cur = mark_cur;
            if (mark_cur >= 0) h->tmp_chunks[mark_cur].used = mark_used;
        }
        --h->tmp_depth;
    }
};

static inline void flush_timers(lair_handle *h);

static inline lair_status sync_status(lair_handle *h) {
    CU(cudaMemcpyAsync(h->h_int, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    flush_timers(h);
    int st = h->h_int[0];
    if (st != 0) {
        CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->s));
        return fail(h, (lair_status)st, "device reported %s", lair_status_string((lair_status)st));
    }
    return LAIR_OK;
}

// read n device ints into pageable host memory (any n)
static inline lair_status read_ints_big(lair_handle *h, const int *d, int n, int *out) {
    CU(cudaMemcpyAsync(out, d, sizeof(int) * n, cudaMemcpyDeviceToHost, h->s));
    return sync_status(h);
}

static inline lair_status read_ints(lair_handle *h, const int *d, int n, int *out) {
    CU(cudaMemcpyAsync(h->h_int + 1, d, sizeof(int) * n, cudaMemcpyDeviceToHost, h->s));
    TRY(sync_status(h));
    memcpy(out, h->h_int + 1, sizeof(int) * n);
    return LAIR_OK;
}

// ---------------------------------------------------------------------------------------
// kernel timers: events around selected launches, read back at the next host sync
// ---------------------------------------------------------------------------------------
static inline int timer_slot(lair_handle *h, const std::string &name, double bytes) {
    for (size_t i = 0; i < h->timers.size(); ++i)
        if (h->timers[i].name == name) return (int)i;
    lair_handle::Timer t;
    t.name = name;
    t.bytes = bytes;
    h->timers.push_back(t);
    return (int)h->timers.size() - 1;
}

static inline cudaEvent_t get_event(lair_handle *h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// begin/end around one launch; in_graph: the events become nodes of the graph being captured
// returns the index of the event pair (for tend), or -1 when timing is off
// set-up phase timer name; with timing >= 2 every level gets its own timer
static inline std::string phase_name(const lair_handle *h, const char *phase, int level) {
    std::string s = std::string("setup_") + phase;
    if (h->o.timing >= 2 && level >= 0) s += "_L" + std::to_string(level);
    return s;
}

static inline int tbegin(lair_handle *h, const std::string &name, double bytes, bool in_graph = false) {
    if (!h->o.timing) return -1;
    int slot = timer_slot(h, name, bytes);
    lair_handle::Pending p{slot, get_event(h), get_event(h), false, h->next_timer_id++};
    // inside stream capture only an external record becomes an event node of the graph
    if (in_graph) cudaEventRecordWithFlags(p.a, h->s, cudaEventRecordExternal);
    else cudaEventRecord(p.a, h->s);
    auto &v = in_graph ? h->graph_events : h->pending;
    v.push_back(p);
    return p.id;
}

static inline void tend(lair_handle *h, int id, bool in_graph = false) {
    if (id < 0) return;
    auto &v = in_graph ? h->graph_events : h->pending;
    for (size_t q = v.size(); q-- > 0;) {
        if (v[q].id != id) continue;
        if (in_graph) cudaEventRecordWithFlags(v[q].b, h->s, cudaEventRecordExternal);
        else cudaEventRecord(v[q].b, h->s);
        v[q].closed = true;
        return;
    }
}

// call only after the stream has been synchronised
static inline void flush_timers(lair_handle *h) {
    if (!h->o.timing) return;
    // pairs still open (a region spanning this synchronisation) stay pending
    std::vector<lair_handle::Pending> open;
    for (auto &p : h->pending) {
        if (!p.closed) {
            open.push_back(p);
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->timers[p.slot].ms += ms;
            h->timers[p.slot].launches += 1;
        }
        h->ev_pool.push_back(p.a);
        h->ev_pool.push_back(p.b);
    }
    h->pending.swap(open);
    if (h->graph_pending) {
        for (auto &p : h->graph_events) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                h->timers[p.slot].ms += ms;
                h->timers[p.slot].launches += 1;
            }
        }
        h->graph_pending = false;
    }
    cudaGetLastError();
}

// exclusive scan of cnt[0..n) into out[0..n] (out[n] = total); returns the total
static inline lair_status scan(lair_handle *h, const int *cnt, int *out, int n, int *total) {
    // cnt must have n+1 entries with cnt[n] = 0
    if (n + 1 <= SMALL_SCAN_MAX) {
        small_scan(n + 1, cnt, out, h->s);
        if (total) TRY(read_ints(h, out + n, 1, total));
        return LAIR_OK;
    }
    const size_t need = scan_state_bytes((long long)n + 1);
    if (need > h->scan_tmp_bytes) {
        if (h->scan_tmp) CU(cudaFreeAsync(h->scan_tmp, h->s));
        CU(cudaMallocAsync(&h->scan_tmp, need, h->s));
        h->scan_tmp_bytes = need;
    }
    CU(launch_scan((long long)n + 1, cnt, out, h->scan_tmp, h->status, h->s));
    if (total) TRY(read_ints(h, out + n, 1, total));
    return LAIR_OK;
}

static inline lair_status new_counts(lair_handle *h, Temps &t, int **p, int n) {
    TRY(t.get(p, (size_t)n + 1));
    CU(cudaMemsetAsync(*p, 0, sizeof(int) * ((size_t)n + 1), h->s));
    return LAIR_OK;
}

static inline double bytes_spmv(const DCsr &M, double sv) {
    return (double)M.nnz * (sv + 4.0) + (double)M.nr * (4.0 + sv) + (double)M.nc * sv;
}
// x = P x_c with one-point P from its column array: a column per row, a gathered x_c per entry, x written
static inline double bytes_p1(const DCsr &P, double sv) {
    return (double)P.nr * (4.0 + sv) + (double)P.nnz * sv;
}

// true for device (or managed) memory
static inline bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// outer loops (lair_solve.cu)
lair_status ensure_work(lair_handle *h, int n, int m);
lair_status precond(lair_handle *h, Hier &H, const double *v, double *z);
lair_status run_solve(lair_handle *h, Hier &H, const double *b, double *x, double tol, int cycle, int max_iter,
                      lair_report *rep, bool scale);
lair_status solve_batched_dev(lair_handle *h, Hier &H, const double *b, double *x, double tol, int max_iter,
                              int *iters, double *rel);
lair_status solve_batched_fgmres(lair_handle *h, Hier &H, const double *b, double *x, double tol, int max_iter,
                                 int *iters, double *rel);

}  // namespace lair
