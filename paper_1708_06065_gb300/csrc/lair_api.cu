// lair_api.cu -- set-up orchestration (Sec. 2.1 and Sec. 4, level by level) and the C ABI declared
// in include/lair.h; the outer iterations are in lair_solve.cu.
//
// Set-up runs level by level on the handle's stream; the host reads back only a few
// sizes per level (coarse count, pattern sizes, bin counts) to size the next
// allocations. The V-cycle of each hierarchy is captured once into a CUDA graph and
// replayed for every preconditioner application.

#include "lair_host.cuh"

namespace lair {

int device_sms() {
    constexpr int MAXDEV = 64;
    static std::atomic<int> cache[MAXDEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 152;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

static thread_local long long *g_launches = nullptr;
void count_launch(int k) {
    if (g_launches) *g_launches += k;
}

cudaError_t lair_pool(cudaMemPool_t *out) {
    static std::mutex mu;
    static cudaMemPool_t pools[POOL_DEVICES] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= POOL_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = POOL_KEEP;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

static std::mutex g_host_mu;
static std::vector<void *> g_host_free;

cudaError_t host_block_get(void **p) {
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        if (!g_host_free.empty()) {
            *p = g_host_free.back();
            g_host_free.pop_back();
            return cudaSuccess;
        }
    }
    return cudaMallocHost(p, HOST_BLOCK);
}

void host_block_put(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_host_mu);
    g_host_free.push_back(p);
}
// ---------------------------------------------------------------------------------------
// graphs and transposes
// ---------------------------------------------------------------------------------------
static lair_status build_strength_graph(lair_handle *h, Temps &t, const DCsr &A, double theta, uint8_t *mask, Graph &G,
                                        int absmode) {
    int *cnt;
    TRY(new_counts(h, t, &cnt, A.nr));
    launch_strength(A, theta, absmode, mask, cnt, h->s);
    G.n = A.nr;
    TRY(t.get(&G.rp, (size_t)A.nr + 1));
    // S is a subset of the pattern of A, so A's entry count bounds it and no read-back is needed
    TRY(scan(h, cnt, G.rp, A.nr, nullptr));
    G.nnz = A.nnz;
    TRY(t.get(&G.col, (size_t)G.nnz));
    launch_graph_fill(A, mask, G, h->s);
    return LAIR_OK;
}

// transpose of an nr x nc CSR (values optional); output rows sorted by column
static lair_status transpose(lair_handle *h, Temps &t, int nr, int nc, int nnz, const int *rp, const int *col,
                             const double *val, int **trp, int **tcol, double **tval, bool keep) {
    int *cnt;
    TRY(new_counts(h, t, &cnt, nc));
    launch_col_count(nr, rp, col, cnt, h->s);
    if (keep) TRY(dalloc(h, trp, (size_t)nc + 1));
    else TRY(t.get(trp, (size_t)nc + 1));
    TRY(scan(h, cnt, *trp, nc, nullptr));
    CU(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)nc + 1), h->s));
    if (keep) {
        TRY(dalloc(h, tcol, (size_t)nnz));
        if (val) TRY(dalloc(h, tval, (size_t)nnz));
    } else {
        TRY(t.get(tcol, (size_t)nnz));
        if (val) TRY(t.get(tval, (size_t)nnz));
    }
    launch_transpose_scatter(nr, rp, col, val, *trp, cnt, *tcol, val ? *tval : nullptr, h->s);
    int *lists;
    TRY(t.get(&lists, 2 * (size_t)nc + 2));
    CU(cudaMemsetAsync(lists, 0, 2 * sizeof(int), h->s));
    launch_sort_rows(nc, *trp, *tcol, val ? *tval : nullptr, lists, h->s);
    return LAIR_OK;
}

// ---------------------------------------------------------------------------------------
// launch-schedule autotuner of the local solves: for a batch of at least
// LOCAL_TUNE_MIN systems whose shape (precision, shared sets, Neumann series, count, mean and largest
// size) has not been seen in this process, every candidate schedule bins and solves the batch, timed
// best of three with CUDA events; the fastest replaces the default when it is more than 5 % faster.
// Each system is solved by the same operations whatever team holds it, so the rows written are the
// same bits under every candidate, and the last run leaves the right result in place.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int LOCAL_TUNE_MIN = 65536;
struct LocalKey {
    int dev, fp32, shared, neumann, count, mean4, smax;
    bool operator<(const LocalKey &o) const {
        return std::tie(dev, fp32, shared, neumann, count, mean4, smax) <
               std::tie(o.dev, o.fp32, o.shared, o.neumann, o.count, o.mean4, o.smax);
    }
};
std::mutex g_local_tune_mu;
std::map<LocalKey, LocalSchedule> g_local_tune;
// (tmax, wmax, warp blocks per SM, thread-kernel block); the first is the default
const LocalSchedule kLocalCandidates[] = {{6, 32, 8, 128}, {4, 32, 8, 128}, {0, 32, 8, 128}, {6, 32, 16, 128},
                                          {6, 32, 4, 128}, {6, 32, 8, 64},  {6, 16, 8, 128}, {2, 32, 16, 64}};
}  // namespace

// bins the ng systems of nb_rp (stride: rows sharing one set) with schedule sch and solves them; hc gets the
// bin counts and the largest size
static lair_status bin_and_solve(lair_handle *h, Temps &t, const LocalArgs &a, int ng, const int *nb_rp, int stride,
                                 int *lists, int *bcounts, const LocalSchedule &sch, void **scratch, size_t *scratch_bytes,
                                 int hc[4]) {
    const bool fp32 = h->o.precision == LAIR_MIXED;
    CU(cudaMemsetAsync(bcounts, 0, sizeof(int) * 4, h->s));
    launch_local_bin(ng, nb_rp, lists, bcounts, bcounts + 3, h->s, stride, sch.tmax, sch.wmax);
    TRY(read_ints(h, bcounts, 4, hc));
    if (hc[2] > 0 && local_cta_scratch_bytes(hc[3], fp32) > *scratch_bytes) {
        unsigned char *sp;
        *scratch_bytes = local_cta_scratch_bytes(hc[3], fp32);
        TRY(t.get(&sp, *scratch_bytes));
        *scratch = sp;
    }
    CU(launch_local_solves(a, ng, lists, bcounts, hc, hc[3], fp32, *scratch, h->s, sch));
    return LAIR_OK;
}

// the local solves of a batch (binned once with the default schedule into lists / bcounts, hc); tuned first when
// the autotuner is on and the batch is large and new
static lair_status run_local_solves(lair_handle *h, Temps &t, const LocalArgs &a, int ng, const int *nb_rp, int stride,
                                    int nnb, int *lists, int *bcounts, int hc[4], int level) {
    const bool fp32 = h->o.precision == LAIR_MIXED;
    void *scratch = nullptr;
    size_t sbytes = 0;
    if (hc[2] > 0) {
        unsigned char *sp;
        sbytes = local_cta_scratch_bytes(hc[3], fp32);
        TRY(t.get(&sp, sbytes));
        scratch = sp;
    }
    LocalSchedule pick;
    bool tuned = false;
    if (h->o.autotune && ng >= LOCAL_TUNE_MIN) {
        int dev = 0;
        CU(cudaGetDevice(&dev));
        const double mean = ng ? (double)nnb / ng : 0.0;
        const LocalKey key{dev, fp32 ? 1 : 0, stride > 1 ? 1 : 0, a.neumann_deg >= 0 ? 1 : 0,
                           (int)std::floor(4.0 * std::log2((double)ng)), (int)std::lround(4.0 * mean),
                           hc[3] > 0 ? (int)std::ceil(std::log2((double)hc[3])) : 0};
        bool found = false;
        {
            std::lock_guard<std::mutex> g(g_local_tune_mu);
            auto it = g_local_tune.find(key);
            if (it != g_local_tune.end()) {
                pick = it->second;
                found = true;
            }
        }
        if (found && h->o.timing) {
            char nm[96];
            snprintf(nm, sizeof nm, "tune_local_L%d:t%dw%dg%db%d cached", level, pick.tmax, pick.wmax,
                     pick.warp_blocks_per_sm, pick.thread_tb);
            h->timers[timer_slot(h, nm, 0.0)].launches += 1;
        }
        if (!found) {
            cudaEvent_t e0 = get_event(h), e1 = get_event(h);
            float best = 3.4e38f, base = 3.4e38f;
            int bi = 0;
            for (int ci = 0; ci < (int)(sizeof(kLocalCandidates) / sizeof(kLocalCandidates[0])); ++ci) {
                const LocalSchedule &c = kLocalCandidates[ci];
                int hcc[4];
                TRY(bin_and_solve(h, t, a, ng, nb_rp, stride, lists, bcounts, c, &scratch, &sbytes, hcc));   // warm
                float tmin = 3.4e38f;
                for (int rep = 0; rep < 3; ++rep) {
                    CU(cudaEventRecord(e0, h->s));
                    CU(launch_local_solves(a, ng, lists, bcounts, hcc, hcc[3], fp32, scratch, h->s, c));
                    CU(cudaEventRecord(e1, h->s));
                    CU(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CU(cudaEventElapsedTime(&ms, e0, e1));
                    tmin = std::min(tmin, ms);
                }
                if (ci == 0) base = tmin;
                if (tmin < best) {
                    best = tmin;
                    bi = ci;
                }
            }
            h->ev_pool.push_back(e0);
            h->ev_pool.push_back(e1);
            if (!(best < 0.95f * base)) {
                bi = 0;
                best = base;
            }
            pick = kLocalCandidates[bi];
            {
                std::lock_guard<std::mutex> g(g_local_tune_mu);
                g_local_tune[key] = pick;
            }
            if (h->o.timing) {
                // the choice and its time (one timer per tuned batch: "tune_local_L<level>:t<tmax>w<wmax>g<cap>b<tb>")
                char nm[96];
                snprintf(nm, sizeof nm, "tune_local_L%d:t%dw%dg%db%d base=%.3fms", level, pick.tmax, pick.wmax,
                         pick.warp_blocks_per_sm, pick.thread_tb, (double)base);
                const int slot = timer_slot(h, nm, 0.0);
                h->timers[slot].ms += best;
                h->timers[slot].launches += 1;
            }
        }
        tuned = true;
    }
    if (!tuned) {
        CU(launch_local_solves(a, ng, lists, bcounts, hc, hc[3], fp32, scratch, h->s));
        return LAIR_OK;
    }
    int hcc[4];
    return bin_and_solve(h, t, a, ng, nb_rp, stride, lists, bcounts, pick, &scratch, &sbytes, hcc);
}

// ---------------------------------------------------------------------------------------
// local solves: neighbourhoods of C points in graph G, systems of matrix B, rows into out
// ---------------------------------------------------------------------------------------
static lair_status local_rows(lair_handle *h, Temps &t, int nc, const int *cpts, const Graph &G, const int8_t *cf,
                              const int *brp, const int *bcol, const double *bval, int **out_rp, int **out_col,
                              double **out_val, float **out_val32, uint8_t *lsflag, int *out_nnz, bool keep,
                              int neumann_deg = -1, int level = -1) {
    const int distance = h->o.distance, d0 = distance < 2 ? distance : 2;
    int *ub, *off, *tmp, *cnt, *nb_rp, *nb_col;
    TRY(new_counts(h, t, &ub, nc));
    launch_nb_bound(nc, cpts, G, cf, d0, ub, h->s);
    TRY(t.get(&off, (size_t)nc + 1));
    int total = 0;
    TRY(scan(h, ub, off, nc, &total));
    TRY(t.get(&tmp, (size_t)total));
    TRY(new_counts(h, t, &cnt, nc));
    launch_nb_fill(nc, cpts, G, cf, d0, off, tmp, cnt, h->s);
    TRY(t.get(&nb_rp, (size_t)nc + 1));
    TRY(scan(h, cnt, nb_rp, nc, nullptr));
    // distances beyond two: expand the sets one distance at a time
    for (int d = 3; d <= distance; ++d) {
        int nn = 0, tot = 0;
        TRY(read_ints(h, nb_rp + nc, 1, &nn));
        int *cur, *ub2, *off2, *tmp2, *cnt2, *rp2;
        TRY(t.get(&cur, (size_t)nn));
        launch_nb_compact(nc, off, tmp, nb_rp, cur, h->s);
        TRY(new_counts(h, t, &ub2, nc));
        launch_nb_expand(0, nc, cpts, G, cf, nb_rp, cur, nullptr, nullptr, ub2, h->s);
        TRY(t.get(&off2, (size_t)nc + 1));
        TRY(scan(h, ub2, off2, nc, &tot));
        TRY(t.get(&tmp2, (size_t)tot));
        TRY(new_counts(h, t, &cnt2, nc));
        launch_nb_expand(1, nc, cpts, G, cf, nb_rp, cur, off2, tmp2, cnt2, h->s);
        TRY(t.get(&rp2, (size_t)nc + 1));
        TRY(scan(h, cnt2, rp2, nc, nullptr));
        off = off2;
        tmp = tmp2;
        cnt = cnt2;
        nb_rp = rp2;
    }
    // size bins of the local systems; one read-back for the bins and the neighbourhood total
    int *lists, *bcounts, *smax;
    TRY(t.get(&lists, (size_t)3 * nc + 1));
    TRY(new_counts(h, t, &bcounts, 5));
    smax = bcounts + 3;
    launch_local_bin(nc, nb_rp, lists, bcounts, smax, h->s);
    CU(cudaMemcpyAsync(bcounts + 4, nb_rp + nc, sizeof(int), cudaMemcpyDeviceToDevice, h->s));
    int hc[5];
    TRY(read_ints(h, bcounts, 5, hc));
    const int nnb = hc[4];
    TRY(t.get(&nb_col, (size_t)nnb));
    launch_nb_compact(nc, off, tmp, nb_rp, nb_col, h->s);

    // output row pointers: nb_rp[c] + c
    const int nout = nnb + nc;
    int *orp;
    if (keep) TRY(dalloc(h, &orp, (size_t)nc + 1)); else TRY(t.get(&orp, (size_t)nc + 1));
    {
        int *c2;   // c2[c] = s_c + 1
        TRY(new_counts(h, t, &c2, nc));
        plus_one(nc, cnt, c2, h->s);
        TRY(scan(h, c2, orp, nc, nullptr));
    }
    int *ocol;
    double *oval;
    float *oval32 = nullptr;
    const bool fp32 = h->o.precision == LAIR_MIXED;
    if (keep) {
        TRY(dalloc(h, &ocol, (size_t)nout));
        TRY(dalloc(h, &oval, (size_t)nout));
        if (fp32 && out_val32) TRY(dalloc(h, &oval32, (size_t)nout));
    } else {
        TRY(t.get(&ocol, (size_t)nout));
        TRY(t.get(&oval, (size_t)nout));
    }
    LocalArgs a{cpts, nb_rp, nb_col, brp, bcol, bval, ocol, oval, oval32, lsflag, neumann_deg};
    TRY(run_local_solves(h, t, a, nc, nb_rp, 1, nnb, lists, bcounts, hc, level));
    *out_nnz = nout;
    *out_rp = orp;
    *out_col = ocol;
    *out_val = oval;
    if (out_val32) *out_val32 = oval32;
    return LAIR_OK;
}

// Z = X Y, canonical accumulation order (see setup_rap.cu)
// Z = X Y, or Z = X Y P when P (one-point: at most one entry per row) is given; the triple product is
// formed in one pass when every row of X Y fits the short-row kernels, else as (X Y) P.
// timed (0 or 1): the product's row pass is timed as "L0_RA" / "L0_RAP" and its entry count kept
// With stage_len, Z is left in the staging area (not compacted): row a is Z.col/Z.val[Z.rp[a],
// Z.rp[a] + (*stage_len)[a]); Z.nnz is then only the capacity.
static lair_status spgemm(lair_handle *h, Temps &t, const DCsr &X, const DCsr &Y, DCsr &Z, bool keep, int timed = -1,
                          const DCsr *P = nullptr, int **stage_len = nullptr) {
    const int nr = X.nr;
    int *ub, *off;
    TRY(new_counts(h, t, &ub, nr));
    launch_spgemm_ub(nr, X.rp, X.col, Y.rp, ub, h->s);
    TRY(t.get(&off, (size_t)nr + 1));
    TRY(scan(h, ub, off, nr, nullptr));
    int *tcol, *cnt, *lists, *bc;
    double *tval;
    TRY(new_counts(h, t, &cnt, nr));
    TRY(t.get(&lists, (size_t)SPGEMM_BINS * nr + 1));
    TRY(new_counts(h, t, &bc, SPGEMM_BINS + 2));
    // thread-per-row merging needs many rows to keep the GPU busy; short products stay on warps
    const bool merge = nr >= SPGEMM_MERGE_MIN_ROWS;
    launch_spgemm_classify(nr, off, X.rp, merge, merge && P == nullptr, P ? SPGEMM_P1_CAP : 0x7fffffff, lists, bc,
                           bc + SPGEMM_BINS, h->s);
    // one read-back: bin counts, largest bound, and the total bound (staging size)
    CU(cudaMemcpyAsync(bc + SPGEMM_BINS + 1, off + nr, sizeof(int), cudaMemcpyDeviceToDevice, h->s));
    int hc[SPGEMM_BINS + 2];
    TRY(read_ints(h, bc, SPGEMM_BINS + 2, hc));
    const int total = hc[SPGEMM_BINS + 1];
    if (P && !spgemm_can_fuse(hc)) {
        DCsr XY;
        TRY(spgemm(h, t, X, Y, XY, false, timed >= 0 ? 0 : -1));
        return spgemm(h, t, XY, *P, Z, keep, timed >= 0 ? 1 : -1, nullptr, stage_len);
    }
    TRY(t.get(&tcol, (size_t)total));
    TRY(t.get(&tval, (size_t)total));
    int *skeys = nullptr;
    double *svals = nullptr;
    const int nbig = hc[SPGEMM_BIN_CTA], ubmax = hc[SPGEMM_BINS];
    if (nbig > 0) {
        size_t cap = spgemm_big_cap(ubmax);
        size_t slots = 2 * cap * (size_t)(nbig < SPGEMM_CTA_GRID ? nbig : SPGEMM_CTA_GRID);
        TRY(t.get(&skeys, slots));
        TRY(t.get(&svals, slots));
    }
    SpgemmArgs g{X.rp, X.col, X.val, Y.rp, Y.col, Y.val, off, tcol, tval, cnt};
    if (P) {
        g.prp = P->rp;
        g.pcol = P->col;
        g.pval = P->val;
        g.pn = P->nr;
        if (hc[SPGEMM_BIN_MERGE] > 0) {
            TRY(t.get(&g.pmap_col, (size_t)P->nr + 1));
            TRY(t.get(&g.pmap_val, (size_t)P->nr + 1));
        }
        if (timed >= 0) h->prod_fused = true;
    }
    int tp = -1;
    if (timed >= 0 && h->o.timing) tp = tbegin(h, timed == 0 ? "L0_RA" : "L0_RAP", 0.0);
    CU(launch_spgemm_rows(g, nr, lists, bc, hc, ubmax, skeys, svals, h->s));
    tend(h, tp);
    Z.nr = nr;
    Z.nc = P ? P->nc : Y.nc;
    if (stage_len && !keep) {
        Z.rp = off;
        Z.col = tcol;
        Z.val = tval;
        Z.nnz = total;
        *stage_len = cnt;
        if (timed >= 0 && h->o.timing) {
            // the exact entry count, for the byte model
            int *cs;
            TRY(t.get(&cs, (size_t)nr + 1));
            TRY(scan(h, cnt, cs, nr, nullptr));
            if (!h->prod_nnz) TRY(dalloc(h, &h->prod_nnz, 2));
            CU(cudaMemcpyAsync(h->prod_nnz + timed, cs + nr, sizeof(int), cudaMemcpyDeviceToDevice, h->s));
        }
        return LAIR_OK;
    }
    if (keep) TRY(dalloc(h, &Z.rp, (size_t)nr + 1)); else TRY(t.get(&Z.rp, (size_t)nr + 1));
    // a kept product is stored at its exact size; a temporary one at the bound (its entry count
    // is then only a capacity and is not read back)
    if (keep) TRY(scan(h, cnt, Z.rp, nr, &Z.nnz));
    else {
        TRY(scan(h, cnt, Z.rp, nr, nullptr));
        Z.nnz = total;
    }
    if (keep) {
        TRY(dalloc(h, &Z.col, (size_t)Z.nnz));
        TRY(dalloc(h, &Z.val, (size_t)Z.nnz));
    } else {
        TRY(t.get(&Z.col, (size_t)Z.nnz));
        TRY(t.get(&Z.val, (size_t)Z.nnz));
    }
    launch_copy_rows(nr, off, tcol, tval, Z, h->s);
    if (timed >= 0 && h->o.timing) {
        if (!h->prod_nnz) TRY(dalloc(h, &h->prod_nnz, 2));
        CU(cudaMemcpyAsync(h->prod_nnz + timed, Z.rp + nr, sizeof(int), cudaMemcpyDeviceToDevice, h->s));
    }
    return LAIR_OK;
}

// C/F splitting of the n points of the graphs (Scf, STcf) into cf (level l): RS, the exact first pass (one
// block per system); AUTO, the first pass in blocks of rs_block points, never spanning two batched systems;
// or PMIS
static lair_status split_points(lair_handle *h, Temps &t, int l, int n, const Graph &Scf, const Graph &STcf,
                                const std::vector<int> &seg_h, int8_t *cf) {
    const lair_options &o = h->o;
    if (o.cf_mode != LAIR_CF_PMIS) {
        // RS: the exact first pass (one block per system); AUTO: the first pass in blocks of rs_block points.
        // Blocks never span two batched systems.
        std::vector<int> cuts = seg_h;
        if (cuts.empty()) cuts = {0, n};
        std::vector<int2> blocks;
        int Bmax = 1;
        for (size_t q = 0; q + 1 < cuts.size(); ++q) {
            const int s0 = cuts[q], s1 = cuts[q + 1];
            const int B = o.cf_mode == LAIR_CF_RS ? (s1 - s0) : o.rs_block;
            if (B > RS_MAX_N)
                return fail(h, LAIR_ERR_UNSUPPORTED,
                            "the first pass runs on at most %d points at once (level %d has %d)", RS_MAX_N, l, B);
            for (int b0 = s0; b0 < s1; b0 += B) {
                int b1 = b0 + B < s1 ? b0 + B : s1;
                blocks.push_back(make_int2(b0, b1));
                if (b1 - b0 > Bmax) Bmax = b1 - b0;
            }
        }
        int2 *bd;
        TRY(t.get(&bd, blocks.size()));
        CU(cudaMemcpyAsync(bd, blocks.data(), sizeof(int2) * blocks.size(), cudaMemcpyHostToDevice, h->s));
        // in-block entries of S, largest in-block row lengths of S and ST: they size the bucket queue
        int *mx, deg[3] = {0, 0, 0};
        TRY(new_counts(h, t, &mx, 3));
        launch_rs_degrees(bd, (int)blocks.size(), Scf, STcf, mx, h->s);
        TRY(read_ints(h, mx, 3, deg));   // also keeps the host block list alive until its copy is done
        int nb = 8;
        while (nb < 2 * deg[2] + 1) nb *= 2;
        const long long dl = 32 + (long long)deg[1] * (1 + deg[2]);
        if (Bmax <= RSB_MAX_N && nb <= 256 && dl <= RSB_MAX_DIRTY &&
            rsb_smem_bytes(Bmax, nb, (int)dl) <= (size_t)200 * 1024) {
            CU(launch_rs_bucket(bd, (int)blocks.size(), Bmax, nb, (int)dl, deg[0], Scf, STcf, cf, h->status, h->s));
        } else {
            CU(launch_rs(n, bd, (int)blocks.size(), Bmax, deg[0], Scf, STcf, cf, h->status, h->s));
        }
    } else {
        double *w;
        int8_t *newc;
        int *und;
        TRY(t.get(&w, (size_t)n));
        TRY(t.get(&newc, (size_t)n));
        int *lists;
        TRY(t.get(&lists, 2 * (size_t)n));
        TRY(new_counts(h, t, &und, 4));
        launch_pmis_init(n, STcf, o.pmis_seed + (uint64_t)l, w, cf, h->s);
        CU(launch_pmis_all(n, Scf, STcf, w, cf, newc, lists, und, h->status, o.wait_polls, h->s));
    }
    return LAIR_OK;
}

// ---------------------------------------------------------------------------------------
// one coarsening step: level l -> level l+1
// ---------------------------------------------------------------------------------------
static lair_status coarsen(lair_handle *h, Hier &H, int l, const int8_t *cf_user, bool *last) {
    Temps t(h);
    Level &L = H.lev[l];
    const DCsr &A = L.A;
    const lair_options &o = h->o;
    const int n = A.nr;
    const bool fp32 = o.precision == LAIR_MIXED;

    int tp = tbegin(h, phase_name(h, "strength", l), 0.0);
    TRY(dalloc(h, &L.strong, (size_t)A.nnz));
    Graph S, ST, Scf, STcf;
    TRY(build_strength_graph(h, t, A, o.theta, L.strong, S, o.strength_abs));
    TRY(transpose(h, t, n, n, S.nnz, S.rp, S.col, nullptr, &ST.rp, &ST.col, nullptr, false));
    ST.n = n;
    ST.nnz = S.nnz;
    if (o.theta_cf != o.theta) {
        uint8_t *m2;
        TRY(t.get(&m2, (size_t)A.nnz));
        TRY(build_strength_graph(h, t, A, o.theta_cf, m2, Scf, o.strength_abs));
        TRY(transpose(h, t, n, n, Scf.nnz, Scf.rp, Scf.col, nullptr, &STcf.rp, &STcf.col, nullptr, false));
        STcf.n = n;
        STcf.nnz = Scf.nnz;
    } else {
        Scf = S;
        STcf = ST;
    }

    // ---- C/F splitting
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "split", l), 0.0);
    TRY(dalloc(h, &L.cf, (size_t)n));
    if (cf_user) {
        CU(cudaMemcpyAsync(L.cf, cf_user, (size_t)n, cudaMemcpyHostToDevice, h->s));
        normalize_cf(n, L.cf, h->s);
    } else {
        TRY(split_points(h, t, l, n, Scf, STcf, L.seg_h, L.cf));
    }
    // the status word (first-pass errors) is checked with the next read-back

    // ---- coarse numbering
    int *flag, *scanv, *cpts;
    TRY(new_counts(h, t, &flag, n));
    launch_cidx(n, L.cf, flag, nullptr, nullptr, 0, h->s);
    TRY(t.get(&scanv, (size_t)n + 1));
    int nc = 0;
    TRY(scan(h, flag, scanv, n, &nc));
    L.nc = nc;
    if (nc == 0 || nc == n) {
        tend(h, tp);
        *last = true;
        return LAIR_OK;
    }
    TRY(dalloc(h, &L.cidx, (size_t)n));
    TRY(dalloc(h, &cpts, (size_t)nc));
    launch_cidx(n, L.cf, scanv, L.cidx, cpts, 1, h->s);
    L.crows = cpts;
    if (n - nc > 0) {
        TRY(dalloc(h, &L.frows, (size_t)(n - nc)));
        launch_frows(n, L.cf, scanv, L.frows, h->s);
    }
    std::vector<int> next_seg;
    if (!L.seg_h.empty()) {
        // a system's first coarse point: number of C points before its first fine point
        const int m = (int)L.seg_h.size();
        int *g;
        TRY(t.get(&g, (size_t)m));
        gather_int(m, L.seg_d, scanv, g, h->s);
        next_seg.resize(m);
        CU(cudaMemcpyAsync(next_seg.data(), g, sizeof(int) * m, cudaMemcpyDeviceToHost, h->s));
        TRY(sync_status(h));
    }

    // ---- restriction (lAIR): local systems of A on the neighbourhoods in S
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "R", l), 0.0);
    TRY(dalloc(h, &L.lsR, (size_t)nc));
    L.R.nr = nc;
    L.R.nc = n;
    if (o.restriction == LAIR_R_NEUMANN) {
        // nAIR: sets from the graph of every nonzero off-diagonal (theta 0 in abs mode), series of degree distance - 1
        Graph GA;
        uint8_t *all;
        TRY(t.get(&all, (size_t)A.nnz));
        TRY(build_strength_graph(h, t, A, 0.0, all, GA, 1));
        TRY(local_rows(h, t, nc, cpts, GA, L.cf, A.rp, A.col, A.val, &L.R.rp, &L.R.col, &L.R.val,
                       fp32 ? &L.R.val32 : nullptr, L.lsR, &L.R.nnz, true, o.distance - 1, l));
    } else {
        TRY(local_rows(h, t, nc, cpts, S, L.cf, A.rp, A.col, A.val, &L.R.rp, &L.R.col, &L.R.val,
                       fp32 ? &L.R.val32 : nullptr, L.lsR, &L.R.nnz, true, -1, l));
    }

    // ---- interpolation
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "P", l), 0.0);
    L.P.nr = n;
    L.P.nc = nc;
    if (o.interp == LAIR_P_ONEPOINT) {
        int *choice, *cnt;
        TRY(t.get(&choice, (size_t)n));
        TRY(new_counts(h, t, &cnt, n));
        launch_onepoint(0, A, L.strong, L.cf, L.cidx, o.strength_abs, choice, cnt, nullptr, h->s);
        TRY(dalloc(h, &L.P.rp, (size_t)n + 1));
        // at most one entry per row: stored with room for n, exact count read back with the
        // other hierarchy totals once the hierarchy is built
        TRY(scan(h, cnt, L.P.rp, n, nullptr));
        L.P.nnz = n;
        TRY(dalloc(h, &L.P.col, (size_t)n));
        TRY(dalloc(h, &L.P.val, (size_t)n));
        if (fp32) TRY(dalloc(h, &L.P.val32, (size_t)n));
        launch_onepoint(1, A, L.strong, L.cf, L.cidx, o.strength_abs, choice, cnt, &L.P, h->s);
    } else {
        // approximate ideal interpolation = lAIR applied to A^T on the transposed graph, transposed back
        int *atrp, *atcol;
        double *atval;
        TRY(transpose(h, t, n, n, A.nnz, A.rp, A.col, A.val, &atrp, &atcol, &atval, false));
        TRY(dalloc(h, &L.lsP, (size_t)nc));
        int *wrp, *wcol;
        double *wval;
        int wnnz = 0;
        TRY(local_rows(h, t, nc, cpts, ST, L.cf, atrp, atcol, atval, &wrp, &wcol, &wval, nullptr, L.lsP, &wnnz,
                       false, -1, l));
        TRY(transpose(h, t, nc, n, wnnz, wrp, wcol, wval, &L.P.rp, &L.P.col, &L.P.val, true));
        L.P.nnz = wnnz;
        if (fp32) {
            TRY(dalloc(h, &L.P.val32, (size_t)wnnz));
            launch_to_f32(wnnz, L.P.val, L.P.val32, h->s);
        }
    }

    // ---- Galerkin product and lumping
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "RAP", l), 0.0);
    DCsr RA, K;
    const bool lump = o.lump_tol > 0.0;
    int *klen = nullptr;   // with lumping, K stays in the product's staging area (rows of length klen)
    if (o.interp == LAIR_P_ONEPOINT) {
        TRY(spgemm(h, t, L.R, A, K, !lump, l == 0 ? 1 : -1, &L.P, lump ? &klen : nullptr));
    } else {
        TRY(spgemm(h, t, L.R, A, RA, false, l == 0 ? 0 : -1));
        TRY(spgemm(h, t, RA, L.P, K, !lump, l == 0 ? 1 : -1, nullptr, lump ? &klen : nullptr));
    }
    Level next;
    if (lump) {
        int *cnt;
        double *nd;
        TRY(new_counts(h, t, &cnt, K.nr));
        TRY(t.get(&nd, 2 * (size_t)K.nr));
        launch_lump(0, K, klen, o.lump_tol, cnt, nd, nullptr, h->status, h->s);
        DCsr Kl;
        Kl.nr = Kl.nc = K.nr;
        TRY(dalloc(h, &Kl.rp, (size_t)K.nr + 1));
        TRY(scan(h, cnt, Kl.rp, K.nr, &Kl.nnz));
        TRY(dalloc(h, &Kl.col, (size_t)Kl.nnz));
        TRY(dalloc(h, &Kl.val, (size_t)Kl.nnz));
        launch_lump(1, K, klen, o.lump_tol, cnt, nd, &Kl, h->status, h->s);
        next.A = Kl;
    } else {
        next.A = K;
    }
    if (!next_seg.empty()) {
        next.seg_h = next_seg;
        TRY(dalloc(h, &next.seg_d, next_seg.size()));
        CU(cudaMemcpyAsync(next.seg_d, next.seg_h.data(), sizeof(int) * next_seg.size(), cudaMemcpyHostToDevice, h->s));
        CU(cudaStreamSynchronize(h->s));   // the host vector is copied from pageable memory
    }
    H.lev.push_back(next);
    tend(h, tp);
    *last = false;
    return LAIR_OK;
}

// local solves on kept sets (defined with the hierarchy refresh below)
static lair_status local_rows_on(lair_handle *h, Temps &t, int nc, const int *cpts, const int *rp, const int *col,
                                 int nnz, const int *brp, const int *bcol, const double *bval, int *ocol, double *oval,
                                 float *oval32, uint8_t *lsflag, int neumann_deg = -1, int rows_per = 1);

// the neighbourhoods (distance o.distance) of the nc points cpts in graph G with labels cf, compacted:
// set c is (*out_col)[(*out_rp)[c] .. (*out_rp)[c + 1]); *out_total entries in all
static lair_status build_sets(lair_handle *h, Temps &t, int nc, const int *cpts, const Graph &G, const int8_t *cf,
                              int **out_rp, int **out_col, int *out_total) {
    const int distance = h->o.distance, d0 = distance < 2 ? distance : 2;
    int *ub, *off, *tmp, *cnt, *nb_rp, *nb_col;
    TRY(new_counts(h, t, &ub, nc));
    launch_nb_bound(nc, cpts, G, cf, d0, ub, h->s);
    TRY(t.get(&off, (size_t)nc + 1));
    int total = 0;
    TRY(scan(h, ub, off, nc, &total));
    TRY(t.get(&tmp, (size_t)total + 1));
    TRY(new_counts(h, t, &cnt, nc));
    launch_nb_fill(nc, cpts, G, cf, d0, off, tmp, cnt, h->s);
    TRY(t.get(&nb_rp, (size_t)nc + 1));
    TRY(scan(h, cnt, nb_rp, nc, nullptr));
    for (int d = 3; d <= distance; ++d) {
        int nn = 0, tot = 0;
        TRY(read_ints(h, nb_rp + nc, 1, &nn));
        int *cur, *ub2, *off2, *tmp2, *cnt2, *rp2;
        TRY(t.get(&cur, (size_t)nn + 1));
        launch_nb_compact(nc, off, tmp, nb_rp, cur, h->s);
        TRY(new_counts(h, t, &ub2, nc));
        launch_nb_expand(0, nc, cpts, G, cf, nb_rp, cur, nullptr, nullptr, ub2, h->s);
        TRY(t.get(&off2, (size_t)nc + 1));
        TRY(scan(h, ub2, off2, nc, &tot));
        TRY(t.get(&tmp2, (size_t)tot + 1));
        TRY(new_counts(h, t, &cnt2, nc));
        launch_nb_expand(1, nc, cpts, G, cf, nb_rp, cur, off2, tmp2, cnt2, h->s);
        TRY(t.get(&rp2, (size_t)nc + 1));
        TRY(scan(h, cnt2, rp2, nc, nullptr));
        off = off2;
        tmp = tmp2;
        nb_rp = rp2;
    }
    int nnb = 0;
    TRY(read_ints(h, nb_rp + nc, 1, &nnb));
    TRY(t.get(&nb_col, (size_t)nnb + 1));
    launch_nb_compact(nc, off, tmp, nb_rp, nb_col, h->s);
    *out_rp = nb_rp;
    *out_col = nb_col;
    *out_total = nnb;
    return LAIR_OK;
}

// one coarsening step of the nodal hierarchy (nodes of k = o.nodal consecutive unknowns): strength,
// splitting, neighbourhoods and the one-point choice on the matrix of block norms, then R, P and R A P on
// the unknowns, lumping by block
static lair_status coarsen_nodal(lair_handle *h, Hier &H, int l, const int8_t *cf_user, bool *last) {
    Temps t(h);
    Level &L = H.lev[l];
    const DCsr &A = L.A;
    const lair_options &o = h->o;
    const int n = A.nr, k = o.nodal, N = n / k;
    const bool fp32 = o.precision == LAIR_MIXED;

    int tp = tbegin(h, phase_name(h, "strength", l), 0.0);
    DCsr B;
    B.nr = B.nc = N;
    int *bcnt;
    TRY(new_counts(h, t, &bcnt, N));
    launch_node_matrix(0, N, k, A, bcnt, nullptr, h->s);
    TRY(t.get(&B.rp, (size_t)N + 1));
    TRY(scan(h, bcnt, B.rp, N, &B.nnz));
    TRY(t.get(&B.col, (size_t)B.nnz + 1));
    TRY(t.get(&B.val, (size_t)B.nnz + 1));
    launch_node_matrix(1, N, k, A, nullptr, &B, h->s);
    uint8_t *smask;
    TRY(t.get(&smask, (size_t)B.nnz + 1));
    Graph S, ST, Scf, STcf;
    TRY(build_strength_graph(h, t, B, o.theta, smask, S, 1));   // abs mode: the entries are norms
    TRY(transpose(h, t, N, N, S.nnz, S.rp, S.col, nullptr, &ST.rp, &ST.col, nullptr, false));
    ST.n = N;
    ST.nnz = S.nnz;
    if (o.theta_cf != o.theta) {
        uint8_t *m2;
        TRY(t.get(&m2, (size_t)B.nnz + 1));
        TRY(build_strength_graph(h, t, B, o.theta_cf, m2, Scf, 1));
        TRY(transpose(h, t, N, N, Scf.nnz, Scf.rp, Scf.col, nullptr, &STcf.rp, &STcf.col, nullptr, false));
        STcf.n = N;
        STcf.nnz = Scf.nnz;
    } else {
        Scf = S;
        STcf = ST;
    }

    tend(h, tp);
    tp = tbegin(h, phase_name(h, "split", l), 0.0);
    int8_t *cfB;
    TRY(t.get(&cfB, (size_t)N));
    if (cf_user) {
        std::vector<int8_t> hb((size_t)N);
        for (int I = 0; I < N; ++I) hb[I] = cf_user[(size_t)I * k];
        CU(cudaMemcpyAsync(cfB, hb.data(), (size_t)N, cudaMemcpyHostToDevice, h->s));
        CU(cudaStreamSynchronize(h->s));
        normalize_cf(N, cfB, h->s);
    } else {
        TRY(split_points(h, t, l, N, Scf, STcf, std::vector<int>(), cfB));
    }
    TRY(dalloc(h, &L.strong, (size_t)A.nnz));
    TRY(dalloc(h, &L.cf, (size_t)n));
    launch_node_expand(n, k, A, B, smask, L.strong, cfB, L.cf, h->s);

    // coarse numbering of the unknowns and of the nodes
    int *flag, *scanv, *cpts;
    TRY(new_counts(h, t, &flag, n));
    launch_cidx(n, L.cf, flag, nullptr, nullptr, 0, h->s);
    TRY(t.get(&scanv, (size_t)n + 1));
    int nc = 0;
    TRY(scan(h, flag, scanv, n, &nc));
    L.nc = nc;
    if (nc == 0 || nc == n) {
        tend(h, tp);
        *last = true;
        return LAIR_OK;
    }
    TRY(dalloc(h, &L.cidx, (size_t)n));
    TRY(dalloc(h, &cpts, (size_t)nc));
    launch_cidx(n, L.cf, scanv, L.cidx, cpts, 1, h->s);
    L.crows = cpts;
    if (n - nc > 0) {
        TRY(dalloc(h, &L.frows, (size_t)(n - nc)));
        launch_frows(n, L.cf, scanv, L.frows, h->s);
    }
    const int NC = nc / k;
    int *flagB, *scanB, *cidxB, *cptsB;
    TRY(new_counts(h, t, &flagB, N));
    launch_cidx(N, cfB, flagB, nullptr, nullptr, 0, h->s);
    TRY(t.get(&scanB, (size_t)N + 1));
    TRY(scan(h, flagB, scanB, N, nullptr));
    TRY(t.get(&cidxB, (size_t)N));
    TRY(t.get(&cptsB, (size_t)NC));
    launch_cidx(N, cfB, scanB, cidxB, cptsB, 1, h->s);

    // restriction: for each unknown of a C node, the local system on every unknown of the node's
    // F-node neighbourhood (together, the block system of Sec. 3.1 for k right-hand sides)
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "R", l), 0.0);
    int *nrp, *ncol, nn = 0, *len;
    TRY(build_sets(h, t, NC, cptsB, S, cfB, &nrp, &ncol, &nn));
    TRY(new_counts(h, t, &len, nc));
    launch_node_rows(0, NC, k, nrp, ncol, cptsB, len, nullptr, nullptr, h->s);
    L.R.nr = nc;
    L.R.nc = n;
    TRY(dalloc(h, &L.R.rp, (size_t)nc + 1));
    TRY(scan(h, len, L.R.rp, nc, &L.R.nnz));
    TRY(dalloc(h, &L.R.col, (size_t)L.R.nnz));
    TRY(dalloc(h, &L.R.val, (size_t)L.R.nnz));
    if (fp32) TRY(dalloc(h, &L.R.val32, (size_t)L.R.nnz));
    launch_node_rows(1, NC, k, nrp, ncol, cptsB, nullptr, L.R.rp, L.R.col, h->s);
    TRY(dalloc(h, &L.lsR, (size_t)nc));
    TRY(local_rows_on(h, t, nc, cpts, L.R.rp, L.R.col, L.R.nnz, A.rp, A.col, A.val, L.R.col, L.R.val,
                      fp32 ? L.R.val32 : nullptr, L.lsR, -1, k));

    // interpolation
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "P", l), 0.0);
    L.P.nr = n;
    L.P.nc = nc;
    if (o.interp == LAIR_P_ONEPOINT) {
        int *choiceB, *cntB, *cnt;
        TRY(t.get(&choiceB, (size_t)N));
        TRY(new_counts(h, t, &cntB, N));
        launch_onepoint(0, B, smask, cfB, cidxB, 1, choiceB, cntB, nullptr, h->s);
        TRY(new_counts(h, t, &cnt, n));
        launch_onepoint_nodal(0, n, k, choiceB, cnt, nullptr, h->s);
        TRY(dalloc(h, &L.P.rp, (size_t)n + 1));
        TRY(scan(h, cnt, L.P.rp, n, nullptr));
        L.P.nnz = n;   // at most one entry per row; the exact count is read with the hierarchy totals
        TRY(dalloc(h, &L.P.col, (size_t)n));
        TRY(dalloc(h, &L.P.val, (size_t)n));
        if (fp32) TRY(dalloc(h, &L.P.val32, (size_t)n));
        launch_onepoint_nodal(1, n, k, choiceB, nullptr, &L.P, h->s);
    } else {
        // approximate ideal interpolation by block: the sets of the transposed node graph, the local
        // systems of A^T, transposed back
        int *qrp, *qcol, qn = 0, *wlen, *wrp, *wcol, wnnz = 0, *atrp, *atcol;
        double *wval, *atval;
        TRY(build_sets(h, t, NC, cptsB, ST, cfB, &qrp, &qcol, &qn));
        TRY(new_counts(h, t, &wlen, nc));
        launch_node_rows(0, NC, k, qrp, qcol, cptsB, wlen, nullptr, nullptr, h->s);
        TRY(t.get(&wrp, (size_t)nc + 1));
        TRY(scan(h, wlen, wrp, nc, &wnnz));
        TRY(t.get(&wcol, (size_t)wnnz));
        TRY(t.get(&wval, (size_t)wnnz));
        launch_node_rows(1, NC, k, qrp, qcol, cptsB, nullptr, wrp, wcol, h->s);
        TRY(transpose(h, t, n, n, A.nnz, A.rp, A.col, A.val, &atrp, &atcol, &atval, false));
        TRY(dalloc(h, &L.lsP, (size_t)nc));
        TRY(local_rows_on(h, t, nc, cpts, wrp, wcol, wnnz, atrp, atcol, atval, wcol, wval, nullptr, L.lsP, -1, k));
        TRY(transpose(h, t, nc, n, wnnz, wrp, wcol, wval, &L.P.rp, &L.P.col, &L.P.val, true));
        L.P.nnz = wnnz;
        if (fp32) {
            TRY(dalloc(h, &L.P.val32, (size_t)wnnz));
            launch_to_f32(wnnz, L.P.val, L.P.val32, h->s);
        }
    }

    // Galerkin product and lumping by block
    tend(h, tp);
    tp = tbegin(h, phase_name(h, "RAP", l), 0.0);
    DCsr RA, K;
    const bool lump = o.lump_tol > 0.0;
    int *klen = nullptr;
    if (o.interp == LAIR_P_ONEPOINT) {
        TRY(spgemm(h, t, L.R, A, K, !lump, l == 0 ? 1 : -1, &L.P, lump ? &klen : nullptr));
    } else {
        TRY(spgemm(h, t, L.R, A, RA, false, l == 0 ? 0 : -1));
        TRY(spgemm(h, t, RA, L.P, K, !lump, l == 0 ? 1 : -1, nullptr, lump ? &klen : nullptr));
    }
    Level next;
    if (lump) {
        int *cnt;
        TRY(new_counts(h, t, &cnt, K.nr));
        launch_lump_nodal(0, k, K, klen, o.lump_tol, cnt, nullptr, h->status, h->s);
        DCsr Kl;
        Kl.nr = Kl.nc = K.nr;
        TRY(dalloc(h, &Kl.rp, (size_t)K.nr + 1));
        TRY(scan(h, cnt, Kl.rp, K.nr, &Kl.nnz));
        TRY(dalloc(h, &Kl.col, (size_t)Kl.nnz));
        TRY(dalloc(h, &Kl.val, (size_t)Kl.nnz));
        launch_lump_nodal(1, k, K, klen, o.lump_tol, nullptr, &Kl, h->status, h->s);
        next.A = Kl;
    } else {
        next.A = K;
    }
    H.lev.push_back(next);
    tend(h, tp);
    *last = false;
    return LAIR_OK;
}

// build sliced-ELL views, all of them with a handful of launches and one synchronisation:
// views are grouped by element type (FP32, FP64); each group gets one slice-offset scan and
// one column and one value array, which its views index with group-wide offsets
struct SellPlan {
    SellView *v;
    const DCsr *M;
    const int *rows_in;   // NULL: all rows in order
    int nrows;
    const double *dinv;   // NULL: no diagonal
    bool fp32;
    const int *seg = nullptr;   // batched systems: first row of every system in the view rows' numbering
    bool zero_stopped = false;  // write 0 to the rows of stopped systems instead of skipping them
};

static lair_status build_sells(lair_handle *h, Hier &H, std::vector<SellPlan> &plans) {
    Temps t(h);
    std::vector<SellDesc> hd;
    std::vector<SellPlan *> hp;
    int win = 0, lin = 0, sl = 0;
    int gp[3] = {0, 0, 0}, glin[3] = {0, 0, 0}, gsl0[2] = {0, 0}, gsl1[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        gp[g] = (int)hd.size();
        glin[g] = lin;
        gsl0[g] = sl;
        for (auto &p : plans) {
            if (p.nrows <= 0 || (p.fp32 ? 0 : 1) != g) continue;
            SellView &v = *p.v;
            v.nrows = p.nrows;
            TRY(dalloc(h, &v.row, (size_t)p.nrows));
            const int nsl = (p.nrows + 31) / 32;
            SellDesc d{};
            d.rows_in = p.rows_in;
            d.rp = p.M->rp;
            d.col = p.M->col;
            d.val = p.M->val;
            d.dinv = p.dinv;
            d.row_out = v.row;
            d.nrows = p.nrows;
            d.win0 = win;
            d.lin0 = lin;
            d.sl0 = sl;
            d.group = g;
            if (p.seg && h->sys_run) {
                int *ss;
                TRY(dalloc(h, &ss, (size_t)nsl));
                d.seg = p.seg;
                d.nseg = h->nseg;
                d.slice_sys = ss;
                v.slice_sys = ss;
                v.run = h->sys_run;
                v.zero_stopped = p.zero_stopped;
            }
            hd.push_back(d);
            hp.push_back(&p);
            win += (p.nrows + 255) / 256;
            lin += nsl;
            sl += nsl;
        }
        gsl1[g] = sl;
        sl += 1;   // the group's end offset
    }
    gp[2] = (int)hd.size();
    glin[2] = lin;
    const int nd = (int)hd.size();
    if (nd == 0) return LAIR_OK;
    for (auto &p : plans)
        if (p.nrows <= 0) p.v->nrows = 0;

    SellDesc *dd;
    int *cnt, *sp, *tot;
    unsigned long long *gsum;
    TRY(dalloc(h, &dd, (size_t)nd));
    TRY(new_counts(h, t, &cnt, sl));
    TRY(t.get(&gsum, 2));
    TRY(t.get(&tot, 6));
    TRY(dalloc(h, &sp, (size_t)sl + 1));
    CU(cudaMemsetAsync(gsum, 0, 2 * sizeof(unsigned long long), h->s));
    CU(cudaMemcpyAsync(dd, hd.data(), sizeof(SellDesc) * nd, cudaMemcpyHostToDevice, h->s));
    launch_sell_prepare_multi(dd, nd, win, lin, cnt, gsum, h->s);
    for (int g = 0; g < 2; ++g) {
        if (gsl1[g] > gsl0[g]) TRY(scan(h, cnt + gsl0[g], sp + gsl0[g], gsl1[g] - gsl0[g], nullptr));
        CU(cudaMemcpyAsync(tot + g, sp + gsl1[g], sizeof(int), cudaMemcpyDeviceToDevice, h->s));
    }
    CU(cudaMemcpyAsync(tot + 2, gsum, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->s));
    int ht[6];
    TRY(read_ints(h, tot, 6, ht));
    unsigned long long hs[2];
    memcpy(hs, ht + 2, sizeof hs);
    for (int g = 0; g < 2; ++g) {
        if (gp[g + 1] == gp[g]) continue;
        if (hs[g] > 0x7fffffffull)
            return fail(h, LAIR_ERR_UNSUPPORTED, "sliced-ELL copies of %llu entries exceed 32-bit offsets", hs[g]);
        const size_t el = g == 0 ? sizeof(float) : sizeof(double);
        int *gcol;
        unsigned char *gval, *gdinv = nullptr;
        TRY(dalloc(h, &gcol, (size_t)ht[g]));
        TRY(dalloc(h, &gval, el * (size_t)ht[g]));
        size_t drows = 0;
        for (int q = gp[g]; q < gp[g + 1]; ++q)
            if (hd[q].dinv) drows += (size_t)hd[q].nrows;
        if (drows) TRY(dalloc(h, &gdinv, el * drows));
        size_t doff = 0;
        for (int q = gp[g]; q < gp[g + 1]; ++q) {
            SellDesc &d = hd[q];
            SellView &v = *hp[q]->v;
            d.slice_ptr = sp + d.sl0;
            d.scol = gcol;
            d.sval = gval;
            d.sdinv = d.dinv ? gdinv + el * doff : nullptr;
            if (d.dinv) doff += (size_t)d.nrows;
            v.slice_ptr = sp + d.sl0;
            v.col = gcol;
            v.val = gval;
            v.dinv = d.sdinv;
        }
    }
    CU(cudaMemcpyAsync(dd, hd.data(), sizeof(SellDesc) * nd, cudaMemcpyHostToDevice, h->s));
    // (a copy from pageable memory is staged before cudaMemcpyAsync returns, so hd may go)
    for (int g = 0; g < 2; ++g) launch_sell_fill_multi(dd, gp[g], gp[g + 1], glin[g], glin[g + 1], g == 0, h->s);
    H.sell_desc = dd;
    for (int g = 0; g < 3; ++g) {
        H.sell_gp[g] = gp[g];
        H.sell_glin[g] = glin[g];
    }
    return LAIR_OK;
}

// refill every view's values (and Jacobi diagonals) from the matrices they were built from
static void refill_sells(lair_handle *h, Hier &H) {
    if (!H.sell_desc) return;
    for (int g = 0; g < 2; ++g)
        launch_sell_fill_multi(H.sell_desc, H.sell_gp[g], H.sell_gp[g + 1], H.sell_glin[g], H.sell_glin[g + 1], g == 0,
                               h->s);
}

// the sliced-ELL views of level l (built for all levels at once when the hierarchy is complete)
static void add_view_plans(lair_handle *h, Hier &H, int l, std::vector<SellPlan> &plans) {
    Level &L = H.lev[l];
    const bool fp32 = h->o.precision == LAIR_MIXED;
    if (!L.coarsest) {
        const int n = L.A.nr, nc = L.nc;
        // the relaxation's matrix: A (point Jacobi) or D^{-1} A (block Jacobi, nodal hierarchy)
        const bool nodal = h->o.nodal > 1;
        const DCsr *Ar = nodal ? &L.Ahat : &L.A;
        const double *dv = nodal ? L.dinv_hat : L.dinv;
        const int *sc = l + 1 < (int)H.lev.size() ? H.lev[l + 1].seg_d : nullptr;
        plans.push_back(SellPlan{&L.AF, Ar, L.frows, n - nc, dv, fp32, L.seg_d});
        plans.push_back(SellPlan{&L.AC, Ar, L.crows, nc, dv, fp32, L.seg_d});
        plans.push_back(SellPlan{&L.Rv, &L.R, nullptr, L.R.nr, nullptr, fp32, sc});
        // one-point P is applied from its column array (p1col), without a view
        if (h->o.interp != LAIR_P_ONEPOINT)
            plans.push_back(SellPlan{&L.Pv, &L.P, nullptr, L.P.nr, nullptr, fp32, L.seg_d});
    }
    // the outer FP64 product writes 0 to the rows of stopped systems: their Krylov vectors, which enter the next
    // cycle's input, stay finite values of this solve
    if (l == 0) plans.push_back(SellPlan{&L.A64, &L.A, nullptr, L.A.nr, nullptr, false, L.seg_d, true});
}

static lair_status finish_level(lair_handle *h, Hier &H, int l) {
    const int tp = tbegin(h, phase_name(h, "finish", l), 0.0);
    Level &L = H.lev[l];
    const int n = L.A.nr;
    const bool fp32 = h->o.precision == LAIR_MIXED;
    TRY(dalloc(h, &L.dinv, (size_t)n));
    if (fp32) TRY(dalloc(h, &L.dinv32, (size_t)n));
    launch_dinv(L.A, L.dinv, L.dinv32, h->status, h->s);
    const bool nodal = h->o.nodal > 1 && !L.coarsest;
    if (nodal) {
        // block Jacobi: Ahat = D^{-1} A (the scaling kernels of the DG option) and its unit diagonal
        const int k = h->o.nodal, N = n / k;
        Temps t(h);
        int *rowcnt;
        TRY(new_counts(h, t, &rowcnt, n));
        launch_block_count(N, k, L.A, rowcnt, h->s);
        L.Ahat.nr = L.Ahat.nc = n;
        TRY(dalloc(h, &L.Ahat.rp, (size_t)n + 1));
        TRY(scan(h, rowcnt, L.Ahat.rp, n, &L.Ahat.nnz));
        TRY(dalloc(h, &L.Ahat.col, (size_t)L.Ahat.nnz));
        TRY(dalloc(h, &L.Ahat.val, (size_t)L.Ahat.nnz));
        TRY(dalloc(h, &L.binv, (size_t)n * k));
        launch_block_fill(N, k, L.A, L.Ahat, L.binv, h->status, h->s);
        TRY(dalloc(h, &L.dinv_hat, (size_t)n));
        if (fp32) {
            TRY(dalloc(h, &L.dinv_hat32, (size_t)n));
            TRY(dalloc(h, &L.binv32, (size_t)n * k));
            launch_to_f32((long long)n * k, L.binv, L.binv32, h->s);
            TRY(dalloc(h, &L.bh32, (size_t)n));
        } else {
            TRY(dalloc(h, &L.bh64, (size_t)n));
        }
        launch_dinv(L.Ahat, L.dinv_hat, L.dinv_hat32, h->status, h->s);
    }
    if (h->o.timing && L.cf && l == 0) {
        Temps t(h);
        unsigned long long *st;
        TRY(t.get(&st, 4));
        CU(cudaMemsetAsync(st, 0, 4 * sizeof(unsigned long long), h->s));
        cf_stats(nodal ? L.Ahat : L.A, L.cf, st, h->s);
        unsigned long long hs[4];
        CU(cudaMemcpyAsync(hs, st, sizeof hs, cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        L.nF = (long long)hs[0]; L.nnzF = (long long)hs[1]; L.nC = (long long)hs[2]; L.nnzC = (long long)hs[3];
    }
    if (fp32) {
        TRY(dalloc(h, &L.A.val32, (size_t)L.A.nnz));
        launch_to_f32(L.A.nnz, L.A.val, L.A.val32, h->s);
        TRY(dalloc(h, &L.b32, (size_t)n));
        TRY(dalloc(h, &L.x32[0], (size_t)n));
        TRY(dalloc(h, &L.x32[1], (size_t)n));
    } else {
        TRY(dalloc(h, &L.b64, (size_t)n));
        TRY(dalloc(h, &L.x64[0], (size_t)n));
        TRY(dalloc(h, &L.x64[1], (size_t)n));
    }
    tend(h, tp);
    return LAIR_OK;
}

static const int relax_seq[3][3] = {{CF_F, CF_F, CF_C}, {CF_F, CF_C, CF_F}, {CF_F, CF_F, -1}};

template <class T> struct CycleBufs;
template <> struct CycleBufs<double> {
    static double *bh(Level &L) { return L.bh64; }
    static const double *binv(Level &L) { return L.binv; }
    static double *b(Level &L) { return L.b64; }
    static double *x(Level &L, int k) { return L.x64[k]; }
    static const double *dinv(Level &L) { return L.dinv; }
};
template <> struct CycleBufs<float> {
    static float *bh(Level &L) { return L.bh32; }
    static const float *binv(Level &L) { return L.binv32; }
    static float *b(Level &L) { return L.b32; }
    static float *x(Level &L, int k) { return L.x32[k]; }
    static const float *dinv(Level &L) { return L.dinv32; }
};

// algorithmic bytes (matrix entries read once, vectors read or written once)
static double bytes_sweep(const Level &L, int target, double sv) {
    double nT = target == CF_F ? (double)L.nF : (double)L.nC, nnzT = target == CF_F ? (double)L.nnzF : (double)L.nnzC;
    return nnzT * (sv + 4.0) + nT * (4.0 + 3.0 * sv) + (double)L.A.nr * sv;
}

template <class T>
static void record_cycle(lair_handle *h, Hier &H, int l) {
    using B = CycleBufs<T>;
    const double sv = sizeof(T);
    Level &L = H.lev[l];
    const bool tm = l == 0;
    if (L.coarsest) {
        dense_apply<T>(L.A.nr, L.Ainv, B::b(L), B::x(L, 0), h->s);
        L.xfinal = 0;
        return;
    }
    if (l == H.bottom_first) {
        const int nl = (int)H.lev.size();
        Level &Z = H.lev[nl - 1];
        BottomCoarse<T> cz;
        cz.n = Z.A.nr;
        cz.Ainv = Z.Ainv;
        cz.b = B::b(Z);
        cz.x = B::x(Z, 0);
        const int *seq = relax_seq[h->o.relax];
        cycle_bottom<T>(static_cast<const BottomLevel<T> *>(H.bottom_desc), nl - 1 - l, cz, seq, h->s);
        int nsw = 0;
        while (nsw < 3 && seq[nsw] >= 0) ++nsw;
        for (int k = l; k < nl - 1; ++k) H.lev[k].xfinal = nsw & 1;
        Z.xfinal = 0;
        return;
    }
    Level &C = H.lev[l + 1];
    int t = tm ? tbegin(h, "L0_restrict", bytes_spmv(L.R, sv), true) : -1;
    sell_spmv<T>(L.Rv, B::b(L), B::b(C), h->s);
    if (tm) tend(h, t, true);
    record_cycle<T>(h, H, l + 1);
    const bool p1 = h->o.interp == LAIR_P_ONEPOINT && L.p1col;
    t = tm ? tbegin(h, "L0_interp", p1 ? bytes_p1(L.P, sv) : bytes_spmv(L.P, sv), true) : -1;
    if (p1) {
        // at most one entry per row of P, every entry 1 (one-point, or the identity blocks of the nodal one-point
        // P): the direct kernel on the dense column array, rows in their own order
        p1_interp<T>(L.P.nr, L.p1col, L.blk_sys, L.blk_sys ? h->sys_run : nullptr, B::x(C, C.xfinal), B::x(L, 0),
                     h->s);
    } else {
        sell_spmv<T>(L.Pv, B::x(C, C.xfinal), B::x(L, 0), h->s);
    }
    if (tm) tend(h, t, true);
    int cur = 0;
    const int n = L.A.nr, nc = L.nc;
    T *rb = B::b(L);
    if (h->o.nodal > 1) {
        // block Jacobi: x += D^{-1} b - (D^{-1} A) x
        block_apply_t<T>(n, h->o.nodal, B::binv(L), B::b(L), B::bh(L), h->s);
        rb = B::bh(L);
    }
    for (int k = 0; k < 3; ++k) {
        int tg = relax_seq[h->o.relax][k];
        if (tg < 0) break;
        t = tm ? tbegin(h, tg == CF_F ? "L0_sweep_F" : "L0_sweep_C", bytes_sweep(L, tg, sv), true) : -1;
        if (tg == CF_F) sell_sweep<T>(L.AF, L.crows, nc, rb, B::x(L, cur), B::x(L, 1 - cur), h->s);
        else sell_sweep<T>(L.AC, L.frows, n - nc, rb, B::x(L, cur), B::x(L, 1 - cur), h->s);
        if (tm) tend(h, t, true);
        cur ^= 1;
    }
    L.xfinal = cur;
}

// ---------------------------------------------------------------------------------------
// launch-schedule autotuner for the cycle's sliced-ELL kernels (restriction, interpolation, F and C
// sweeps): every candidate (threads per block, grid cap) is timed with CUDA events on the level's own
// buffers (best of five), a candidate replaces the default schedule only when it is more than 5 % faster,
// views of fewer than TUNE_MIN_ROWS rows keep the default (their few-microsecond timings alone did not carry
// over into the captured cycle),
// and the choice is cached for the process by view shape (kind, precision, rows in quarter octaves, mean
// row length), so later hierarchies with similar levels take it without timing. One thread owns each row
// in these kernels, so the schedule never changes a result.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int TUNE_MIN_ROWS = 65536;
struct TuneKey {
    int dev, kind, fp32, rows, len;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, kind, fp32, rows, len) < std::tie(o.dev, o.kind, o.fp32, o.rows, o.len);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int3> g_tune;
// (threads per block, grid cap in blocks per SM, rows per thread); the first is the default schedule
const int3 kTuneCandidates[] = {{256, 16, 1}, {256, 4, 1}, {256, 8, 1},  {256, 32, 1}, {128, 8, 1},
                                {128, 16, 1}, {128, 32, 1}, {128, 64, 1}, {256, 16, 2}, {256, 32, 2},
                                {128, 32, 2}, {128, 64, 2}};
}  // namespace

template <class T>
static lair_status autotune_level(lair_handle *h, Hier &H, int l, cudaEvent_t e0, cudaEvent_t e1) {
    using B = CycleBufs<T>;
    Level &L = H.lev[l];
    if (L.coarsest) return LAIR_OK;
    Level &C = H.lev[l + 1];
    const int n = L.A.nr, nc = L.nc;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    bool cleared = false;
    const double lenA = n ? (double)L.A.nnz / n : 0.0;
    struct Job { SellView *v; double len; };
    const Job jobs[4] = {{&L.Rv, L.R.nr ? (double)L.R.nnz / L.R.nr : 0.0},
                         {&L.Pv, L.P.nr ? (double)L.P.nnz / L.P.nr : 0.0}, {&L.AF, lenA}, {&L.AC, lenA}};
    auto run = [&](int kind) {
        switch (kind) {
            case 0: sell_spmv<T>(L.Rv, B::b(L), B::b(C), h->s); break;
            case 1: sell_spmv<T>(L.Pv, B::x(C, 0), B::x(L, 0), h->s); break;
            case 2: sell_sweep<T>(L.AF, L.crows, nc, B::b(L), B::x(L, 0), B::x(L, 1), h->s); break;
            default: sell_sweep<T>(L.AC, L.frows, n - nc, B::b(L), B::x(L, 0), B::x(L, 1), h->s); break;
        }
    };
    for (int kind = 0; kind < 4; ++kind) {
        SellView &v = *jobs[kind].v;
        if (v.nrows < TUNE_MIN_ROWS) continue;
        const TuneKey key{dev, kind, (int)sizeof(T), (int)std::floor(4.0 * std::log2((double)v.nrows)),
                          (int)std::lround(jobs[kind].len)};
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                v.tb = it->second.x;
                v.grid = it->second.y;
                v.rpt = it->second.z;
                continue;
            }
        }
        if (!cleared) {
            // the buffers the timing runs read: zeros, so no candidate meets stray values
            CU(cudaMemsetAsync(B::b(L), 0, sizeof(T) * (size_t)n, h->s));
            CU(cudaMemsetAsync(B::x(L, 0), 0, sizeof(T) * (size_t)n, h->s));
            CU(cudaMemsetAsync(B::b(C), 0, sizeof(T) * (size_t)C.A.nr, h->s));
            CU(cudaMemsetAsync(B::x(C, 0), 0, sizeof(T) * (size_t)C.A.nr, h->s));
            cleared = true;
        }
        float best = 3.4e38f, base = 3.4e38f;
        const int sms = device_sms();
        int3 pick = make_int3(kTuneCandidates[0].x, kTuneCandidates[0].y * sms, kTuneCandidates[0].z);
        for (const int3 &c : kTuneCandidates) {
            const int3 cand = make_int3(c.x, c.y * sms, c.z);
            v.tb = cand.x;
            v.grid = cand.y;
            v.rpt = cand.z;
            run(kind);   // warm
            float tmin = 3.4e38f;
            for (int rep = 0; rep < 5; ++rep) {
                CU(cudaEventRecord(e0, h->s));
                run(kind);
                CU(cudaEventRecord(e1, h->s));
                CU(cudaEventSynchronize(e1));
                float ms = 0.f;
                CU(cudaEventElapsedTime(&ms, e0, e1));
                tmin = std::min(tmin, ms);
            }
            if (&c == kTuneCandidates) base = tmin;   // the default schedule
            if (tmin < best) {
                best = tmin;
                pick = cand;
            }
        }
        if (!(best < 0.95f * base)) pick = make_int3(kTuneCandidates[0].x, kTuneCandidates[0].y * sms, kTuneCandidates[0].z);
        v.tb = pick.x;
        v.grid = pick.y;
        v.rpt = pick.z;
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[key] = pick;
    }
    return LAIR_OK;
}

static lair_status autotune_views(lair_handle *h, Hier &H) {
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    lair_status st = LAIR_OK;
    for (int l = 0; l < (int)H.lev.size() && st == LAIR_OK; ++l)
        st = h->o.precision == LAIR_MIXED ? autotune_level<float>(h, H, l, e0, e1)
                                          : autotune_level<double>(h, H, l, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// The smallest levels (at most BOTTOM_ROWS rows, below the finest, at least one besides the coarsest) run in the
// one-CTA bottom kernel: their descriptors in the cycle's precision, uploaded once; the views and buffers they
// point to live as long as the hierarchy (a refresh refills them in place).
template <class T>
static lair_status prepare_bottom(lair_handle *h, Hier &H) {
    using B = CycleBufs<T>;
    H.bottom_first = -1;
    const int nl = (int)H.lev.size();
    // (a coarsest level of more than 512 unknowns keeps its many-CTA dense product)
    if (h->o.nodal > 1 || nl < 3 || H.lev[nl - 1].A.nr > 512) return LAIR_OK;
    int first = -1;
    for (int l = 1; l <= nl - 2 && first < 0; ++l)
        if (H.lev[l].A.nr <= BOTTOM_ROWS) first = l;
    if (first < 0) return LAIR_OK;
    std::vector<BottomLevel<T>> d(nl - 1 - first);
    for (int i = 0; i < (int)d.size(); ++i) {
        Level &L = H.lev[first + i];
        BottomLevel<T> &t = d[i];
        t.n = L.A.nr;
        t.nc = L.nc;
        t.R = L.Rv;
        t.P = L.Pv;
        t.AF = L.AF;
        t.AC = L.AC;
        t.p1col = h->o.interp == LAIR_P_ONEPOINT ? L.p1col : nullptr;
        t.crows = L.crows;
        t.frows = L.frows;
        t.b = B::b(L);
        t.x[0] = B::x(L, 0);
        t.x[1] = B::x(L, 1);
    }
    const size_t bytes = sizeof(BottomLevel<T>) * d.size();
    char *desc = nullptr;
    TRY(dalloc(h, &desc, bytes));
    CU(cudaMemcpyAsync(desc, d.data(), bytes, cudaMemcpyHostToDevice, h->s));
    CU(cudaStreamSynchronize(h->s));
    H.bottom_desc = desc;
    H.bottom_first = first;
    return LAIR_OK;
}

static lair_status capture_cycle(lair_handle *h, Hier &H) {
    if (h->o.precision == LAIR_MIXED) TRY(prepare_bottom<float>(h, H));
    else TRY(prepare_bottom<double>(h, H));
    long long dummy = 0;
    long long *saved = g_launches;
    g_launches = &dummy;
    cudaGraph_t g;
    CU(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    h->graph_events.clear();
    int tall = tbegin(h, "vcycle", 0.0, true);
    if (h->o.precision == LAIR_MIXED) record_cycle<float>(h, H, 0);
    else record_cycle<double>(h, H, 0);
    tend(h, tall, true);
    cudaError_t e = cudaStreamEndCapture(h->s, &g);
    g_launches = saved;
    CU(e);
    CU(cudaGraphInstantiate(&H.graph, g, 0));
    size_t nn = 0;
    CU(cudaGraphGetNodes(g, nullptr, &nn));
    H.graph_nodes = (int)nn;
    CU(cudaGraphDestroy(g));
    return LAIR_OK;
}

static lair_status build_hierarchy(lair_handle *h, Hier &H, const DCsr &A0, const int8_t *cf_user) {
    auto t0 = std::chrono::steady_clock::now();
    const lair_options &o = h->o;
    H.lev.clear();
    Level L0;
    int tp = tbegin(h, "setup_level0", 0.0);
    {
        Temps t(h);
        DCsr A = A0;
        if (o.block_size > 1) {
            const int bs = o.block_size, nblk = A.nr / bs;
            int *rowcnt;
            TRY(new_counts(h, t, &rowcnt, A.nr));
            if (!launch_block_count(nblk, bs, A, rowcnt, h->s))
                return fail(h, LAIR_ERR_UNSUPPORTED, "block_size %d", bs);
            DCsr B;
            B.nr = B.nc = A.nr;
            TRY(dalloc(h, &B.rp, (size_t)A.nr + 1));
            TRY(scan(h, rowcnt, B.rp, A.nr, &B.nnz));
            TRY(dalloc(h, &B.col, (size_t)B.nnz));
            TRY(dalloc(h, &B.val, (size_t)B.nnz));
            H.bs = bs;
            TRY(dalloc(h, &H.blk_inv, (size_t)A.nr * bs));
            launch_block_fill(nblk, bs, A, B, H.blk_inv, h->status, h->s);   // block size checked above
            TRY(sync_status(h));
            A = B;
        }
        if (o.lump_level0 && o.lump_tol > 0.0) {
            int *cnt;
            double *nd;
            TRY(new_counts(h, t, &cnt, A.nr));
            TRY(t.get(&nd, 2 * (size_t)A.nr));
            if (o.nodal > 1) launch_lump_nodal(0, o.nodal, A, nullptr, o.lump_tol, cnt, nullptr, h->status, h->s);
            else launch_lump(0, A, nullptr, o.lump_tol, cnt, nd, nullptr, h->status, h->s);
            DCsr Kl;
            Kl.nr = Kl.nc = A.nr;
            TRY(dalloc(h, &Kl.rp, (size_t)A.nr + 1));
            TRY(scan(h, cnt, Kl.rp, A.nr, &Kl.nnz));
            TRY(dalloc(h, &Kl.col, (size_t)Kl.nnz));
            TRY(dalloc(h, &Kl.val, (size_t)Kl.nnz));
            if (o.nodal > 1) launch_lump_nodal(1, o.nodal, A, nullptr, o.lump_tol, nullptr, &Kl, h->status, h->s);
            else launch_lump(1, A, nullptr, o.lump_tol, cnt, nd, &Kl, h->status, h->s);
            TRY(sync_status(h));
            A = Kl;
        }
        L0.A = A;
    }
    if (!h->seg0.empty()) {
        L0.seg_h = h->seg0;
        TRY(dalloc(h, &L0.seg_d, L0.seg_h.size()));
        CU(cudaMemcpyAsync(L0.seg_d, L0.seg_h.data(), sizeof(int) * L0.seg_h.size(), cudaMemcpyHostToDevice, h->s));
        CU(cudaStreamSynchronize(h->s));
    }
    H.lev.push_back(L0);
    tend(h, tp);
    for (int l = 0;; ++l) {
        const int n = H.lev[l].A.nr;
        bool last = n <= o.coarse_max || l + 1 >= o.max_levels;
        if (!last) {
            if (o.nodal > 1) TRY(coarsen_nodal(h, H, l, l == 0 ? cf_user : nullptr, &last));
            else TRY(coarsen(h, H, l, l == 0 ? cf_user : nullptr, &last));
        }
        if (last) H.lev[l].coarsest = true;
        TRY(finish_level(h, H, l));
        if (last) {
            Level &L = H.lev[l];
            if (n > 4096)
                return fail(h, LAIR_ERR_COARSENING_STALLED, "coarsening stopped at level %d with %d unknowns", l, n);
            tp = tbegin(h, "setup_coarsest", 0.0);
            Temps t(h);
            double *D;
            int *perm;
            TRY(t.get(&D, (size_t)n * n));
            TRY(t.get(&perm, (size_t)n));
            TRY(dalloc(h, &L.Ainv, (size_t)n * n));
            launch_dense_setup(L.A, D, perm, L.Ainv, h->status, h->s);
            tend(h, tp);
            TRY(sync_status(h));
            break;
        }
    }
    {
        // least-squares rows of all levels and the exact entry counts of the one-point P,
        // with one read-back
        Temps t(h);
        const int nl = (int)H.lev.size();
        int *c2;
        TRY(new_counts(h, t, &c2, 2 + nl));
        for (int l = 0; l < nl; ++l) {
            Level &L = H.lev[l];
            if (L.coarsest) continue;
            if (L.lsR) count_flags(L.nc, L.lsR, c2, h->s);
            if (L.lsP) count_flags(L.nc, L.lsP, c2 + 1, h->s);
            if (o.interp == LAIR_P_ONEPOINT && L.P.rp)
                CU(cudaMemcpyAsync(c2 + 2 + l, L.P.rp + L.P.nr, sizeof(int), cudaMemcpyDeviceToDevice, h->s));
        }
        std::vector<int> hc(2 + nl);
        TRY(read_ints_big(h, c2, 2 + nl, hc.data()));
        H.singular_R = hc[0];
        H.singular_P = hc[1];
        for (int l = 0; l < nl; ++l)
            if (o.interp == LAIR_P_ONEPOINT && H.lev[l].P.rp && !H.lev[l].coarsest) H.lev[l].P.nnz = hc[2 + l];
        if (h->prod_nnz) {
            int pn[2];
            TRY(read_ints(h, h->prod_nnz, 2, pn));
            // algorithmic bytes: every factor read once, the product written once.
            // R A: R, A -> RA. (R A) P: RA, P -> K. Fused: R, A, P -> K.
            const Level &L0r = H.lev[0];
            const double n0 = L0r.A.nr, nc0 = L0r.nc;
            const double rd_R = 12.0 * L0r.R.nnz + 4.0 * (nc0 + 1), rd_A = 12.0 * L0r.A.nnz + 4.0 * (n0 + 1);
            const double rd_P = 12.0 * L0r.P.nnz + 4.0 * (n0 + 1);
            if (h->prod_fused) {
                h->timers[timer_slot(h, "L0_RAP", 0.0)].bytes = rd_R + rd_A + rd_P + 12.0 * pn[1];
            } else {
                h->timers[timer_slot(h, "L0_RA", 0.0)].bytes = rd_R + rd_A + 12.0 * pn[0];
                h->timers[timer_slot(h, "L0_RAP", 0.0)].bytes = 12.0 * pn[0] + 4.0 * (nc0 + 1) + rd_P + 12.0 * pn[1];
            }
        }
    }
    {
        int tv = tbegin(h, "setup_views", 0.0);
        if (h->nseg > 0 && !h->sys_run) {
            TRY(dalloc(h, &h->sys_run, (size_t)h->nseg));
            CU(cudaMemsetAsync(h->sys_run, 1, (size_t)h->nseg, h->s));
        }
        if (o.interp == LAIR_P_ONEPOINT)
            for (auto &L : H.lev) {
                if (L.coarsest || !L.P.rp) continue;
                TRY(dalloc(h, &L.p1col, (size_t)L.P.nr));
                launch_p1_cols(L.P.nr, L.P.rp, L.P.col, L.p1col, h->s);
                if (L.seg_d && h->sys_run) {
                    TRY(dalloc(h, &L.blk_sys, (size_t)(L.P.nr + 31) / 32));
                    launch_blk_sys(L.P.nr, L.seg_d, h->nseg, L.blk_sys, h->s);
                }
            }
        std::vector<SellPlan> plans;
        for (int l = 0; l < (int)H.lev.size(); ++l) add_view_plans(h, H, l, plans);
        TRY(build_sells(h, H, plans));
        tend(h, tv);
    }
    if (o.autotune) {
        tp = tbegin(h, "setup_autotune", 0.0);
        TRY(autotune_views(h, H));
        tend(h, tp);
    }
    tp = tbegin(h, "setup_graph", 0.0);
    TRY(capture_cycle(h, H));
    tend(h, tp);
    CU(cudaStreamSynchronize(h->s));
    flush_timers(h);
    H.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return LAIR_OK;
}

// ---------------------------------------------------------------------------------------
// refresh: new values on the set-up matrix's pattern (backward Euler steps I + dt S, Sec. 4.1.1,
// with a new dt or new coefficients). The splittings, neighbourhoods and the patterns of R, P and
// every coarse operator are kept, so is every allocation, view and the captured cycle graph; every
// value is recomputed in the set-up's arithmetic.
// ---------------------------------------------------------------------------------------

// local solves on kept sets: set c is row c of (rp, col) without cpts[c] (nnz entries in all); the
// solution row is written at rp[c] in the layout local_rows writes it
static lair_status local_rows_on(lair_handle *h, Temps &t, int nc, const int *cpts, const int *rp, const int *col,
                                 int nnz, const int *brp, const int *bcol, const double *bval, int *ocol, double *oval,
                                 float *oval32, uint8_t *lsflag, int neumann_deg, int rows_per) {
    if (nc <= 0) return LAIR_OK;
    int *nb_rp, *nb_col, *lists, *bcounts;
    TRY(t.get(&nb_rp, (size_t)nc + 1));
    TRY(t.get(&nb_col, (size_t)(nnz - nc) + 1));
    launch_nb_from_rows(nc, rp, col, cpts, nb_rp, nb_col, h->s);
    // with rows_per > 1 (nodal hierarchy) consecutive groups of rows share one set and one factorisation
    const int ng = nc / rows_per;
    TRY(t.get(&lists, (size_t)3 * ng + 1));
    TRY(new_counts(h, t, &bcounts, 5));
    launch_local_bin(ng, nb_rp, lists, bcounts, bcounts + 3, h->s, rows_per);
    int hc[4];
    TRY(read_ints(h, bcounts, 4, hc));
    LocalArgs a{cpts, nb_rp, nb_col, brp, bcol, bval, ocol, oval, oval32, lsflag, neumann_deg, rows_per};
    return run_local_solves(h, t, a, ng, nb_rp, rows_per, nnz - nc, lists, bcounts, hc, -1);
}

static lair_status refresh_level(lair_handle *h, Hier &H, int l) {
    Temps t(h);
    Level &L = H.lev[l];
    const DCsr &A = L.A;
    const int n = A.nr, nc = L.nc;
    const bool fp32 = h->o.precision == LAIR_MIXED;
    const int rows_per = h->o.nodal > 1 ? h->o.nodal : 1;
    TRY(local_rows_on(h, t, nc, L.crows, L.R.rp, L.R.col, L.R.nnz, A.rp, A.col, A.val, L.R.col, L.R.val,
                      fp32 ? L.R.val32 : nullptr, L.lsR,
                      h->o.restriction == LAIR_R_NEUMANN ? h->o.distance - 1 : -1, rows_per));
    if (h->o.interp != LAIR_P_ONEPOINT) {
        // lAIP: the sets are the columns of P without their C point; the local systems are those of A^T,
        // solved into W = P^T by rows and transposed back onto P's pattern
        int *ptrp, *ptcol, *atrp, *atcol, *wcol, *prp, *pcol;
        double *atval, *wval, *pval;
        TRY(transpose(h, t, n, nc, L.P.nnz, L.P.rp, L.P.col, nullptr, &ptrp, &ptcol, nullptr, false));
        TRY(transpose(h, t, n, n, A.nnz, A.rp, A.col, A.val, &atrp, &atcol, &atval, false));
        TRY(t.get(&wcol, (size_t)L.P.nnz));
        TRY(t.get(&wval, (size_t)L.P.nnz));
        TRY(local_rows_on(h, t, nc, L.crows, ptrp, ptcol, L.P.nnz, atrp, atcol, atval, wcol, wval, nullptr, L.lsP, -1,
                          rows_per));
        TRY(transpose(h, t, nc, n, L.P.nnz, ptrp, wcol, wval, &prp, &pcol, &pval, false));
        CU(cudaMemcpyAsync(L.P.val, pval, sizeof(double) * (size_t)L.P.nnz, cudaMemcpyDeviceToDevice, h->s));
        if (fp32) launch_to_f32(L.P.nnz, L.P.val, L.P.val32, h->s);
    }
    // one-point P keeps its values (all 1)
    DCsr RA, K;
    int *klen = nullptr;
    if (h->o.interp == LAIR_P_ONEPOINT) {
        TRY(spgemm(h, t, L.R, A, K, false, -1, &L.P, &klen));
    } else {
        TRY(spgemm(h, t, L.R, A, RA, false));
        TRY(spgemm(h, t, RA, L.P, K, false, -1, nullptr, &klen));
    }
    // without lumping the kept pattern is the whole product and nothing is added to the diagonal
    if (h->o.nodal > 1 && h->o.lump_tol > 0.0) launch_lump_nodal_kept(h->o.nodal, K, klen, H.lev[l + 1].A, h->status, h->s);
    else launch_lump_kept(K, klen, H.lev[l + 1].A, h->status, h->s);
    return LAIR_OK;
}

static lair_status refresh_hierarchy(lair_handle *h, Hier &H, const DCsr &Ain) {
    auto t0 = std::chrono::steady_clock::now();
    const lair_options &o = h->o;
    const bool fp32 = o.precision == LAIR_MIXED;
    int tp = tbegin(h, "refresh", 0.0);
    {
        Temps t(h);
        Level &L0 = H.lev[0];
        const bool lump0 = o.lump_level0 && o.lump_tol > 0.0;
        DCsr A = Ain;
        if (H.bs > 1) {
            const int bs = H.bs, nblk = A.nr / bs;
            DCsr B = L0.A;
            if (lump0) {
                int *rowcnt;
                TRY(new_counts(h, t, &rowcnt, A.nr));
                launch_block_count(nblk, bs, A, rowcnt, h->s);
                TRY(t.get(&B.rp, (size_t)A.nr + 1));
                TRY(scan(h, rowcnt, B.rp, A.nr, &B.nnz));
                TRY(t.get(&B.col, (size_t)B.nnz));
                TRY(t.get(&B.val, (size_t)B.nnz));
            }
            launch_block_fill(nblk, bs, A, B, H.blk_inv, h->status, h->s);
            A = B;
        }
        if (lump0 && o.nodal > 1) launch_lump_nodal_kept(o.nodal, A, nullptr, L0.A, h->status, h->s);
        else if (lump0) launch_lump_kept(A, nullptr, L0.A, h->status, h->s);
        else if (A.val != L0.A.val)
            CU(cudaMemcpyAsync(L0.A.val, A.val, sizeof(double) * (size_t)A.nnz, cudaMemcpyDeviceToDevice, h->s));
    }
    const int nl = (int)H.lev.size();
    for (int l = 0; l + 1 < nl; ++l) TRY(refresh_level(h, H, l));
    {
        Temps t(h);
        int *c2;
        TRY(new_counts(h, t, &c2, 2));
        for (int l = 0; l < nl; ++l) {
            Level &L = H.lev[l];
            launch_dinv(L.A, L.dinv, L.dinv32, h->status, h->s);
            if (fp32) launch_to_f32(L.A.nnz, L.A.val, L.A.val32, h->s);
            if (o.nodal > 1 && !L.coarsest) {
                const int k = o.nodal;
                launch_block_fill(L.A.nr / k, k, L.A, L.Ahat, L.binv, h->status, h->s);
                launch_dinv(L.Ahat, L.dinv_hat, L.dinv_hat32, h->status, h->s);
                if (fp32) launch_to_f32((long long)L.A.nr * k, L.binv, L.binv32, h->s);
            }
            if (L.coarsest) {
                const int n = L.A.nr;
                double *D;
                int *perm;
                TRY(t.get(&D, (size_t)n * n));
                TRY(t.get(&perm, (size_t)n));
                launch_dense_setup(L.A, D, perm, L.Ainv, h->status, h->s);
            } else {
                if (L.lsR) count_flags(L.nc, L.lsR, c2, h->s);
                if (L.lsP) count_flags(L.nc, L.lsP, c2 + 1, h->s);
            }
        }
        refill_sells(h, H);
        int hc[2];
        TRY(read_ints(h, c2, 2, hc));   // also checks the status word
        H.singular_R = hc[0];
        H.singular_P = hc[1];
    }
    tend(h, tp);
    CU(cudaStreamSynchronize(h->s));
    flush_timers(h);
    H.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return LAIR_OK;
}

// ---------------------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------
// input: copy and check the caller's CSR
// ---------------------------------------------------------------------------------------
__global__ void k_check_csr(int n, long long nnz, const long long *rp64, int *rp, const int *col, const double *val,
                            int *status, int need_diag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        long long b = rp64[i];
        rp[i] = (int)b;
        if ((i == 0 && b != 0) || (i == n && b != nnz)) set_status(status, LAIR_ERR_NOT_SQUARE);
        if (i == n || b < 0 || rp64[i + 1] > nnz) continue;
        long long e = rp64[i + 1];
        if (e < b) { set_status(status, LAIR_ERR_NOT_SQUARE); continue; }
        bool diag = false;
        for (long long k = b; k < e; ++k) {
            int c = col[k];
            if (c < 0 || c >= n) { set_status(status, LAIR_ERR_UNSORTED_CSR); break; }
            if (k > b && col[k - 1] == c) { set_status(status, LAIR_ERR_DUPLICATE_ENTRY); break; }
            if (k > b && col[k - 1] > c) { set_status(status, LAIR_ERR_UNSORTED_CSR); break; }
            if (c == i && val[k] != 0.0) diag = true;
        }
        if (need_diag && !diag) set_status(status, LAIR_ERR_ZERO_DIAGONAL);
    }
}

__global__ void k_plus_one(int n, const int *a, int *b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i] + 1;
}
void plus_one(int n, const int *a, int *b, cudaStream_t s) {
    k_plus_one<<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
    count_launch();
}

__global__ void k_count_flags(int n, const uint8_t *f, int *out) {
    int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += f[i] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}
void count_flags(int n, const uint8_t *f, int *out, cudaStream_t s) {
    k_count_flags<<<grid_for(n, 256), 256, 0, s>>>(n, f, out);
    count_launch();
}

__global__ void k_normalize_cf(int n, int8_t *cf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) cf[i] = cf[i] ? CF_C : CF_F;
}
void normalize_cf(int n, int8_t *cf, cudaStream_t s) {
    k_normalize_cf<<<grid_for(n, 256), 256, 0, s>>>(n, cf);
    count_launch();
}

// h_int: 64 ints, h_dbl: 64 doubles, in one recycled pinned block
static lair_status host_scratch(lair_handle *h) {
    void *blk = nullptr;
    CU(host_block_get(&blk));
    h->h_int = static_cast<int *>(blk);
    h->h_dbl = reinterpret_cast<double *>(static_cast<char *>(blk) + 512);
    return LAIR_OK;
}

static lair_status load_matrix(lair_handle *h, const lair_csr *A) {
    if (A->n <= 0 || A->nnz < A->n || A->n > 0x7fffffff || A->nnz > 0x7fffffff)
        return fail(h, LAIR_ERR_INVALID_ARG, "matrix sizes n=%lld nnz=%lld out of range", (long long)A->n,
                    (long long)A->nnz);
    if (!A->row_ptr || !A->col || !A->val) return fail(h, LAIR_ERR_INVALID_ARG, "NULL matrix array");
    const int n = (int)A->n, nnz = (int)A->nnz;
    DCsr &M = h->A_in;
    M.nr = M.nc = n;
    M.nnz = nnz;
    TRY(dalloc(h, &M.rp, (size_t)n + 1));
    TRY(dalloc(h, &M.col, (size_t)nnz));
    TRY(dalloc(h, &M.val, (size_t)nnz));
    long long *rp64;
    TRY(dalloc(h, &rp64, (size_t)n + 1, false));
    cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!A->on_device) {
        if (A->row_ptr[0] != 0 || A->row_ptr[n] != A->nnz) {
            dfree(h, rp64);
            return fail(h, LAIR_ERR_NOT_SQUARE, "row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
        }
    }
    CU(cudaMemcpyAsync(rp64, A->row_ptr, sizeof(long long) * ((size_t)n + 1), kind, h->s));
    CU(cudaMemcpyAsync(M.col, A->col, sizeof(int) * (size_t)nnz, kind, h->s));
    CU(cudaMemcpyAsync(M.val, A->val, sizeof(double) * (size_t)nnz, kind, h->s));
    k_check_csr<<<grid_for((long long)n + 1, 256), 256, 0, h->s>>>(n, (long long)nnz, rp64, M.rp, M.col, M.val, h->status,
                                                                    h->o.block_size > 1 ? 0 : 1);
    count_launch();
    dfree(h, rp64);
    TRY(sync_status(h));
    return LAIR_OK;
}

}  // namespace lair

// =======================================================================================
// C ABI
// =======================================================================================
using namespace lair;

namespace {
struct LaunchScope {
    long long *saved;
    explicit LaunchScope(lair_handle *h) : saved(g_launches) { g_launches = h ? &h->launches : nullptr; }
    ~LaunchScope() { g_launches = saved; }
};
}  // namespace

extern "C" {

const char *lair_status_string(lair_status s) {
    switch (s) {
        case LAIR_OK: return "LAIR_OK";
        case LAIR_ERR_INVALID_ARG: return "LAIR_ERR_INVALID_ARG";
        case LAIR_ERR_NOT_SQUARE: return "LAIR_ERR_NOT_SQUARE";
        case LAIR_ERR_UNSORTED_CSR: return "LAIR_ERR_UNSORTED_CSR";
        case LAIR_ERR_DUPLICATE_ENTRY: return "LAIR_ERR_DUPLICATE_ENTRY";
        case LAIR_ERR_ZERO_DIAGONAL: return "LAIR_ERR_ZERO_DIAGONAL";
        case LAIR_ERR_COARSENING_STALLED: return "LAIR_ERR_COARSENING_STALLED";
        case LAIR_ERR_NOT_CONVERGED: return "LAIR_ERR_NOT_CONVERGED";
        case LAIR_ERR_NAN: return "LAIR_ERR_NAN";
        case LAIR_ERR_OOM: return "LAIR_ERR_OOM";
        case LAIR_ERR_ARENA_OVERFLOW: return "LAIR_ERR_ARENA_OVERFLOW";
        case LAIR_ERR_DEVICE_TIMEOUT: return "LAIR_ERR_DEVICE_TIMEOUT";
        case LAIR_ERR_CUDA: return "LAIR_ERR_CUDA";
        case LAIR_ERR_UNSUPPORTED: return "LAIR_ERR_UNSUPPORTED";
    }
    return "LAIR_UNKNOWN_STATUS";
}

const char *lair_last_error(const lair_handle *h) { return h ? h->err.c_str() : "no handle"; }

int64_t lair_kernel_launches(const lair_handle *h) { return h ? h->launches : 0; }

lair_status lair_kernel_timers(const lair_handle *h, lair_kernel_timer *out, int cap, int *count) {
    if (!h || !count) return LAIR_ERR_INVALID_ARG;
    *count = (int)h->timers.size();
    for (int i = 0; i < *count && i < cap && out; ++i) {
        const auto &t = h->timers[i];
        memset(out[i].name, 0, sizeof out[i].name);
        strncpy(out[i].name, t.name.c_str(), sizeof out[i].name - 1);
        out[i].launches = t.launches;
        out[i].total_ms = t.ms;
        out[i].bytes_per_launch = t.bytes;
    }
    return LAIR_OK;
}

lair_status lair_options_default(lair_options *o) {
    if (!o) return LAIR_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->cf_mode = LAIR_CF_AUTO;
    o->distance = 1;
    o->theta = 0.25;
    o->theta_cf = 0.25;
    o->interp = LAIR_P_LAIP;
    o->relax = LAIR_RELAX_FFC;
    o->lump_tol = 1e-3;
    o->precision = LAIR_FP64;
    o->coarse_max = 128;
    o->max_levels = 25;
    o->rs_block = 4096;
    o->pmis_seed = 0x5eedULL;
    o->fgmres_restart = 30;
    o->autotune = 1;
    return LAIR_OK;
}

static lair_status check_options(lair_handle *h, const lair_options *o) {
    if (o->cf_mode < 0 || o->cf_mode > 3) return fail(h, LAIR_ERR_INVALID_ARG, "cf_mode %d", o->cf_mode);
    if (o->cf_mode == LAIR_CF_USER && !o->cf_user) return fail(h, LAIR_ERR_INVALID_ARG, "cf_user is NULL");
    if (o->distance < 1 || o->distance > 4) return fail(h, LAIR_ERR_INVALID_ARG, "distance must be 1 to 4");
    if (o->interp < 0 || o->interp > 1) return fail(h, LAIR_ERR_INVALID_ARG, "interp %d", o->interp);
    if (o->restriction < 0 || o->restriction > 1)
        return fail(h, LAIR_ERR_INVALID_ARG, "restriction %d", o->restriction);
    if (o->nodal < 0) return fail(h, LAIR_ERR_INVALID_ARG, "nodal %d", o->nodal);
    if (o->autotune < 0 || o->autotune > 1) return fail(h, LAIR_ERR_INVALID_ARG, "autotune %d", o->autotune);
    if (o->wait_polls < 0) return fail(h, LAIR_ERR_INVALID_ARG, "wait_polls %d", o->wait_polls);
    if (o->nodal > NODAL_MAX) return fail(h, LAIR_ERR_UNSUPPORTED, "nodal <= %d", NODAL_MAX);
    if (o->nodal > 1 && o->block_size > 1)
        return fail(h, LAIR_ERR_INVALID_ARG, "nodal and block_size exclude each other");
    if (o->nodal > 1 && o->restriction != LAIR_R_LAIR)
        return fail(h, LAIR_ERR_UNSUPPORTED, "the nodal hierarchy builds R by lAIR only");
    if (o->relax < 0 || o->relax > 2) return fail(h, LAIR_ERR_INVALID_ARG, "relax %d", o->relax);
    if (o->precision < 0 || o->precision > 1) return fail(h, LAIR_ERR_INVALID_ARG, "precision %d", o->precision);
    if (o->coarse_max < 1 || o->coarse_max > 4096) return fail(h, LAIR_ERR_INVALID_ARG, "coarse_max in [1, 4096]");
    if (o->max_levels < 1) return fail(h, LAIR_ERR_INVALID_ARG, "max_levels >= 1");
    if (o->rs_block < 1 || o->rs_block > RS_MAX_N) return fail(h, LAIR_ERR_INVALID_ARG, "rs_block in [1, %d]", RS_MAX_N);
    if (o->block_size > 8) return fail(h, LAIR_ERR_UNSUPPORTED, "block_size <= 8");
    if (o->fgmres_restart < 0 || o->fgmres_restart > 31) return fail(h, LAIR_ERR_INVALID_ARG, "fgmres_restart in [1, 31]");
    if (!(o->theta >= 0.0) || !(o->theta_cf >= 0.0) || !(o->lump_tol >= 0.0))
        return fail(h, LAIR_ERR_INVALID_ARG, "thresholds must be >= 0");
    return LAIR_OK;
}

lair_status lair_setup(const lair_csr *A, const lair_options *o, lair_handle **out) {
    if (!A || !out) return LAIR_ERR_INVALID_ARG;
    *out = nullptr;
    lair_handle *h = new lair_handle();
    *out = h;
    LaunchScope ls(h);
    if (o) h->o = *o;
    else lair_options_default(&h->o);
    TRY(check_options(h, &h->o));
    if (h->o.block_size > 1 && A->n % h->o.block_size)
        return fail(h, LAIR_ERR_INVALID_ARG, "n is not a multiple of block_size");
    if (h->o.nodal > 1 && A->n % h->o.nodal) return fail(h, LAIR_ERR_INVALID_ARG, "n is not a multiple of nodal");
    if (h->o.nodal > 1 && h->o.cf_mode == LAIR_CF_USER) {
        // a node's unknowns share one label: every node's k entries must agree (as C or F)
        const int k = h->o.nodal;
        for (int64_t I = 0; I < A->n / k; ++I)
            for (int u = 1; u < k; ++u)
                if ((h->o.cf_user[I * k + u] != 0) != (h->o.cf_user[I * k] != 0))
                    return fail(h, LAIR_ERR_INVALID_ARG, "cf_user: the %d entries of node %lld differ", k, (long long)I);
    }
    h->s = (cudaStream_t)h->o.stream;
    if (!h->s) {
        // a blocking stream: ordered with the legacy default stream, and capturable into graphs
        CU(cudaStreamCreate(&h->own));
        h->s = h->own;
    }
    TRY(host_scratch(h));
    TRY(dalloc(h, &h->status, 1));
    CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->s));
    TRY(load_matrix(h, A));
    const int8_t *cfu = h->o.cf_mode == LAIR_CF_USER ? h->o.cf_user : nullptr;
    TRY(build_hierarchy(h, h->H, h->A_in, cfu));
    h->o.cf_user = nullptr;   // never retained
    return LAIR_OK;
}

lair_status lair_refresh(lair_handle *h, const double *val) {
    if (!h || !val) return LAIR_ERR_INVALID_ARG;
    if (h->H.lev.empty() || !h->H.lev.back().Ainv) return fail(h, LAIR_ERR_INVALID_ARG, "no hierarchy to refresh");
    LaunchScope ls(h);
    const DCsr &A = h->A_in;
    CU(cudaMemcpyAsync(A.val, val, sizeof(double) * (size_t)A.nnz,
                       is_device_ptr(val) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
    TRY(refresh_hierarchy(h, h->H, A));
    if (h->HT) {
        Temps t(h);
        DCsr AT;
        AT.nr = AT.nc = A.nr;
        AT.nnz = A.nnz;
        TRY(transpose(h, t, A.nr, A.nr, A.nnz, A.rp, A.col, A.val, &AT.rp, &AT.col, &AT.val, false));
        TRY(refresh_hierarchy(h, *h->HT, AT));
    }
    return LAIR_OK;
}

lair_status lair_setup_batched(const lair_csr *A, int nsys, const int64_t *sys_offsets, const lair_options *o,
                               lair_handle **out) {
    if (!A || !out || nsys < 1 || !sys_offsets) return LAIR_ERR_INVALID_ARG;
    *out = nullptr;
    lair_handle *h = new lair_handle();
    *out = h;
    LaunchScope ls(h);
    if (o) h->o = *o;
    else lair_options_default(&h->o);
    TRY(check_options(h, &h->o));
    if (h->o.cf_mode == LAIR_CF_USER) return fail(h, LAIR_ERR_INVALID_ARG, "user splitting is not available for batches");
    if (h->o.block_size > 1) return fail(h, LAIR_ERR_UNSUPPORTED, "block scaling is not available for batches");
    if (h->o.nodal > 1) return fail(h, LAIR_ERR_UNSUPPORTED, "the nodal hierarchy is not available for batches");
    if (sys_offsets[0] != 0 || sys_offsets[nsys] != A->n)
        return fail(h, LAIR_ERR_INVALID_ARG, "system offsets must run from 0 to n");
    h->seg0.resize(nsys + 1);
    for (int q = 0; q <= nsys; ++q) {
        if (q > 0 && sys_offsets[q] < sys_offsets[q - 1]) return fail(h, LAIR_ERR_INVALID_ARG, "offsets must not decrease");
        h->seg0[q] = (int)sys_offsets[q];
    }
    h->nseg = nsys;
    h->s = (cudaStream_t)h->o.stream;
    if (!h->s) {
        CU(cudaStreamCreate(&h->own));
        h->s = h->own;
    }
    TRY(host_scratch(h));
    CU(cudaMallocHost(&h->h_seg, sizeof(double) * nsys));
    CU(cudaMallocHost(&h->h_act, nsys));
    TRY(dalloc(h, &h->status, 1));
    CU(cudaMemsetAsync(h->status, 0, sizeof(int), h->s));
    TRY(load_matrix(h, A));
    TRY(build_hierarchy(h, h->H, h->A_in, nullptr));
    return LAIR_OK;
}

lair_status lair_solve_batched(lair_handle *h, const double *b, double *x, double tol, int cycle, int max_iter,
                               int *iters, double *rel) {
    if (!h || !b || !x || !(tol >= 0.0) || max_iter < 0 || cycle < 0 || cycle > 1) return LAIR_ERR_INVALID_ARG;
    if (h->nseg < 1 || h->H.lev.empty()) return fail(h, LAIR_ERR_INVALID_ARG, "handle was not set up with lair_setup_batched");
    LaunchScope ls(h);
    const int n = h->H.lev[0].A.nr;
    TRY(ensure_work(h, n, 0));
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    CU(cudaMemcpyAsync(h->wb, b, sizeof(double) * n, bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
    CU(cudaMemcpyAsync(h->wx, x, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
    lair_status st = cycle == LAIR_CYCLE_FGMRES ? solve_batched_fgmres(h, h->H, h->wb, h->wx, tol, max_iter, iters, rel)
                                                : solve_batched_dev(h, h->H, h->wb, h->wx, tol, max_iter, iters, rel);
    if (st != LAIR_OK && st != LAIR_ERR_NOT_CONVERGED) return st;
    CU(cudaMemcpyAsync(x, h->wx, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    return st;
}

lair_status lair_batch_setup_solve(int nsys, const lair_csr *A, const double *const *b, double *const *x,
                                   const lair_options *o, double tol, int cycle, int max_iter, int *iters, double *rel) {
    if (nsys < 1 || !A || !b || !x) return LAIR_ERR_INVALID_ARG;
    // concatenate on the host (the systems may live on the host or on the device)
    std::vector<int64_t> off(nsys + 1, 0), noff(nsys + 1, 0);
    for (int q = 0; q < nsys; ++q) {
        if (A[q].n < 1 || A[q].nnz < 0 || !A[q].row_ptr || !A[q].col || !A[q].val || !b[q] || !x[q])
            return LAIR_ERR_INVALID_ARG;
        off[q + 1] = off[q] + A[q].n;
        noff[q + 1] = noff[q] + A[q].nnz;
    }
    if (off[nsys] > 0x7fffffff || noff[nsys] > 0x7fffffff) return LAIR_ERR_UNSUPPORTED;
    const int64_t n = off[nsys], nnz = noff[nsys];
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> col(nnz);
    std::vector<double> val(nnz), bb(n), xx(n);
    for (int q = 0; q < nsys; ++q) {
        const int64_t nq = A[q].n, zq = A[q].nnz;
        std::vector<int64_t> rq(nq + 1);
        cudaMemcpyKind k = A[q].on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        if (cudaMemcpy(rq.data(), A[q].row_ptr, sizeof(int64_t) * (nq + 1), k) != cudaSuccess ||
            cudaMemcpy(col.data() + noff[q], A[q].col, sizeof(int32_t) * zq, k) != cudaSuccess ||
            cudaMemcpy(val.data() + noff[q], A[q].val, sizeof(double) * zq, k) != cudaSuccess ||
            cudaMemcpy(bb.data() + off[q], b[q], sizeof(double) * nq, cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(xx.data() + off[q], x[q], sizeof(double) * nq, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return LAIR_ERR_CUDA;
        }
        if (rq[0] != 0 || rq[nq] != zq) return LAIR_ERR_NOT_SQUARE;
        for (int64_t i = 0; i <= nq; ++i) rp[off[q] + i] = rq[i] + noff[q];
        for (int64_t k2 = noff[q]; k2 < noff[q + 1]; ++k2) col[k2] += (int32_t)off[q];
    }
    lair_csr M{n, nnz, rp.data(), col.data(), val.data(), 0};
    lair_handle *h = nullptr;
    lair_status st = lair_setup_batched(&M, nsys, off.data(), o, &h);
    if (st == LAIR_OK) st = lair_solve_batched(h, bb.data(), xx.data(), tol, cycle, max_iter, iters, rel);
    if (st == LAIR_OK || st == LAIR_ERR_NOT_CONVERGED)
        for (int q = 0; q < nsys; ++q)
            if (cudaMemcpy(x[q], xx.data() + off[q], sizeof(double) * A[q].n, cudaMemcpyDefault) != cudaSuccess) {
                cudaGetLastError();
                st = LAIR_ERR_CUDA;
                break;
            }
    lair_free(h);
    return st;
}

lair_status lair_solve(lair_handle *h, const double *b, double *x, double tol, int cycle, int max_iter,
                       lair_report *rep) {
    if (!h || !b || !x || !(tol >= 0.0) || max_iter < 0 || cycle < 0 || cycle > 1) return LAIR_ERR_INVALID_ARG;
    if (h->H.lev.empty()) return fail(h, LAIR_ERR_INVALID_ARG, "handle has no hierarchy");
    LaunchScope ls(h);
    return run_solve(h, h->H, b, x, tol, cycle, max_iter, rep, true);
}

lair_status lair_precond_apply(lair_handle *h, const double *b, double *x) {
    if (!h || !b || !x) return LAIR_ERR_INVALID_ARG;
    if (h->H.lev.empty()) return fail(h, LAIR_ERR_INVALID_ARG, "handle has no hierarchy");
    LaunchScope ls(h);
    const int n = h->H.lev[0].A.nr;
    TRY(ensure_work(h, n, 0));
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    CU(cudaMemcpyAsync(h->wb, b, sizeof(double) * n, bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
    TRY(precond(h, h->H, h->wb, h->wx));
    CU(cudaMemcpyAsync(x, h->wx, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    return LAIR_OK;
}

lair_status lair_adjoint(lair_handle *h, const double *g, double *lambda, double tol, int cycle, int max_iter,
                         lair_report *rep) {
    if (!h || !g || !lambda || !(tol >= 0.0) || max_iter < 0 || cycle < 0 || cycle > 1) return LAIR_ERR_INVALID_ARG;
    if (h->o.block_size > 1) return fail(h, LAIR_ERR_UNSUPPORTED, "adjoint with block scaling is not supported");
    LaunchScope ls(h);
    if (!h->HT) {
        h->HT = new Hier();
        Temps t(h);
        DCsr AT;
        AT.nr = AT.nc = h->A_in.nr;
        AT.nnz = h->A_in.nnz;
        TRY(transpose(h, t, AT.nr, AT.nc, AT.nnz, h->A_in.rp, h->A_in.col, h->A_in.val, &AT.rp, &AT.col, &AT.val, true));
        lair_options save = h->o;
        if (h->o.cf_mode == LAIR_CF_USER) h->o.cf_mode = LAIR_CF_AUTO;
        lair_status st = build_hierarchy(h, *h->HT, AT, nullptr);
        h->o = save;
        if (st != LAIR_OK) {
            delete h->HT;
            h->HT = nullptr;
            return st;
        }
    }
    return run_solve(h, *h->HT, g, lambda, tol, cycle, max_iter, rep, false);
}

lair_status lair_grad_A(lair_handle *h, const double *lambda, const double *x, double *grad) {
    if (!h || !lambda || !x || !grad) return LAIR_ERR_INVALID_ARG;
    LaunchScope ls(h);
    const DCsr &A = h->A_in;
    const bool dev = is_device_ptr(grad);
    if (dev) {
        grad_A(A, lambda, x, grad, h->s);
    } else {
        TRY(ensure_work(h, A.nr, 0));
        double *g;
        TRY(dalloc(h, &g, (size_t)A.nnz, false));
        CU(cudaMemcpyAsync(h->wb, lambda, sizeof(double) * A.nr, cudaMemcpyHostToDevice, h->s));
        CU(cudaMemcpyAsync(h->wx, x, sizeof(double) * A.nr, cudaMemcpyHostToDevice, h->s));
        grad_A(A, h->wb, h->wx, g, h->s);
        CU(cudaMemcpyAsync(grad, g, sizeof(double) * A.nnz, cudaMemcpyDeviceToHost, h->s));
        dfree(h, g);
    }
    CU(cudaStreamSynchronize(h->s));
    return LAIR_OK;
}

lair_status lair_hierarchy_info(const lair_handle *h, lair_level_info *out, int max_levels, int *nlevels) {
    if (!h || !nlevels) return LAIR_ERR_INVALID_ARG;
    *nlevels = (int)h->H.lev.size();
    for (int l = 0; l < *nlevels && l < max_levels && out; ++l) {
        const Level &L = h->H.lev[l];
        out[l].n = L.A.nr;
        out[l].nnz = L.A.nnz;
        out[l].nc = L.coarsest ? 0 : L.nc;
        out[l].nnz_R = L.coarsest ? 0 : L.R.nnz;
        out[l].nnz_P = L.coarsest ? 0 : L.P.nnz;
        out[l].is_coarsest = L.coarsest ? 1 : 0;
    }
    return LAIR_OK;
}

lair_status lair_export_csr(const lair_handle *hc, int level, int which, int64_t *row_ptr, int32_t *col, double *val) {
    lair_handle *h = const_cast<lair_handle *>(hc);
    if (!h || level < 0 || level >= (int)h->H.lev.size() || which < 0 || which > 2) return LAIR_ERR_INVALID_ARG;
    const Level &L = h->H.lev[level];
    const DCsr &M = which == 0 ? L.A : (which == 1 ? L.R : L.P);
    if (which > 0 && L.coarsest) return fail(h, LAIR_ERR_INVALID_ARG, "coarsest level has no transfer operators");
    if (row_ptr) {
        std::vector<int> rp(M.nr + 1);
        CU(cudaMemcpyAsync(rp.data(), M.rp, sizeof(int) * (M.nr + 1), cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        for (int i = 0; i <= M.nr; ++i) row_ptr[i] = rp[i];
    }
    if (col) CU(cudaMemcpyAsync(col, M.col, sizeof(int) * M.nnz, cudaMemcpyDeviceToHost, h->s));
    if (val) CU(cudaMemcpyAsync(val, M.val, sizeof(double) * M.nnz, cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    return LAIR_OK;
}

lair_status lair_export_cf(const lair_handle *hc, int level, int8_t *cf, uint8_t *strong, uint8_t *ls_R, uint8_t *ls_P) {
    lair_handle *h = const_cast<lair_handle *>(hc);
    if (!h || level < 0 || level >= (int)h->H.lev.size()) return LAIR_ERR_INVALID_ARG;
    const Level &L = h->H.lev[level];
    if (L.coarsest) return fail(h, LAIR_ERR_INVALID_ARG, "coarsest level has no splitting");
    if (cf) CU(cudaMemcpyAsync(cf, L.cf, L.A.nr, cudaMemcpyDeviceToHost, h->s));
    if (strong) CU(cudaMemcpyAsync(strong, L.strong, L.A.nnz, cudaMemcpyDeviceToHost, h->s));
    if (ls_R && L.lsR) CU(cudaMemcpyAsync(ls_R, L.lsR, L.nc, cudaMemcpyDeviceToHost, h->s));
    if (ls_P && L.lsP) CU(cudaMemcpyAsync(ls_P, L.lsP, L.nc, cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    return LAIR_OK;
}

void lair_free(lair_handle *h) {
    if (!h) return;
    if (h->H.graph) cudaGraphExecDestroy(h->H.graph);
    if (h->HT) {
        if (h->HT->graph) cudaGraphExecDestroy(h->HT->graph);
        delete h->HT;
    }
    for (void *p : h->allocs) cudaFreeAsync(p, h->s);
    if (h->scan_tmp) cudaFreeAsync(h->scan_tmp, h->s);
    cudaStreamSynchronize(h->s);
    for (auto &p : h->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto &p : h->graph_events) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    if (h->own) cudaStreamDestroy(h->own);
    if (h->h_bat) cudaFreeHost(h->h_bat);
    if (h->h_ring) cudaFreeHost(h->h_ring);
    for (cudaEvent_t e : h->ring_ev)
        if (e) cudaEventDestroy(e);
    if (h->h_batcnt) cudaFreeHost(h->h_batcnt);
    if (h->h_seg) cudaFreeHost(h->h_seg);
    if (h->h_act) cudaFreeHost(h->h_act);
    host_block_put(h->h_int);   // h_dbl lives in the same block
    cudaGetLastError();
    delete h;
}

}  // extern "C"
