// setup_graph.cu -- strength of connection, strength graphs, C/F splitting,
// coarse numbering and restriction neighbourhoods (the integer part of the
// lAIR set-up, Sec. 3.1 and Sec. 4).
#include <cooperative_groups.h>

#include "setup_kernels.cuh"

namespace lair {

// -------------------------------------------------------------------------------------
// Strength of connection (Sec. 4): j in N_i iff j != i and
//   -a_ij >= theta * m_i (signed) or |a_ij| >= theta * m_i (abs), m_i = max_{k!=i} |a_ik|.
// m_i = 0 gives no strong connections; a stored zero is never strong. theta*m_i is one
// rounded multiply. One thread per row (rows are short on every level we build).
// -------------------------------------------------------------------------------------
__global__ void k_strength(int n, const int *__restrict__ rp, const int *__restrict__ col,
                           const double *__restrict__ val, double theta, int absmode,
                           uint8_t *__restrict__ mask, int *__restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int b = rp[i], e = rp[i + 1];
        double m = 0.0;
        for (int k = b; k < e; ++k)
            if (col[k] != i && fabs(val[k]) > m) m = fabs(val[k]);
        double thr = __dmul_rn(theta, m);
        int c = 0;
        for (int k = b; k < e; ++k) {
            double a = val[k];
            int s = 0;
            if (col[k] != i && m > 0.0 && a != 0.0) s = absmode ? (fabs(a) >= thr) : (-a >= thr);
            mask[k] = (uint8_t)s;
            c += s;
        }
        cnt[i] = c;
    }
}

__global__ void k_graph_fill(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const uint8_t *__restrict__ mask, const int *__restrict__ grp,
                             int *__restrict__ gcol) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int p = grp[i];
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (mask[k]) gcol[p++] = col[k];
    }
}

// -------------------------------------------------------------------------------------
// Transposes (pattern, or pattern + values): count, scan, scatter with atomic cursors,
// then an insertion sort per output row so that the result is deterministic.
// -------------------------------------------------------------------------------------
__global__ void k_col_count(int nr, const int *__restrict__ rp, const int *__restrict__ col, int *__restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(&cnt[col[k]], 1);
}

__global__ void k_transpose_scatter(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                                    const double *__restrict__ val, const int *__restrict__ trp,
                                    int *__restrict__ cursor, int *__restrict__ tcol, double *__restrict__ tval) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            int j = col[k];
            int d = trp[j] + atomicAdd(&cursor[j], 1);
            tcol[d] = i;
            if (val) tval[d] = val[k];
        }
}

// Row sort after a transpose, by row length: up to SORT_REG entries in one thread's registers;
// up to SORT_WARP by a warp (32 R entries in registers, R = 1, 2, 4 or 8, bitonic network with
// shuffles across lanes and register exchanges within a lane); up to SORT_CTA by a CTA in
// shared memory (bitonic); longer rows by insertion. The columns of a row are distinct. The
// short-row pass appends the other rows to two lists (counts in lists[0], lists[1]) with one
// atomic per warp and list.
constexpr int SORT_REG = 8;
constexpr int SORT_WARP = 256;
constexpr int SORT_CTA = 4096;
constexpr int SORT_CTA_THREADS = 256;

__device__ void insertion_sort_row(int b, int e, int *col, double *val) {
    for (int k = b + 1; k < e; ++k) {
        const int c = col[k];
        const double v = val ? val[k] : 0.0;
        int m = k - 1;
        while (m >= b && col[m] > c) {
            col[m + 1] = col[m];
            if (val) val[m + 1] = val[m];
            --m;
        }
        col[m + 1] = c;
        if (val) val[m + 1] = v;
    }
}

// appends row i to list l (0 or 1) if want; all active lanes call it together
__device__ __forceinline__ void list_append(int *lists, int nr, int l, bool want, int i) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, want);
    if (!m) return;
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    int base = 0;
    if (lane == lead) base = atomicAdd(&lists[l], __popc(m));
    base = __shfl_sync(act, base, lead);
    if (want) lists[2 + l * nr + base + __popc(m & ((1u << lane) - 1u))] = i;
}

// lists: [0] warp-list count, [1] CTA-list count, then nr entries of each list
__global__ void k_sort_rows(int nr, const int *__restrict__ rp, int *__restrict__ col, double *__restrict__ val,
                            int *__restrict__ lists) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const int b = rp[i], e = rp[i + 1];
        const int len = e - b;
        list_append(lists, nr, 0, len > SORT_REG && len <= SORT_WARP, i);
        list_append(lists, nr, 1, len > SORT_WARP && len <= SORT_CTA, i);
        if (len > SORT_CTA) insertion_sort_row(b, e, col, val);
        if (len > SORT_REG) continue;
        int c[SORT_REG];
        double v[SORT_REG];
#pragma unroll
        for (int k = 0; k < SORT_REG; ++k) {
            c[k] = k < len ? col[b + k] : 0x7fffffff;
            v[k] = (k < len && val) ? val[b + k] : 0.0;
        }
        // odd-even transposition network
#pragma unroll
        for (int pass = 0; pass < SORT_REG; ++pass)
#pragma unroll
            for (int k = pass & 1; k + 1 < SORT_REG; k += 2)
                if (c[k] > c[k + 1]) {
                    int tc = c[k]; c[k] = c[k + 1]; c[k + 1] = tc;
                    double tv = v[k]; v[k] = v[k + 1]; v[k + 1] = tv;
                }
#pragma unroll
        for (int k = 0; k < SORT_REG; ++k)
            if (k < len) {
                col[b + k] = c[k];
                if (val) val[b + k] = v[k];
            }
    }
}

// one row of at most 32 R entries sorted by a warp
template <int R>
__device__ __forceinline__ void warp_sort_row(int b, int len, int *col, double *val, int lane) {
    int key[R];
    double v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = 32 * r + lane;
        key[r] = e < len ? col[b + e] : 0x7fffffff;
        v[r] = (e < len && val) ? val[b + e] : 0.0;
    }
    warp_bitonic<R>(key, v, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = 32 * r + lane;
        if (e < len) {
            col[b + e] = key[r];
            if (val) val[b + e] = v[r];
        }
    }
}

// one warp per row of the warp list
__global__ void k_sort_rows_warp(int nr, const int *__restrict__ rp, int *__restrict__ col, double *__restrict__ val,
                                 const int *__restrict__ lists) {
    const int lane = threadIdx.x & 31;
    const int cnt = lists[0];
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < cnt; t += (gridDim.x * blockDim.x) >> 5) {
        const int i = lists[2 + t];
        const int b = rp[i], len = rp[i + 1] - b;
        if (len <= 32) warp_sort_row<1>(b, len, col, val, lane);
        else if (len <= 64) warp_sort_row<2>(b, len, col, val, lane);
        else if (len <= 128) warp_sort_row<4>(b, len, col, val, lane);
        else warp_sort_row<8>(b, len, col, val, lane);
    }
}

// one CTA per row of the CTA list: bitonic sort in shared memory
__global__ void __launch_bounds__(SORT_CTA_THREADS) k_sort_rows_cta(int nr, const int *__restrict__ rp,
                                                                     int *__restrict__ col, double *__restrict__ val,
                                                                     const int *__restrict__ lists) {
    __shared__ int sk[SORT_CTA];
    __shared__ double sv[SORT_CTA];
    const int cnt = lists[1];
    for (int t = blockIdx.x; t < cnt; t += gridDim.x) {
        const int i = lists[2 + nr + t];
        const int b = rp[i], len = rp[i + 1] - b;
        int P = 2 * SORT_WARP;
        while (P < len) P <<= 1;
        for (int q = threadIdx.x; q < P; q += blockDim.x) {
            sk[q] = q < len ? col[b + q] : 0x7fffffff;
            sv[q] = (q < len && val) ? val[b + q] : 0.0;
        }
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = threadIdx.x; q < P; q += blockDim.x) {
                    const int o = q ^ j;
                    if (o > q) {
                        const bool up = (q & k) == 0;
                        if (up ? sk[q] > sk[o] : sk[q] < sk[o]) {
                            const int tk = sk[q]; sk[q] = sk[o]; sk[o] = tk;
                            const double tv = sv[q]; sv[q] = sv[o]; sv[o] = tv;
                        }
                    }
                }
                __syncthreads();
            }
        for (int q = threadIdx.x; q < len; q += blockDim.x) {
            col[b + q] = sk[q];
            if (val) val[b + q] = sv[q];
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------------------------
// PMIS: w_i = |ST_i| + u_i with u_i = (splitmix64((seed << 32) ^ i) >> 11) * 2^-53
// (splitmix64 is Vigna's published mixer). |ST_i| = 0 -> F. Rounds: every undecided i
// whose (w_i, -i) beats every undecided neighbour in S_i u ST_i becomes C; then the
// undecided points of ST_i of each new C point i become F.
// -------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_pmis_init(int n, const int *__restrict__ st_rp, uint64_t seed, double *__restrict__ w,
                            int8_t *__restrict__ cf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lam = st_rp[i + 1] - st_rp[i];
        double u = __dmul_rn(__ull2double_rn(splitmix64((seed << 32) ^ (uint64_t)i) >> 11), 0x1.0p-53);
        w[i] = lam == 0 ? -1.0 : __dadd_rn((double)lam, u);    // -1: decided
        cf[i] = lam == 0 ? CF_F : CF_U;
    }
}

__device__ __forceinline__ bool beats(double wi, int i, double wj, int j) {
    return (wi > wj) || (wi == wj && i < j);
}

// -------------------------------------------------------------------------------------
// PMIS rounds. A round: every undecided point whose weight beats those of all undecided points
// in S_i and ST_i is selected; stop when no point was undecided; selected points become C and
// their undecided dependants (ST_i) F. A decided point's weight is set to -1, so the select
// pass reads one array per neighbour. All rounds of a level run in one launch: one thread-block
// cluster for small levels (k_pmis_cluster), a cooperative grid above (k_pmis_coop), whose
// grid-barrier waits are bounded by `limit` polls; a wait that gives up sets
// LAIR_ERR_DEVICE_TIMEOUT and the block returns (so do the others at their next barrier).
// -------------------------------------------------------------------------------------
// true if w_i beats the weight of every undecided j among col[b..e) (decided points carry
// weight -1); the neighbours are read four at a time so that their loads overlap
// (L2: the weights are read from L2, past this SM's L1, as other CTAs update them between rounds)
template <bool L2 = false>
__device__ __forceinline__ bool pmis_beats_all(double wi, int i, int b, int e, const int *__restrict__ col,
                                               const double *w) {
    for (int p = b; p < e; p += 4) {
        int j[4];
        double wj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = p + u < e ? col[p + u] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) wj[u] = j[u] >= 0 ? (L2 ? __ldcg(w + j[u]) : w[j[u]]) : -1.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (wj[u] >= 0.0 && !beats(wi, i, wj[u], j[u])) return false;
    }
    return true;
}

constexpr int PMIS_THREADS = 1024;   // few large CTAs keep the grid barrier short
constexpr int PMIS_CLUSTER = 8;      // levels of at most 8 * 1024 points: one cluster, one point per thread

// The PMIS rounds of a small level in one thread-block cluster: the same rounds as k_pmis_coop,
// with the hardware cluster barrier between the passes. Counts of undecided points are summed
// through distributed shared memory; weights and markers written by other CTAs are read from L2.
__global__ void __launch_bounds__(PMIS_THREADS) k_pmis_cluster(int n, Graph S, Graph ST, double *w,
                                                      int8_t *__restrict__ cf, int8_t *__restrict__ newc) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ int cnt_sh;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned ncta = cluster.num_blocks();
    for (int round = 0; round <= n; ++round) {
        int und = 0;
        int8_t nc = 0;
        if (i < n) {
            const double wi = __ldcg(w + i);
            if (wi >= 0.0) {
                und = 1;
                nc = pmis_beats_all<true>(wi, i, S.rp[i], S.rp[i + 1], S.col, w) &&
                     pmis_beats_all<true>(wi, i, ST.rp[i], ST.rp[i + 1], ST.col, w);
            }
        }
        und = __syncthreads_count(und);
        if (threadIdx.x == 0) cnt_sh = und;
        cluster.sync();
        int total = 0;
        for (unsigned r = 0; r < ncta; ++r) total += *cluster.map_shared_rank(&cnt_sh, r);
        if (total == 0) break;
        if (nc) {
            cf[i] = CF_C;
            w[i] = -1.0;
            for (int p = ST.rp[i]; p < ST.rp[i + 1]; ++p) {
                const int j = ST.col[p];
                if (__ldcg(cf + j) == CF_U) {
                    cf[j] = CF_F;
                    w[j] = -1.0;
                }
            }
        }
        __threadfence();
        cluster.sync();
    }
    cluster.sync();   // no CTA leaves while another may still read its counter
}

// true if w_i beats the weight of every undecided neighbour in S_i and in ST_i: the two rows are read side by
// side, two entries of each at a time, so that a point waits on one chain of loads instead of two
__device__ __forceinline__ bool pmis_beats_both(double wi, int i, const Graph &S, const Graph &ST, const double *w) {
    const int sb = S.rp[i], se = S.rp[i + 1], tb = ST.rp[i], te = ST.rp[i + 1];
    for (int k = 0; sb + k < se || tb + k < te; k += 2) {
        int j[4];
        double wj[4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            j[u] = sb + k + u < se ? S.col[sb + k + u] : -1;
            j[2 + u] = tb + k + u < te ? ST.col[tb + k + u] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) wj[u] = j[u] >= 0 ? w[j[u]] : -1.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (wj[u] >= 0.0 && !beats(wi, i, wj[u], j[u])) return false;
    }
    return true;
}

// All PMIS rounds of a level in one cooperative launch, one thread per candidate point. The candidates of
// round 0 are all points; every select pass appends the points it finds undecided to a list (warp-aggregated
// atomics, two lists used in turn), and that list is the next round's candidates and this round's marking
// set, so rounds after the first few touch only the points still undecided. The order of a list varies from
// run to run; the sets do not: the selection is a function of the weights alone, and two selected points never
// lie in each other's ST (they would beat each other), so marking C and F in one pass is race-free.
// ctl[0] the grid barrier's arrival counter, ctl[2 + r % 2] the length of round r's list (all zero on entry);
// lists: 2 n ints.
__global__ void __launch_bounds__(PMIS_THREADS, 2) k_pmis_coop(int n, Graph S, Graph ST, double *w,
                                                   int8_t *__restrict__ cf, int8_t *__restrict__ newc, int *lists,
                                                   int *ctl, int *status, long long limit) {
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned *bar = reinterpret_cast<unsigned *>(ctl);
    unsigned passed = 0;
    int m_in = n;
    for (int round = 0; round <= n; ++round) {
        const int *in = round == 0 ? nullptr : lists + (size_t)((round - 1) & 1) * n;
        int *out = lists + (size_t)(round & 1) * n;
        int *cnt = ctl + 2 + (round & 1);
        for (int base = t0 - lane; base < m_in; base += stride) {
            const int idx = base + lane;
            int i = 0;
            double wi = -1.0;
            if (idx < m_in) {
                i = in ? in[idx] : idx;
                wi = w[i];
            }
            const bool und = wi >= 0.0;
            const unsigned bal = __ballot_sync(0xffffffffu, und);
            if (!bal) continue;
            const int leader = __ffs(bal) - 1;
            int pos = 0;
            if (lane == leader) pos = atomicAdd(cnt, __popc(bal));
            pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(bal & ((1u << lane) - 1u));
            if (und) {
                out[pos] = i;
                newc[i] = pmis_beats_both(wi, i, S, ST, w);
            }
        }
        if (!grid_barrier(bar, status, limit, passed)) return;
        const int m = *(volatile int *)cnt;
        if (m == 0) return;
        if (t0 == 0) ctl[2 + ((round + 1) & 1)] = 0;   // read by everyone a round ago, appended to next round
        for (int idx = t0; idx < m; idx += stride) {
            const int i = out[idx];
            if (!newc[i]) continue;
            cf[i] = CF_C;
            w[i] = -1.0;
            for (int p = ST.rp[i]; p < ST.rp[i + 1]; ++p) {
                const int j = ST.col[p];
                if (cf[j] == CF_U) {
                    cf[j] = CF_F;
                    w[j] = -1.0;
                }
            }
        }
        if (!grid_barrier(bar, status, limit, passed)) return;
        m_in = m;
    }
}

// -------------------------------------------------------------------------------------
// Classical first pass (Sec. 4, no second pass), run independently on index blocks
// [b0, b0 + B) of the level, one warp per block, everything of a block in shared memory.
// Inside a block, lambda_i = |ST_i n block|; points without any strong connection in
// the whole graph start as F. Each step takes the undecided point with the largest
// lambda (ties: smallest index) as C; its undecided in-block dependants (ST_i) become F;
// each undecided in-block k in S_j of a new F point j gets lambda += 1; each undecided
// in-block k in S_i gets lambda -= 1. With one block covering the level this is exactly
// the classical first pass.
// Keys pack (lambda + 1) << 16 | (0xFFFF - local index) (0 = decided), so the largest key
// is the point to take. A 32-ary max tree (leaves, level 1 = max of 32 leaves, level 2 =
// max of 32 level-1 nodes, at most 32 of them) finds it in three warp reductions.
// -------------------------------------------------------------------------------------
constexpr int8_t CF_NEWF = 2;   // F point created in the current step
constexpr int RS_SMEM_MAX = 200 * 1024;

__device__ __forceinline__ unsigned warp_max_u32(unsigned v) { return __reduce_max_sync(0xffffffffu, v); }

__device__ void rs_rebuild(int n, int n1, const unsigned *key, unsigned *l1, unsigned *l2, unsigned lane) {
    for (int g = lane; g < n1; g += 32) {
        unsigned m = 0;
        for (int t = 0; t < 32 && 32 * g + t < n; ++t) m = max(m, key[32 * g + t]);
        l1[g] = m;
    }
    __syncwarp();
    {
        unsigned m = 0;
        for (int t = 0; t < 32 && 32 * (int)lane + t < n1; ++t) m = max(m, l1[32 * lane + t]);
        l2[lane] = m;
    }
    __syncwarp();
}

// in-block view of a strength graph: rows and neighbours as local indices 0..n-1
struct StagedView {         // copied to shared memory, out-of-block entries removed
    const uint16_t *rp;       // row offsets (the staged area holds fewer than 65536 entries per graph)
    const uint16_t *col;
    __device__ int beg(int li) const { return rp[li]; }
    __device__ int end(int li) const { return rp[li + 1]; }
    __device__ int at(int p) const { return col[p]; }    // always in the block
};
struct GlobalView {         // read from global memory, out-of-block entries reported as -1
    const int *rp, *col;
    int b0, b1;
    __device__ int beg(int li) const { return rp[b0 + li]; }
    __device__ int end(int li) const { return rp[b0 + li + 1]; }
    __device__ int at(int p) const { int j = col[p]; return (j >= b0 && j < b1) ? j - b0 : -1; }
};

// marks the level-1 node of leaf k as changed: bit (k / 32) % 32 of word k / 1024
__device__ __forceinline__ void rs_mark(unsigned *gmask, int k) { atomicOr(&gmask[k >> 10], 1u << ((k >> 5) & 31)); }

template <class V>
__device__ void rs_steps(int n, const V &S, const V &ST, unsigned *key, unsigned *l1, unsigned *l2, unsigned *gmask,
                         int8_t *cf) {
    const unsigned lane = threadIdx.x;
    const int n1 = (n + 31) / 32;
    for (long long step = 0; step <= (long long)n; ++step) {
        unsigned v = l2[lane];
        const unsigned best = warp_max_u32(v);
        if (best == 0u) break;
        const int h = __ffs(__ballot_sync(0xffffffffu, v == best)) - 1;
        int g1 = 32 * h + (int)lane;
        v = g1 < n1 ? l1[g1] : 0u;
        const int g = 32 * h + __ffs(__ballot_sync(0xffffffffu, v == best)) - 1;
        int leaf = 32 * g + (int)lane;
        v = leaf < n ? key[leaf] : 0u;
        const int i = 32 * g + __ffs(__ballot_sync(0xffffffffu, v == best)) - 1;
        if (lane == 0) {
            cf[i] = CF_C;
            key[i] = 0u;
            rs_mark(gmask, i);
        }
        __syncwarp();
        // undecided in-block dependants of i become F (marked as new for this step)
        for (int p = ST.beg(i) + lane; p < ST.end(i); p += 32) {
            int j = ST.at(p);
            if (j >= 0 && cf[j] == CF_U) {
                cf[j] = CF_NEWF;
                key[j] = 0u;
                rs_mark(gmask, j);
            }
        }
        __syncwarp();
        // lambda_k += 1 for undecided in-block k in S_j of every new F point j
        for (int p = ST.beg(i) + lane; p < ST.end(i); p += 32) {
            int j = ST.at(p);
            if (j < 0 || cf[j] != CF_NEWF) continue;
            for (int q = S.beg(j); q < S.end(j); ++q) {
                int k = S.at(q);
                if (k >= 0 && cf[k] == CF_U) {
                    atomicAdd(&key[k], 1u << 16);
                    rs_mark(gmask, k);
                }
            }
        }
        // lambda_k -= 1 for undecided in-block k in S_i
        for (int q = S.beg(i) + lane; q < S.end(i); q += 32) {
            int k = S.at(q);
            if (k >= 0 && cf[k] == CF_U) {
                atomicSub(&key[k], 1u << 16);
                rs_mark(gmask, k);
            }
        }
        __syncwarp();
        for (int p = ST.beg(i) + lane; p < ST.end(i); p += 32) {
            int j = ST.at(p);
            if (j >= 0 && cf[j] == CF_NEWF) cf[j] = CF_F;
        }
        // recompute the changed level-1 nodes (one warp reduction each), then their level-2 nodes
        const unsigned word = gmask[lane];
        __syncwarp();
        gmask[lane] = 0u;
        unsigned hs = __ballot_sync(0xffffffffu, word != 0u);
        while (hs) {
            const int hh = __ffs(hs) - 1;
            hs &= hs - 1;
            unsigned bits = __shfl_sync(0xffffffffu, word, hh);
            while (bits) {
                const int gg = 32 * hh + __ffs(bits) - 1;
                bits &= bits - 1;
                const int lf = 32 * gg + (int)lane;
                const unsigned m = warp_max_u32(lf < n ? key[lf] : 0u);
                if (lane == 0) l1[gg] = m;
            }
            __syncwarp();
            const int gq = 32 * hh + (int)lane;
            const unsigned m = warp_max_u32(gq < n1 ? l1[gq] : 0u);
            if (lane == 0) l2[hh] = m;
        }
        __syncwarp();
    }
}

// copy the in-block part of graph G (rows b0..b1-1) into shared memory; returns false if it
// does not fit in cap bytes (nothing is used then)
__device__ bool rs_stage(const Graph &G, int b0, int b1, uint16_t *rp, uint16_t *col, size_t cap_entries) {
    const unsigned lane = threadIdx.x;
    const int n = b1 - b0;
    // counts, then an exclusive scan in lane-contiguous chunks
    const int chunk = (n + 31) / 32;
    const int r0 = min(n, (int)lane * chunk), r1 = min(n, r0 + chunk);
    int mine = 0;
    for (int li = r0; li < r1; ++li) {
        int c = 0;
        for (int p = G.rp[b0 + li]; p < G.rp[b0 + li + 1]; ++p) c += (G.col[p] >= b0 && G.col[p] < b1);
        rp[li] = c;
        mine += c;
    }
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if ((size_t)total > cap_entries || total > 65535) return false;
    int run = incl - mine;
    for (int li = r0; li < r1; ++li) {
        int c = rp[li];
        rp[li] = (uint16_t)run;
        run += c;
    }
    if (lane == 31) rp[n] = (uint16_t)total;
    __syncwarp();
    for (int li = r0; li < r1; ++li) {
        int q = rp[li];
        for (int p = G.rp[b0 + li]; p < G.rp[b0 + li + 1]; ++p) {
            int j = G.col[p];
            if (j >= b0 && j < b1) col[q++] = (uint16_t)(j - b0);
        }
    }
    __syncwarp();
    return true;
}

__global__ void __launch_bounds__(32) k_rs_split(int n_all, const int2 *__restrict__ blocks, Graph S, Graph ST,
                                                 int8_t *__restrict__ cf_out, int *status, int smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int b0 = blocks[blockIdx.x].x;          // this warp's index block [b0, b1)
    const int b1 = blocks[blockIdx.x].y;
    const int n = b1 - b0;
    const int n1 = (n + 31) / 32;
    unsigned *key = reinterpret_cast<unsigned *>(smem);
    unsigned *l1 = key + n;
    unsigned *l2 = l1 + n1;
    int8_t *cf = reinterpret_cast<int8_t *>(l2 + 32);
    uint16_t *srp = reinterpret_cast<uint16_t *>(cf + ((n + 15) & ~15));   // staged graphs: row offsets of S, ST
    uint16_t *strp = srp + (n + 1);
    uint16_t *scol = strp + (n + 1);                   // then the columns of S and of ST
    __shared__ unsigned gmask[32];                     // changed level-1 nodes of the current step
    const unsigned lane = threadIdx.x;
    gmask[lane] = 0u;

    for (int li = lane; li < n; li += 32) {
        const int i = b0 + li;
        int lam = 0;
        for (int p = ST.rp[i]; p < ST.rp[i + 1]; ++p) lam += (ST.col[p] >= b0 && ST.col[p] < b1);
        bool iso = (S.rp[i + 1] == S.rp[i]) && (ST.rp[i + 1] == ST.rp[i]);
        cf[li] = iso ? CF_F : CF_U;
        key[li] = iso ? 0u : (((unsigned)(lam + 1)) << 16) | (0xFFFFu - (unsigned)li);
    }
    __syncwarp();
    rs_rebuild(n, n1, key, l1, l2, lane);

    // both in-block graphs have the same number of entries; stage them if they fit
    const size_t used = (size_t)(reinterpret_cast<unsigned char *>(scol) - smem);
    const size_t cap = used < (size_t)smem_bytes ? ((size_t)smem_bytes - used) / (2 * sizeof(uint16_t)) : 0;
    bool staged = rs_stage(S, b0, b1, srp, scol, cap);
    if (staged) {
        const int e = srp[n];
        staged = rs_stage(ST, b0, b1, strp, scol + e, cap);
    }
    if (staged) {
        StagedView vs{srp, scol}, vt{strp, scol + srp[n]};
        rs_steps(n, vs, vt, key, l1, l2, gmask, cf);
    } else {
        GlobalView vs{S.rp, S.col, b0, b1}, vt{ST.rp, ST.col, b0, b1};
        rs_steps(n, vs, vt, key, l1, l2, gmask, cf);
    }
    for (int li = lane; li < n; li += 32) {
        int8_t c = cf[li];
        if (c != CF_C && c != CF_F) set_status(status, LAIR_ERR_DEVICE_TIMEOUT);
        cf_out[b0 + li] = c;
    }
}

// the largest number of in-block entries of S over the blocks (S and ST have the same count)
__global__ void __launch_bounds__(32) k_rs_count(const int2 *__restrict__ blocks, Graph S, int *__restrict__ maxcnt) {
    const int b0 = blocks[blockIdx.x].x, b1 = blocks[blockIdx.x].y;
    int c = 0;
    for (int i = b0 + threadIdx.x; i < b1; i += 32)
        for (int p = S.rp[i]; p < S.rp[i + 1]; ++p) c += (S.col[p] >= b0 && S.col[p] < b1);
    c = __reduce_add_sync(0xffffffffu, c);
    if (threadIdx.x == 0) atomicMax(maxcnt, c);
}

// per block: the in-block entries of S (for staging), and the largest in-block row lengths of S and ST;
// out[0..2] take the maxima over all blocks
__global__ void __launch_bounds__(32) k_rs_degrees(const int2 *__restrict__ blocks, Graph S, Graph ST,
                                                   int *__restrict__ out) {
    const int b0 = blocks[blockIdx.x].x, b1 = blocks[blockIdx.x].y;
    int c = 0, ms = 0, mt = 0;
    for (int i = b0 + threadIdx.x; i < b1; i += 32) {
        int ds = 0, dt = 0;
        for (int p = S.rp[i]; p < S.rp[i + 1]; ++p) ds += (S.col[p] >= b0 && S.col[p] < b1);
        for (int p = ST.rp[i]; p < ST.rp[i + 1]; ++p) dt += (ST.col[p] >= b0 && ST.col[p] < b1);
        c += ds;
        ms = max(ms, ds);
        mt = max(mt, dt);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    ms = __reduce_max_sync(0xffffffffu, ms);
    mt = __reduce_max_sync(0xffffffffu, mt);
    if (threadIdx.x == 0) {
        atomicMax(&out[0], c);
        atomicMax(&out[1], ms);
        atomicMax(&out[2], mt);
    }
}

// -------------------------------------------------------------------------------------
// The same first pass with a bucket queue, for blocks of at most RSB_MAX_N points whose lambda
// stays below nb buckets (lambda_k <= 2 |ST_k n block|: it starts at the in-block count and each
// dependant adds one when it becomes F). Bucket b is a bitmap over the block of the undecided
// points with lambda = b, so the point to take (largest lambda, then smallest index) is the lowest
// set bit of the highest non-empty bucket. The graphs are read through the cache; shared memory
// holds only the buckets and per-point bytes, so many blocks run on one SM at once. A step:
//   1. find i, which becomes C;
//   2. its undecided in-block dependants (ST_i) become F and leave their buckets;
//   3. lambda_k += 1 for undecided in-block k in S_j of every new F point j and lambda_k -= 1 for
//      undecided in-block k in S_i (byte atomics on lambda; each changed k is listed once);
//   4. every listed k moves from the bucket of its previous lambda to that of its new one.
// The sequence of points taken is the one of the tree version above (and of the oracle).
// -------------------------------------------------------------------------------------
struct RsbLayout {
    int W;                                // bitmap words per bucket (a multiple of 128)
    size_t bm, cnt, dflag, dlist, lam, bkt, cf, total;   // byte offsets in dynamic shared memory
};

__host__ __device__ inline size_t rsb_round16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline RsbLayout rsb_layout(int n, int nb, int dl) {
    RsbLayout L;
    L.W = (((n + 31) / 32) + 127) / 128 * 128;
    size_t o = 0;
    L.bm = o;    o += rsb_round16((size_t)nb * L.W * sizeof(unsigned));
    L.cnt = o;   o += rsb_round16((size_t)nb * sizeof(int));
    L.dflag = o; o += rsb_round16((size_t)L.W * sizeof(unsigned));
    L.dlist = o; o += rsb_round16((size_t)dl * sizeof(int));
    L.lam = o;   o += rsb_round16((size_t)n);          // one byte per point, updated by 32-bit atomics
    L.bkt = o;   o += rsb_round16((size_t)n);
    L.cf = o;    o += rsb_round16((size_t)n);
    L.total = o;
    return L;
}

struct RsbShared {
    unsigned *bm;      // nb bitmaps of W words
    int *cnt;          // points per bucket
    unsigned *dflag;   // listed in this step
    int *dlist;        // points whose lambda changed in this step
    unsigned *lamw;    // byte k: lambda_k
    uint8_t *bkt;      // the bucket that holds k
    int8_t *cf;
    int *ndirty;
};

// the steps of the bucket-queue first pass over in-block views of S and ST (local indices)
template <class V>
__device__ void rsb_steps(int n, int nb, int W, int dl, int top, const V &Sv, const V &STv, const RsbShared &q,
                          int *status) {
    const unsigned lane = threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    const int per = W / 32;                    // bitmap words scanned by each lane (4 or more, contiguous)
    for (int step = 0; step <= n; ++step) {
        // 1. the highest non-empty bucket at or below top, then its lowest set bit
        int b = -1;
        for (int t0 = top; t0 >= 0; t0 -= 32) {
            const int c = t0 - (int)lane;
            const unsigned m = __ballot_sync(FULL, c >= 0 && q.cnt[c] > 0);
            if (m) {
                b = t0 - (__ffs(m) - 1);
                break;
            }
        }
        if (b < 0) break;
        top = b;
        const unsigned *row = q.bm + (size_t)b * W + (size_t)lane * per;
        int fw = -1;
        unsigned fv = 0u;
        for (int r = 0; r < per && fw < 0; r += 4) {
            const uint4 u = *reinterpret_cast<const uint4 *>(row + r);
            if (u.x) { fw = r; fv = u.x; }
            else if (u.y) { fw = r + 1; fv = u.y; }
            else if (u.z) { fw = r + 2; fv = u.z; }
            else if (u.w) { fw = r + 3; fv = u.w; }
        }
        const unsigned fm = __ballot_sync(FULL, fw >= 0);
        if (fm == 0u) {                        // a count without its bit: cannot happen
            if (lane == 0) set_status(status, LAIR_ERR_DEVICE_TIMEOUT);
            break;
        }
        const int src = __ffs(fm) - 1;
        fw = __shfl_sync(FULL, fw, src) + src * per;
        fv = __shfl_sync(FULL, fv, src);
        const int li = 32 * fw + __ffs(fv) - 1;
        // 2. li becomes C; its undecided in-block dependants become F (new in this step)
        if (lane == 0) {
            q.cf[li] = CF_C;
            atomicAnd(&q.bm[b * W + (li >> 5)], ~(1u << (li & 31)));
            atomicSub(&q.cnt[b], 1);
        }
        const int sb = STv.beg(li), se = STv.end(li);
        for (int p = sb + (int)lane; p < se; p += 32) {
            const int j = STv.at(p);
            if (j >= 0 && q.cf[j] == CF_U) {
                q.cf[j] = CF_NEWF;
                const int bj = q.bkt[j];
                atomicAnd(&q.bm[bj * W + (j >> 5)], ~(1u << (j & 31)));
                atomicSub(&q.cnt[bj], 1);
            }
        }
        __syncwarp();
        // 3. lambda updates; the first touch of a point lists it
        auto touch = [&](int k, bool inc) {
            const unsigned sh = 8u * (unsigned)(k & 3);
            atomicAdd(&q.lamw[k >> 2], inc ? (1u << sh) : (0u - (1u << sh)));
            const unsigned bit = 1u << (k & 31);
            if (!(atomicOr(&q.dflag[k >> 5], bit) & bit)) {
                const int pos = atomicAdd(q.ndirty, 1);
                if (pos < dl) q.dlist[pos] = k;
                else set_status(status, LAIR_ERR_ARENA_OVERFLOW);
            }
        };
        for (int p = sb + (int)lane; p < se; p += 32) {
            const int j = STv.at(p);
            if (j < 0 || q.cf[j] != CF_NEWF) continue;
            for (int r = Sv.beg(j); r < Sv.end(j); ++r) {
                const int k = Sv.at(r);
                if (k >= 0 && q.cf[k] == CF_U) touch(k, true);
            }
        }
        for (int r = Sv.beg(li) + (int)lane; r < Sv.end(li); r += 32) {
            const int k = Sv.at(r);
            if (k >= 0 && q.cf[k] == CF_U) touch(k, false);
        }
        __syncwarp();
        // 4. listed points change bucket
        const int nd = min(*q.ndirty, dl);
        int hi = 0;
        for (int d = lane; d < nd; d += 32) {
            const int k = q.dlist[d];
            const unsigned bit = 1u << (k & 31);
            atomicAnd(&q.dflag[k >> 5], ~bit);
            const int lam = (int)((q.lamw[k >> 2] >> (8 * (k & 3))) & 0xFFu);
            const int ob = q.bkt[k];
            if (lam == ob) continue;
            if (lam >= nb) {
                set_status(status, LAIR_ERR_ARENA_OVERFLOW);
                continue;
            }
            atomicAnd(&q.bm[ob * W + (k >> 5)], ~bit);
            atomicOr(&q.bm[lam * W + (k >> 5)], bit);
            atomicSub(&q.cnt[ob], 1);
            atomicAdd(&q.cnt[lam], 1);
            q.bkt[k] = (uint8_t)lam;
            hi = max(hi, lam);
        }
        top = max(top, (int)__reduce_max_sync(FULL, (unsigned)hi));
        __syncwarp();
        if (lane == 0) *q.ndirty = 0;
        for (int p = sb + (int)lane; p < se; p += 32) {
            const int j = STv.at(p);
            if (j >= 0 && q.cf[j] == CF_NEWF) q.cf[j] = CF_F;
        }
        __syncwarp();
    }
}

// smem_bytes: the bucket layout of the largest block, plus (stage != 0) room to stage both in-block graphs
// (uint16 row offsets and columns) so that each step reads shared memory only. Staging pays when the level
// has at most one block per SM; with more blocks it costs occupancy, which hides more of each step's
// latency than the staging saves (measured), and the graphs are read through the cache.
__global__ void __launch_bounds__(32) k_rs_bucket(const int2 *__restrict__ blocks, Graph S, Graph ST, int nb, int dl,
                                                  int8_t *__restrict__ cf_out, int *status, int stage,
                                                  int smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int ndirty;
    const int b0 = blocks[blockIdx.x].x, b1 = blocks[blockIdx.x].y;
    const int n = b1 - b0;
    const RsbLayout Lo = rsb_layout(n, nb, dl);
    const int W = Lo.W;
    RsbShared q;
    q.bm = reinterpret_cast<unsigned *>(smem + Lo.bm);
    q.cnt = reinterpret_cast<int *>(smem + Lo.cnt);
    q.dflag = reinterpret_cast<unsigned *>(smem + Lo.dflag);
    q.dlist = reinterpret_cast<int *>(smem + Lo.dlist);
    q.lamw = reinterpret_cast<unsigned *>(smem + Lo.lam);
    q.bkt = smem + Lo.bkt;
    q.cf = reinterpret_cast<int8_t *>(smem + Lo.cf);
    q.ndirty = &ndirty;
    const unsigned lane = threadIdx.x;

    for (int e = lane; e < nb * W; e += 32) q.bm[e] = 0u;
    for (int e = lane; e < nb; e += 32) q.cnt[e] = 0;
    for (int e = lane; e < W; e += 32) q.dflag[e] = 0u;
    for (int e = lane; e < (n + 3) / 4; e += 32) q.lamw[e] = 0u;
    if (lane == 0) ndirty = 0;
    __syncwarp();
    int top = 0;
    for (int li = lane; li < n; li += 32) {
        const int i = b0 + li;
        int lam = 0;
        for (int p = ST.rp[i]; p < ST.rp[i + 1]; ++p) lam += (ST.col[p] >= b0 && ST.col[p] < b1);
        const bool iso = (S.rp[i + 1] == S.rp[i]) && (ST.rp[i + 1] == ST.rp[i]);
        q.cf[li] = iso ? CF_F : CF_U;
        q.bkt[li] = 0;
        if (iso) continue;
        if (lam >= nb) {                       // the host sized nb above every reachable lambda
            set_status(status, LAIR_ERR_ARENA_OVERFLOW);
            lam = nb - 1;
        }
        atomicAdd(&q.lamw[li >> 2], (unsigned)lam << (8 * (li & 3)));
        q.bkt[li] = (uint8_t)lam;
        atomicOr(&q.bm[lam * W + (li >> 5)], 1u << (li & 31));
        atomicAdd(&q.cnt[lam], 1);
        top = max(top, lam);
    }
    top = (int)__reduce_max_sync(0xffffffffu, (unsigned)top);
    __syncwarp();
    bool staged = false;
    uint16_t *srp = reinterpret_cast<uint16_t *>(smem + Lo.total);
    uint16_t *strp = srp + (n + 1);
    uint16_t *scol = strp + (n + 1);
    if (stage) {
        const size_t used = (size_t)(reinterpret_cast<unsigned char *>(scol) - smem);
        const size_t cap = used < (size_t)smem_bytes ? ((size_t)smem_bytes - used) / (2 * sizeof(uint16_t)) : 0;
        staged = rs_stage(S, b0, b1, srp, scol, cap);
        if (staged) staged = rs_stage(ST, b0, b1, strp, scol + srp[n], cap);
    }
    if (staged) {
        StagedView vs{srp, scol}, vt{strp, scol + srp[n]};
        rsb_steps(n, nb, W, dl, top, vs, vt, q, status);
    } else {
        GlobalView vs{S.rp, S.col, b0, b1}, vt{ST.rp, ST.col, b0, b1};
        rsb_steps(n, nb, W, dl, top, vs, vt, q, status);
    }
    for (int li = lane; li < n; li += 32) {
        const int8_t c = q.cf[li];
        if (c != CF_C && c != CF_F) set_status(status, LAIR_ERR_DEVICE_TIMEOUT);
        cf_out[b0 + li] = c;
    }
}

size_t rsb_smem_bytes(int n, int nb, int dl) { return rsb_layout(n, nb, dl).total; }

// the bytes to stage both in-block graphs of the fullest block as well
static size_t rsb_stage_bytes(int n, int max_inblock) {
    return 2 * sizeof(uint16_t) * ((size_t)n + 1) + 2 * sizeof(uint16_t) * (size_t)max_inblock + 16;
}

// shared memory of one block: the fixed part (keys, tree, splitting, row offsets) plus room for
// both staged in-block graphs of the fullest block, up to RS_SMEM_MAX bytes in all (blocks that
// do not fit then read their graphs from global memory)
size_t rs_smem_bytes(int n, int max_inblock) {
    int n1 = (n + 31) / 32;
    size_t fixed = sizeof(unsigned) * ((size_t)n + n1 + 32) + (((size_t)n + 15) & ~(size_t)15) +
                   sizeof(uint16_t) * 2 * ((size_t)n + 1);
    size_t want = fixed + 2 * sizeof(uint16_t) * (size_t)max_inblock + 16;
    return want < RS_SMEM_MAX ? want : (fixed < RS_SMEM_MAX ? RS_SMEM_MAX : fixed);
}

// -------------------------------------------------------------------------------------
// coarse numbering
// -------------------------------------------------------------------------------------
__global__ void k_cflag(int n, const int8_t *__restrict__ cf, int *__restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = cf[i] == CF_C;
}

__global__ void k_cidx(int n, const int8_t *__restrict__ cf, const int *__restrict__ scan, int *__restrict__ cidx,
                       int *__restrict__ cpts) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (cf[i] == CF_C) {
            cidx[i] = scan[i];
            cpts[scan[i]] = i;
        } else {
            cidx[i] = -1;
        }
    }
}

// -------------------------------------------------------------------------------------
// Neighbourhoods (Sec. 3.1; F-F-C only, Sec. 4). For C point i in graph G:
// distance 1: G_i n F; distance 2 adds G_j n F for each j in G_i n F; each further distance
// (k_nb_expand) adds G_j n F for each j of the previous set. Sorted, unique.
// -------------------------------------------------------------------------------------
__global__ void k_nb_bound(int nc, const int *__restrict__ cpts, Graph G, const int8_t *__restrict__ cf,
                           int distance, int *__restrict__ ub) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int i = cpts[c];
        int u = 0;
        for (int p = G.rp[i]; p < G.rp[i + 1]; ++p) {
            int j = G.col[p];
            if (cf[j] != CF_F) continue;
            u += 1;
            if (distance >= 2) u += G.rp[j + 1] - G.rp[j];
        }
        ub[c] = u;
    }
}

__global__ void k_nb_fill(int nc, const int *__restrict__ cpts, Graph G, const int8_t *__restrict__ cf,
                          int distance, const int *__restrict__ off, int *__restrict__ tmp, int *__restrict__ cnt) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int i = cpts[c];
        int *t = tmp + off[c];
        int m = 0;
        for (int p = G.rp[i]; p < G.rp[i + 1]; ++p) {
            int j = G.col[p];
            if (cf[j] != CF_F) continue;
            t[m++] = j;
            if (distance >= 2)
                for (int q = G.rp[j]; q < G.rp[j + 1]; ++q) {
                    int k = G.col[q];
                    if (cf[k] == CF_F && k != i) t[m++] = k;
                }
        }
        // insertion sort + unique
        for (int a = 1; a < m; ++a) {
            int v = t[a], b = a - 1;
            while (b >= 0 && t[b] > v) { t[b + 1] = t[b]; --b; }
            t[b + 1] = v;
        }
        int u = 0;
        for (int a = 0; a < m; ++a)
            if (u == 0 || t[u - 1] != t[a]) t[u++] = t[a];
        cnt[c] = u;
    }
}

// One more distance (distances beyond two): the current set of C point c (nb_rp / nb_col) plus
// G_j n F for every j in it. phase 0: the bound |set| + sum |G_j|; phase 1: the sorted, unique set
// written at off[c] with its size in cnt[c].
__global__ void k_nb_expand(int phase, int nc, const int *__restrict__ cpts, Graph G, const int8_t *__restrict__ cf,
                            const int *__restrict__ nb_rp, const int *__restrict__ nb_col, const int *__restrict__ off,
                            int *__restrict__ tmp, int *__restrict__ cnt) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int i = cpts[c];
        const int b = nb_rp[c], e = nb_rp[c + 1];
        if (phase == 0) {
            int u = e - b;
            for (int a = b; a < e; ++a) u += G.rp[nb_col[a] + 1] - G.rp[nb_col[a]];
            cnt[c] = u;
            continue;
        }
        int *t = tmp + off[c];
        int m = 0;
        for (int a = b; a < e; ++a) {
            const int j = nb_col[a];
            t[m++] = j;
            for (int q = G.rp[j]; q < G.rp[j + 1]; ++q) {
                const int k = G.col[q];
                if (cf[k] == CF_F && k != i) t[m++] = k;
            }
        }
        for (int a = 1; a < m; ++a) {
            int v = t[a], bb = a - 1;
            while (bb >= 0 && t[bb] > v) { t[bb + 1] = t[bb]; --bb; }
            t[bb + 1] = v;
        }
        int u = 0;
        for (int a = 0; a < m; ++a)
            if (u == 0 || t[u - 1] != t[a]) t[u++] = t[a];
        cnt[c] = u;
    }
}

__global__ void k_nb_compact(int nc, const int *__restrict__ off, const int *__restrict__ tmp,
                             const int *__restrict__ nb_rp, int *__restrict__ nb_col) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int b = nb_rp[c], e = nb_rp[c + 1];
        const int *t = tmp + off[c];
        for (int k = b; k < e; ++k) nb_col[k] = t[k - b];
    }
}

// -------------------------------------------------------------------------------------
// exclusive scan of m <= SMALL_SCAN_MAX ints in one CTA, in tiles of 16384: warp w scans the
// 512 entries [512 w, 512 w + 512) of a tile as 16 coalesced strips of 32 held in registers
// -------------------------------------------------------------------------------------
constexpr int SCAN_STRIPS = 16;
constexpr int SCAN_TILE = 1024 * SCAN_STRIPS;

__global__ void __launch_bounds__(1024) k_small_scan(int m, const int *__restrict__ in, int *__restrict__ out) {
    __shared__ int wsum[32];
    __shared__ int tile_total;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int carry = 0;
    for (int base = 0; base < m; base += SCAN_TILE) {
        const int seg = base + w * 32 * SCAN_STRIPS + lane;
        int v[SCAN_STRIPS];
#pragma unroll
        for (int k = 0; k < SCAN_STRIPS; ++k) v[k] = seg + 32 * k < m ? in[seg + 32 * k] : 0;
        int run = 0;
#pragma unroll
        for (int k = 0; k < SCAN_STRIPS; ++k) {
            int x = v[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            v[k] = run + x - v[k];
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) wsum[w] = run;
        __syncthreads();
        if (w == 0) {
            const int sv = wsum[lane];
            int x = sv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            wsum[lane] = x - sv;
            if (lane == 31) tile_total = x;
        }
        __syncthreads();
        const int off = carry + wsum[w];
#pragma unroll
        for (int k = 0; k < SCAN_STRIPS; ++k)
            if (seg + 32 * k < m) out[seg + 32 * k] = off + v[k];
        carry += tile_total;
        __syncthreads();
    }
}

void small_scan(int m, const int *in, int *out, cudaStream_t s) {
    k_small_scan<<<1, 1024, 0, s>>>(m, in, out);
    count_launch();
}

// -------------------------------------------------------------------------------------
// exclusive scan of any length in one pass (decoupled look-back). A CTA takes the next tile
// index from a counter (so every tile before it belongs to a CTA that is already running or
// done), scans its LB_TILE entries as k_small_scan does, publishes the tile total, reads the
// published totals and prefixes of the tiles before it 32 at a time until it meets a prefix,
// and publishes its own inclusive prefix. state[t] packs (flag << 32) | value in one 64-bit
// word (flag 0: nothing yet, 1: tile total, 2: inclusive prefix); state and the counter are
// zero on entry. Every wait is bounded: one that runs out sets LAIR_ERR_DEVICE_TIMEOUT and the
// CTA goes on with what it has.
// -------------------------------------------------------------------------------------
constexpr int LB_THREADS = 512;
constexpr int LB_STRIPS = 8;
constexpr int LB_TILE = LB_THREADS * LB_STRIPS;
constexpr long long LB_WAIT_POLLS = 1ll << 22;

__global__ void __launch_bounds__(LB_THREADS) k_scan_lookback(long long m, const int *__restrict__ in,
                                                              int *__restrict__ out, unsigned long long *state,
                                                              int *counter, int *status) {
    __shared__ int wsum[LB_THREADS / 32];
    __shared__ int tile_s, prefix_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) tile_s = atomicAdd(counter, 1);
    __syncthreads();
    const long long tile = tile_s;
    const long long seg = tile * LB_TILE + (long long)w * 32 * LB_STRIPS + lane;
    int v[LB_STRIPS];
#pragma unroll
    for (int k = 0; k < LB_STRIPS; ++k) v[k] = seg + 32 * k < m ? in[seg + 32 * k] : 0;
    int run = 0;
#pragma unroll
    for (int k = 0; k < LB_STRIPS; ++k) {
        int x = v[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        v[k] = run + x - v[k];
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) wsum[w] = run;
    __syncthreads();
    if (w == 0) {
        const int sv = lane < LB_THREADS / 32 ? wsum[lane] : 0;
        int x = sv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < LB_THREADS / 32) wsum[lane] = x - sv;
        const int total = __shfl_sync(0xffffffffu, x, 31);
        if (lane == 0) {
            atomicExch(&state[tile], ((tile == 0 ? 2ull : 1ull) << 32) | (unsigned)total);
        }
        // look back over the tiles before this one
        int excl = 0;
        long long spins = 0;
        for (long long hi = tile - 1; hi >= 0; hi -= 32) {
            const long long p = hi - lane;
            unsigned long long st = p >= 0 ? *(volatile unsigned long long *)&state[p] : (2ull << 32);
            while (__any_sync(0xffffffffu, (st >> 32) == 0ull)) {
                if (++spins > LB_WAIT_POLLS) {
                    if (lane == 0) set_status(status, LAIR_ERR_DEVICE_TIMEOUT);
                    st = (2ull << 32);
                    break;
                }
                __nanosleep(32);
                if ((st >> 32) == 0ull) st = *(volatile unsigned long long *)&state[p];
            }
            const unsigned pm = __ballot_sync(0xffffffffu, (st >> 32) == 2ull);
            const int stop = pm ? __ffs(pm) - 1 : 31;
            excl += __reduce_add_sync(0xffffffffu, lane <= stop ? (unsigned)(st & 0xffffffffull) : 0u);
            if (pm) break;
        }
        if (lane == 0) {
            prefix_s = excl;
            if (tile > 0) atomicExch(&state[tile], (2ull << 32) | (unsigned)(excl + total));
        }
    }
    __syncthreads();
    const int off = prefix_s + wsum[w];
#pragma unroll
    for (int k = 0; k < LB_STRIPS; ++k)
        if (seg + 32 * k < m) out[seg + 32 * k] = off + v[k];
}

size_t scan_state_bytes(long long m) { return (size_t)((m + LB_TILE - 1) / LB_TILE) * 8 + 16; }

// state: scan_state_bytes(m) bytes of scratch; out may be in (each tile reads its inputs before it writes)
cudaError_t launch_scan(long long m, const int *in, int *out, void *state, int *status, cudaStream_t s) {
    const long long tiles = (m + LB_TILE - 1) / LB_TILE;
    cudaError_t e = cudaMemsetAsync(state, 0, scan_state_bytes(m), s);
    if (e != cudaSuccess) return e;
    unsigned long long *st = static_cast<unsigned long long *>(state);
    int *counter = reinterpret_cast<int *>(st + tiles);
    k_scan_lookback<<<(unsigned)(tiles > 0 ? tiles : 1), LB_THREADS, 0, s>>>(m, in, out, st, counter, status);
    count_launch();
    return cudaGetLastError();
}

// -------------------------------------------------------------------------------------
// host wrappers
// -------------------------------------------------------------------------------------
static const int TB = 256;

void launch_strength(const DCsr &A, double theta, int absmode, uint8_t *mask, int *cnt, cudaStream_t s) {
    k_strength<<<grid_for(A.nr, TB), TB, 0, s>>>(A.nr, A.rp, A.col, A.val, theta, absmode, mask, cnt);
    count_launch();
}

void launch_graph_fill(const DCsr &A, const uint8_t *mask, const Graph &G, cudaStream_t s) {
    k_graph_fill<<<grid_for(A.nr, TB), TB, 0, s>>>(A.nr, A.rp, A.col, mask, G.rp, G.col);
    count_launch();
}

void launch_col_count(int nr, const int *rp, const int *col, int *cnt, cudaStream_t s) {
    k_col_count<<<grid_for(nr, TB), TB, 0, s>>>(nr, rp, col, cnt);
    count_launch();
}

void launch_transpose_scatter(int nr, const int *rp, const int *col, const double *val, const int *trp,
                              int *cursor, int *tcol, double *tval, cudaStream_t s) {
    k_transpose_scatter<<<grid_for(nr, TB), TB, 0, s>>>(nr, rp, col, val, trp, cursor, tcol, tval);
    count_launch();
}

// lists: 2 * nr + 2 ints of scratch, the first two zero
void launch_sort_rows(int nr, const int *rp, int *col, double *val, int *lists, cudaStream_t s) {
    if (nr <= 0) return;
    k_sort_rows<<<grid_for(nr, 128), 128, 0, s>>>(nr, rp, col, val, lists);
    k_sort_rows_warp<<<device_sms() * 8, 256, 0, s>>>(nr, rp, col, val, lists);
    k_sort_rows_cta<<<device_sms() * 2, SORT_CTA_THREADS, 0, s>>>(nr, rp, col, val, lists);
    count_launch(3);
}

void launch_pmis_init(int n, const Graph &ST, uint64_t seed, double *w, int8_t *cf, cudaStream_t s) {
    k_pmis_init<<<grid_for(n, TB), TB, 0, s>>>(n, ST.rp, seed, w, cf);
    count_launch();
}

// ctl: 4 ints, zero
cudaError_t launch_pmis_all(int n, const Graph &S, const Graph &ST, double *w, int8_t *cf, int8_t *newc, int *lists,
                            int *ctl, int *status, int wait_polls, cudaStream_t s) {
    long long limit = wait_polls > 0 ? (long long)wait_polls : GRID_WAIT_POLLS;
    if (n <= PMIS_CLUSTER * PMIS_THREADS) {
        const int c = n > 0 ? (n + PMIS_THREADS - 1) / PMIS_THREADS : 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(PMIS_THREADS);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k_pmis_cluster, n, S, ST, w, cf, newc) == cudaSuccess) {
            count_launch();
            return cudaSuccess;
        }
        cudaGetLastError();   // not launchable here: use the grid-wide version
    }
    int dev = 0, per_sm = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pmis_coop, PMIS_THREADS, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // two CTAs per SM where they fit: twice the loads in flight in each round, for two barrier arrivals per SM
    int grid = sms * (per_sm < 2 ? per_sm : 2);
    const int need = (n + PMIS_THREADS - 1) / PMIS_THREADS;
    if (grid > need) grid = need > 0 ? need : 1;
    void *args[] = {(void *)&n,     (void *)&S,   (void *)&ST,     (void *)&w,    (void *)&cf,
                    (void *)&newc,  (void *)&lists, (void *)&ctl, (void *)&status, (void *)&limit};
    e = cudaLaunchCooperativeKernel((const void *)k_pmis_coop, dim3(grid), dim3(PMIS_THREADS), args, 0, s);
    count_launch();
    return e;
}


// blocks: nblocks (b0, b1) pairs on the device, every block at most Bmax points
void launch_rs_count(const int2 *blocks, int nblocks, const Graph &S, int *maxcnt, cudaStream_t s) {
    k_rs_count<<<nblocks, 32, 0, s>>>(blocks, S, maxcnt);
    count_launch();
}

void launch_rs_degrees(const int2 *blocks, int nblocks, const Graph &S, const Graph &ST, int *out, cudaStream_t s) {
    k_rs_degrees<<<nblocks, 32, 0, s>>>(blocks, S, ST, out);
    count_launch();
}

cudaError_t launch_rs_bucket(const int2 *blocks, int nblocks, int Bmax, int nb, int dl, int max_inblock,
                             const Graph &S, const Graph &ST, int8_t *cf, int *status, cudaStream_t s) {
    size_t bytes = rsb_smem_bytes(Bmax, nb, dl);
    int stage = 0;
    if (nblocks <= device_sms()) {
        const size_t want = bytes + rsb_stage_bytes(Bmax, max_inblock);
        stage = 1;
        bytes = want < (size_t)RS_SMEM_MAX ? want : (bytes > (size_t)RS_SMEM_MAX ? bytes : (size_t)RS_SMEM_MAX);
    }
    cudaError_t e = cudaFuncSetAttribute(k_rs_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_rs_bucket<<<nblocks, 32, bytes, s>>>(blocks, S, ST, nb, dl, cf, status, stage, (int)bytes);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rs(int n, const int2 *blocks, int nblocks, int Bmax, int max_inblock, const Graph &S, const Graph &ST,
                      int8_t *cf, int *status, cudaStream_t s) {
    size_t bytes = rs_smem_bytes(Bmax, max_inblock);
    cudaError_t e = cudaFuncSetAttribute(k_rs_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_rs_split<<<nblocks, 32, bytes, s>>>(n, blocks, S, ST, cf, status, (int)bytes);
    count_launch();
    return cudaGetLastError();
}

void launch_cidx(int n, const int8_t *cf, int *flag, int *cidx, int *cpts, int phase, cudaStream_t s) {
    if (phase == 0) k_cflag<<<grid_for(n, TB), TB, 0, s>>>(n, cf, flag);
    else k_cidx<<<grid_for(n, TB), TB, 0, s>>>(n, cf, flag, cidx, cpts);
    count_launch();
}

void launch_nb_bound(int nc, const int *cpts, const Graph &G, const int8_t *cf, int distance, int *ub, cudaStream_t s) {
    k_nb_bound<<<grid_for(nc, TB), TB, 0, s>>>(nc, cpts, G, cf, distance, ub);
    count_launch();
}

void launch_nb_fill(int nc, const int *cpts, const Graph &G, const int8_t *cf, int distance, const int *off, int *tmp,
                    int *cnt, cudaStream_t s) {
    k_nb_fill<<<grid_for(nc, 128), 128, 0, s>>>(nc, cpts, G, cf, distance, off, tmp, cnt);
    count_launch();
}

void launch_nb_expand(int phase, int nc, const int *cpts, const Graph &G, const int8_t *cf, const int *nb_rp,
                      const int *nb_col, const int *off, int *tmp, int *cnt, cudaStream_t s) {
    k_nb_expand<<<grid_for(nc, TB), TB, 0, s>>>(phase, nc, cpts, G, cf, nb_rp, nb_col, off, tmp, cnt);
    count_launch();
}

void launch_nb_compact(int nc, const int *off, const int *tmp, const int *nb_rp, int *nb_col, cudaStream_t s) {
    k_nb_compact<<<grid_for(nc, TB), TB, 0, s>>>(nc, off, tmp, nb_rp, nb_col);
    count_launch();
}

// neighbourhoods read off a kept operator (hierarchy refresh): row c of (rp, col) is the neighbourhood of C point
// cpts[c] plus that point itself (R = [Z I] by rows, P^T by rows), so set c is the row without cpts[c]
__global__ void k_nb_from_rows(int nc, const int *__restrict__ rp, const int *__restrict__ col,
                               const int *__restrict__ cpts, int *__restrict__ nb_rp, int *__restrict__ nb_col) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int b = rp[c], e = rp[c + 1], self = cpts[c];
        int q = b - c;
        nb_rp[c] = q;
        if (c == nc - 1) nb_rp[nc] = e - nc;
        for (int k = b; k < e; ++k)
            if (col[k] != self) nb_col[q++] = col[k];
    }
}

void launch_nb_from_rows(int nc, const int *rp, const int *col, const int *cpts, int *nb_rp, int *nb_col,
                         cudaStream_t s) {
    if (nc <= 0) return;
    k_nb_from_rows<<<grid_for(nc, TB), TB, 0, s>>>(nc, rp, col, cpts, nb_rp, nb_col);
    count_launch();
}

}  // namespace lair
