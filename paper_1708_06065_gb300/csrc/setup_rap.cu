// setup_rap.cu -- Galerkin coarse operator K = R A P (Sec. 2.1), lumping of small
// entries into the diagonal (Sec. 3.3), Jacobi diagonals, FP32 copies, and the
// dense factorisation of the coarsest level.
//
// Products are formed row by row as Z = X Y (first R A, then (R A) P). Entry (a, l)
// of a row starts at 0 and receives fma(x_ak, y_kl, .) for the k of row a of X in
// ascending order, exactly one update per k; the pattern is the full symbolic
// product (structural zeros kept). This fixed order makes K a deterministic function
// of R, A and P, independent of the thread layout.
#include "setup_kernels.cuh"

namespace lair {

constexpr int WARP_CAP = 2048;      // largest hash table of the warp kernels (rows with ub <= WARP_CAP / 2)

__global__ void k_spgemm_ub(int nr, const int *__restrict__ xrp, const int *__restrict__ xcol,
                            const int *__restrict__ yrp, int *__restrict__ ub) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nr; a += gridDim.x * blockDim.x) {
        int u = 0;
        for (int p = xrp[a]; p < xrp[a + 1]; ++p) {
            int k = xcol[p];
            u += yrp[k + 1] - yrp[k];
        }
        ub[a] = u;
    }
}

// bins by the row's upper bound: 0: ub <= 128 (256 slots), 1: ub <= 512 (1024), 2: ub <= 1024 (2048), 3: larger;
// with merge, rows of X with at most SPGEMM_MERGE_K entries go to the merge bin whatever their bound
__device__ __forceinline__ int spgemm_bin(int u) { return u <= 128 ? 0 : (u <= 512 ? 1 : (u <= WARP_CAP / 2 ? 2 : 3)); }

__global__ void k_spgemm_classify(int nr, const int *__restrict__ off, const int *__restrict__ xrp, bool merge,
                                  bool merge2, int merge_ub_max, int *__restrict__ lists, int *__restrict__ counts,
                                  int *__restrict__ ubmax) {
    const unsigned lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x - lane; base < nr; base += stride) {
        const int a = (int)(base + lane);
        const bool act = a < nr;
        const int u = act ? off[a + 1] - off[a] : 0;
        const int xl = act ? xrp[a + 1] - xrp[a] : 0;
        const int b = (merge && xl <= SPGEMM_MERGE_K && u <= merge_ub_max) ? SPGEMM_BIN_MERGE
                    : (merge2 && xl <= SPGEMM_MERGE_K2) ? SPGEMM_BIN_MERGE2 : spgemm_bin(u);
        for (int bb = 0; bb < SPGEMM_BINS; ++bb) {       // one atomic per warp and bin
            const unsigned m = __ballot_sync(0xffffffffu, act && b == bb);
            if (!m) continue;
            int p0 = 0;
            if (lane == __ffs(m) - 1) p0 = atomicAdd(&counts[bb], __popc(m));
            p0 = __shfl_sync(0xffffffffu, p0, __ffs(m) - 1);
            if (act && b == bb) lists[(size_t)bb * nr + p0 + __popc(m & ((1u << lane) - 1u))] = a;
        }
        if (act && b == SPGEMM_BIN_CTA) atomicMax(ubmax, u);
    }
}

// One thread per row a of a merge bin: the rows of Y named by the (at most K) entries
// of row a of X are merged in column order; column j receives fma(x_ak, y_kj, .) for those k in
// ascending order, starting from 0 -- the same updates in the same order as the hashed kernels,
// written directly in column order.
template <int K>
__device__ __forceinline__ int merge_row(const SpgemmArgs &g, int a, int o) {
    const int xb = g.xrp[a], nk = g.xrp[a + 1] - xb;
    int pos[K], end[K], cj[K];
    double xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        pos[u] = 0;
        end[u] = 0;
        xv[u] = 0.0;
        if (u < nk) {
            const int k = g.xcol[xb + u];
            pos[u] = g.yrp[k];
            end[u] = g.yrp[k + 1];
            xv[u] = g.xval[xb + u];
        }
        cj[u] = pos[u] < end[u] ? g.ycol[pos[u]] : 0x7fffffff;
    }
    int c = 0;
    for (;;) {
        int j = 0x7fffffff;
#pragma unroll
        for (int u = 0; u < K; ++u) j = min(j, cj[u]);
        if (j == 0x7fffffff) break;
        double v = 0.0;
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (cj[u] == j) {
                v = __fma_rn(xv[u], g.yval[pos[u]], v);
                ++pos[u];
                cj[u] = pos[u] < end[u] ? g.ycol[pos[u]] : 0x7fffffff;
            }
        g.tcol[o + c] = j;
        g.tval[o + c] = v;
        ++c;
    }
    return c;
}

template <int K>
__global__ void __launch_bounds__(K <= 8 ? 256 : 128) k_spgemm_merge(SpgemmArgs g, const int *__restrict__ list,
                                                                     const int *__restrict__ count) {
    const int n = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int a = list[t];
        g.cnt[a] = merge_row<K>(g, a, g.off[a]);
    }
}

// The fused triple product X Y P for a one-point P (at most one entry per row), one thread per row of X
// with at most K entries and a bound ub <= SPGEMM_P1_CAP. Row a of X Y is merged in column order as above;
// each finished entry (l, v), in ascending l, looks up P's row l in the direct map (pmap_col[l],
// pmap_val[l]: -1 / 0 for an empty row) and waits in a register queue of P1_LAG entries, so that the
// lookup is in flight while the merge goes on; the entry leaving the queue adds fma(v, p_l, .) to column
// P(l) of the result, a short list in the thread's own column of shared memory (entry e at
// e * blockDim + thread: no bank conflicts). The list is put in column order by insertion and written
// out. Every result entry thus receives its terms in ascending l, starting from 0: the fma sequence of
// the hashed fused kernels. The result has at most ub entries, so the list holds SPGEMM_P1_CAP.
constexpr int P1_LAG = 4;

template <int K>
__global__ void __launch_bounds__(SPGEMM_P1_THREADS) k_spgemm_merge_p1(SpgemmArgs g, const int *__restrict__ list,
                                                                       const int *__restrict__ count,
                                                                       const int *__restrict__ pmap_col,
                                                                       const double *__restrict__ pmap_val) {
    __shared__ int lcol[SPGEMM_P1_CAP * SPGEMM_P1_THREADS];
    __shared__ double lval[SPGEMM_P1_CAP * SPGEMM_P1_THREADS];
    constexpr int T = SPGEMM_P1_THREADS;
    int *mc = lcol + threadIdx.x;
    double *mv = lval + threadIdx.x;
    const int n = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int a = list[t];
        const int xb = g.xrp[a], nk = g.xrp[a + 1] - xb;
        int pos[K], end[K], cj[K];
        double xv[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
            pos[u] = 0;
            end[u] = 0;
            xv[u] = 0.0;
            if (u < nk) {
                const int k = g.xcol[xb + u];
                pos[u] = g.yrp[k];
                end[u] = g.yrp[k + 1];
                xv[u] = g.xval[xb + u];
            }
            cj[u] = pos[u] < end[u] ? g.ycol[pos[u]] : 0x7fffffff;
        }
        int nout = 0;
        // the queue: slot 0 is the oldest; qb < -1 marks an empty slot
        int qb[P1_LAG];
        double qv[P1_LAG], qp[P1_LAG];
#pragma unroll
        for (int q = 0; q < P1_LAG; ++q) {
            qb[q] = -2;
            qv[q] = 0.0;
            qp[q] = 0.0;
        }
        auto add = [&](int b, double v, double pv) {
            if (b < 0) return;
            int f = 0;
            while (f < nout && mc[f * T] != b) ++f;
            if (f == nout) {
                mc[f * T] = b;
                mv[f * T] = __fma_rn(v, pv, 0.0);
                ++nout;
            } else {
                mv[f * T] = __fma_rn(v, pv, mv[f * T]);
            }
        };
        for (;;) {
            int j = 0x7fffffff;
#pragma unroll
            for (int u = 0; u < K; ++u) j = min(j, cj[u]);
            if (j == 0x7fffffff) break;
            double v = 0.0;
#pragma unroll
            for (int u = 0; u < K; ++u)
                if (cj[u] == j) {
                    v = __fma_rn(xv[u], g.yval[pos[u]], v);
                    ++pos[u];
                    cj[u] = pos[u] < end[u] ? g.ycol[pos[u]] : 0x7fffffff;
                }
            // the oldest entry leaves the queue; (j, v) enters with its lookup issued now
            add(qb[0], qv[0], qp[0]);
#pragma unroll
            for (int q = 0; q + 1 < P1_LAG; ++q) {
                qb[q] = qb[q + 1];
                qv[q] = qv[q + 1];
                qp[q] = qp[q + 1];
            }
            qb[P1_LAG - 1] = pmap_col[j];
            qp[P1_LAG - 1] = pmap_val[j];
            qv[P1_LAG - 1] = v;
        }
#pragma unroll
        for (int q = 0; q < P1_LAG; ++q) add(qb[q], qv[q], qp[q]);
        for (int x = 1; x < nout; ++x) {
            const int kc = mc[x * T];
            const double kv = mv[x * T];
            int y = x - 1;
            while (y >= 0 && mc[y * T] > kc) {
                mc[(y + 1) * T] = mc[y * T];
                mv[(y + 1) * T] = mv[y * T];
                --y;
            }
            mc[(y + 1) * T] = kc;
            mv[(y + 1) * T] = kv;
        }
        const int o = g.off[a];
        for (int e = 0; e < nout; ++e) {
            g.tcol[o + e] = mc[e * T];
            g.tval[o + e] = mv[e * T];
        }
        g.cnt[a] = nout;
    }
}

// direct map of a P with at most one entry per row: (column, value) of row l, or (-1, 0)
__global__ void k_p1_map(int n, const int *__restrict__ prp, const int *__restrict__ pcol, const double *__restrict__ pval,
                         int *__restrict__ mcol, double *__restrict__ mval) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const int b = prp[l];
        const bool has = prp[l + 1] > b;
        mcol[l] = has ? pcol[b] : -1;
        mval[l] = has ? pval[b] : 0.0;
    }
}

__device__ __forceinline__ unsigned hash_slot(int key, unsigned mask) { return ((unsigned)key * 2654435761u) & mask; }

constexpr int XCHUNK = 64;            // entries of an X row staged at a time
// per-warp staging after the hash table: x (XCHUNK doubles), px/py (2 x 32 doubles), Y row starts
// (XCHUNK ints), offsets (XCHUNK + 1 ints); 16-byte aligned
constexpr size_t SPGEMM_EXTRA = ((XCHUNK * sizeof(double) + 64 * sizeof(double) + (2 * XCHUNK + 1) * sizeof(int)) + 15) &
                                ~(size_t)15;

// the cnt compacted (column, value) pairs of a row, sorted by column, written to col/val
template <int R>
__device__ __forceinline__ void sorted_out(const int *keys, const double *vals, int cnt, int *col, double *val, int lane) {
    int k[R];
    double v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = 32 * r + lane;
        k[r] = e < cnt ? keys[e] : 0x7fffffff;
        v[r] = e < cnt ? vals[e] : 0.0;
    }
    warp_bitonic<R>(k, v, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = 32 * r + lane;
        if (e < cnt) {
            col[e] = k[r];
            val[e] = v[r];
        }
    }
}

// the leader of group grp (lanes holding column l) adds the group's products px[b] * py[b] to
// the table entry of l, in ascending lane order
__device__ __forceinline__ void hash_group_fma(int *keys, double *vals, unsigned mask, int l, unsigned grp,
                                               const double *px, const double *py) {
    unsigned h = hash_slot(l, mask);
    double v;
    for (;;) {
        const int prev = atomicCAS(&keys[h], -1, l);
        if (prev == -1) {
            v = 0.0;
            break;
        }
        if (prev == l) {
            v = vals[h];
            break;
        }
        h = (h + 1) & mask;
    }
    for (unsigned m = grp; m; m &= m - 1) {
        const int b = __ffs(m) - 1;
        v = __fma_rn(px[b], py[b], v);
    }
    vals[h] = v;
}

// compact the occupied slots of a table of cap slots to [0, cnt); returns cnt
__device__ __forceinline__ int compact_table(int *keys, double *vals, unsigned cap, unsigned lane) {
    int cnt = 0;
    for (unsigned base = 0; base < cap; base += 32) {
        const int key = keys[base + lane];
        const double v = vals[base + lane];
        const unsigned occ = __ballot_sync(0xffffffffu, key != -1);
        __syncwarp();
        if (key != -1) {
            const int pos = cnt + __popc(occ & ((1u << lane) - 1u));
            keys[pos] = key;
            vals[pos] = v;
        }
        cnt += __popc(occ);
        __syncwarp();
    }
    return cnt;
}

template <int R>
__device__ __forceinline__ void sorted_out(const int *keys, const double *vals, int cnt, int *col, double *val, int lane);

// write the compacted table [0, cnt) sorted by column (cnt <= 32 * RMAX)
template <int RMAX>
__device__ __forceinline__ void write_sorted(const int *keys, const double *vals, int cnt, int *col, double *val, int lane) {
    if (cnt <= 32) sorted_out<1>(keys, vals, cnt, col, val, lane);
    else if (RMAX >= 2 && cnt <= 64) sorted_out<(RMAX >= 2 ? 2 : 1)>(keys, vals, cnt, col, val, lane);
    else if (RMAX >= 4 && cnt <= 128) sorted_out<(RMAX >= 4 ? 4 : 1)>(keys, vals, cnt, col, val, lane);
    else if (RMAX >= 8 && cnt <= 256) sorted_out<(RMAX >= 8 ? 8 : 1)>(keys, vals, cnt, col, val, lane);
    else if (RMAX >= 16) sorted_out<(RMAX >= 16 ? 16 : 1)>(keys, vals, cnt, col, val, lane);
}

// Loads the compacted entries [0, cnt) of a row table of cap slots into registers (entry
// e = 32 r + lane in kk[r], vv[r]; padding INT_MAX / 0) and finds each entry's rank by column
// through a bitmap of the row's column span kept in the free upper half of the table
// (cnt <= cap / 2): bitmap words in vals[cap/2, cap), word prefix counts in keys[cap/2, cap).
// Lane l owns words l, l + 32, ..., so neither pass has bank conflicts. Returns false (ranks not
// set, registers loaded) when the span exceeds 32 cap columns.
template <int R>
__device__ __forceinline__ bool bitmap_ranks(int *keys, double *vals, int cnt, unsigned cap, int lane, int (&kk)[R],
                                             double (&vv)[R], int (&pos)[R]) {
    int mn = 0x7fffffff, mx = -1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = 32 * r + lane;
        kk[r] = e < cnt ? keys[e] : 0x7fffffff;
        vv[r] = e < cnt ? vals[e] : 0.0;
        if (e < cnt) {
            mn = min(mn, kk[r]);
            mx = max(mx, kk[r]);
        }
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (cnt == 0) return true;
    if ((long long)mx - mn >= 32ll * cap) return false;
    const int used = ((mx - mn) >> 5) + 1;
    unsigned *bm = reinterpret_cast<unsigned *>(vals + cap / 2);
    unsigned short *pre = reinterpret_cast<unsigned short *>(keys + cap / 2);
    __syncwarp();
    for (int w = lane; w < used; w += 32) bm[w] = 0u;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (32 * r + lane < cnt) {
            const int d = kk[r] - mn;
            atomicOr(&bm[d >> 5], 1u << (d & 31));
        }
    __syncwarp();
    int carry = 0;
    for (int base = 0; base < used; base += 32) {
        const int w = base + lane;
        const int c = w < used ? __popc(bm[w]) : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (w < used) pre[w] = (unsigned short)(carry + incl - c);
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        pos[r] = 0;
        if (32 * r + lane < cnt) {
            const int d = kk[r] - mn;
            pos[r] = pre[d >> 5] + __popc(bm[d >> 5] & ((1u << (d & 31)) - 1u));
        }
    }
    return true;
}

// write the compacted table [0, cnt) ordered by column: bitmap ranks for rows of up to 128 entries
// whose column span allows it, the bitonic network otherwise
template <int RMAX>
__device__ __forceinline__ void write_ordered(int *keys, double *vals, int cnt, unsigned cap, int *col, double *val,
                                              int lane) {
    if (cnt <= 128) {
        bool done = false;
        if (cnt <= 32) {
            int kk[1], pos[1];
            double vv[1];
            if ((done = bitmap_ranks<1>(keys, vals, cnt, cap, lane, kk, vv, pos)))
                if (lane < cnt) { col[pos[0]] = kk[0]; val[pos[0]] = vv[0]; }
        } else {
            int kk[4], pos[4];
            double vv[4];
            if ((done = bitmap_ranks<4>(keys, vals, cnt, cap, lane, kk, vv, pos))) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (32 * r + lane < cnt) { col[pos[r]] = kk[r]; val[pos[r]] = vv[r]; }
            }
        }
        if (done) return;
        __syncwarp();
    }
    write_sorted<RMAX>(keys, vals, cnt, col, val, lane);
}

// Fused (X Y) P for a one-point P. The cnt entries of row (X Y)_a, compacted in [0, cnt), are sorted
// by column j in registers; the table is cleared and entry (j, z) adds fma(z, p_j, .) to column
// P(j) in ascending j, 32 entries at a time, grouped by target column as in the product pass: the
// same sequence of fma as forming X Y and then (X Y) P. Returns the entry count of the result row,
// written sorted to col/val.
template <int R>
__device__ int fused_p_tail(const SpgemmArgs &g, int *keys, double *vals, unsigned cap, int cnt, double *px, double *py,
                            int *col, double *val, unsigned lane) {
    int k[R], lk[R];
    double v[R], pv[R];
    bool ranked = false;
    if (R <= 4) {
        int pos[R];
        ranked = bitmap_ranks<R>(keys, vals, cnt, cap, (int)lane, k, v, pos);
        if (ranked) {
            // permute in place through the registers, then read back in column order
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (32 * r + (int)lane < cnt) {
                    keys[pos[r]] = k[r];
                    vals[pos[r]] = v[r];
                }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int e = 32 * r + (int)lane;
                k[r] = e < cnt ? keys[e] : 0x7fffffff;
                v[r] = e < cnt ? vals[e] : 0.0;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = 32 * r + (int)lane;
            k[r] = e < cnt ? keys[e] : 0x7fffffff;
            v[r] = e < cnt ? vals[e] : 0.0;
        }
    }
    if (!ranked) warp_bitonic<R>(k, v, (int)lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        lk[r] = -1;
        pv[r] = 0.0;
        if (32 * r + (int)lane < cnt) {
            const int pb = g.prp[k[r]], pe = g.prp[k[r] + 1];
            if (pe > pb) {
                lk[r] = g.pcol[pb];
                pv[r] = g.pval[pb];
            }
        }
    }
    __syncwarp();
    for (unsigned e = lane; e < cap; e += 32) keys[e] = -1;
    __syncwarp();
    const unsigned mask = cap - 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (32 * r >= cnt) break;
        const bool act = lk[r] >= 0;
        if (act) {
            px[lane] = v[r];
            py[lane] = pv[r];
        }
        const unsigned am = __ballot_sync(0xffffffffu, act);
        __syncwarp();
        if (act) {
            const unsigned grp = __match_any_sync(am, lk[r]);
            if ((int)lane == __ffs(grp) - 1) hash_group_fma(keys, vals, mask, lk[r], grp, px, py);
        }
        __syncwarp();
    }
    const int cntk = compact_table(keys, vals, cap, lane);
    write_ordered<R>(keys, vals, cntk, cap, col, val, (int)lane);
    return cntk;
}

template <int CAP>
__host__ __device__ constexpr size_t spgemm_warp_bytes() { return (size_t)CAP * (sizeof(double) + sizeof(int)) + SPGEMM_EXTRA; }

// One warp per output row a with a hash table of CAP slots (rows with ub <= CAP / 2). The products
// x_ak * y_kl of the row are laid out flat in ascending (k, position in row k of Y) order and taken
// 32 at a time; lanes holding the same column l are grouped with __match_any_sync and the lowest lane
// of a group (the smallest k) applies the group's products in ascending k, so every entry receives its
// fma updates in ascending k exactly as in a sequential loop. The occupied slots are then compacted
// and ordered by column with a register bitonic network (rank counting for the largest rows).
template <int CAP, int WARPS, bool FUSE>
__global__ void __launch_bounds__(32 * WARPS, CAP == 256 ? 6 : 1) k_spgemm_warp(SpgemmArgs g, const int *__restrict__ list,
                                                           const int *__restrict__ count) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    unsigned char *mine = smem + (size_t)w * spgemm_warp_bytes<CAP>();
    double *vals = reinterpret_cast<double *>(mine);
    int *keys = reinterpret_cast<int *>(vals + CAP);
    double *sxv = reinterpret_cast<double *>(keys + CAP);      // CAP * 12 bytes: 16-aligned for CAP >= 4
    double *px = sxv + XCHUNK;
    double *py = px + 32;
    int *sy = reinterpret_cast<int *>(py + 32);                // first entry of row k of Y per staged k
    int *soff = sy + XCHUNK;
    const int n = *count;
    const int nwarps = gridDim.x * WARPS;
    for (int t = blockIdx.x * WARPS + w; t < n; t += nwarps) {
        const int a = list[t];
        const int ub = g.off[a + 1] - g.off[a];
        unsigned cap = 32;
        while ((int)cap < 2 * ub) cap <<= 1;
        const unsigned mask = cap - 1;
        for (unsigned e = lane; e < cap; e += 32) keys[e] = -1;
        const int xb = g.xrp[a], xe = g.xrp[a + 1];
        for (int c0 = xb; c0 < xe; c0 += XCHUNK) {
            const int cn = min(XCHUNK, xe - c0);
            __syncwarp();
            // stage k, x and flat offsets of this chunk (warp scan of the row lengths of Y)
            int carry = 0;
            for (int b = 0; b < cn; b += 32) {
                int len = 0;
                if (b + (int)lane < cn) {
                    const int k = g.xcol[c0 + b + lane];
                    const int y0 = g.yrp[k];
                    sy[b + lane] = y0;
                    sxv[b + lane] = g.xval[c0 + b + lane];
                    len = g.yrp[k + 1] - y0;
                }
                int incl = len;
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)lane >= o) incl += v;
                }
                if (b + (int)lane < cn) soff[b + lane] = carry + incl - len;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) soff[cn] = carry;
            __syncwarp();
            const int total = carry;
            // product p of the chunk: column, x and y value (the y loads of the next 32 products are
            // issued before the current ones are accumulated)
            auto fetch = [&](int p, int &l, double &xv, double &yv) {
                int lo = 0, hi = cn - 1;       // last chunk entry with soff <= p
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (soff[mid] <= p) lo = mid; else hi = mid - 1;
                }
                const int q = sy[lo] + (p - soff[lo]);
                xv = sxv[lo];
                l = g.ycol[q];
                yv = g.yval[q];
            };
            int l = -1;
            double xv = 0.0, yv = 0.0;
            if ((int)lane < total) fetch((int)lane, l, xv, yv);
            for (int base = 0; base < total; base += 32) {
                const bool act = base + (int)lane < total;
                int ln = -1;
                double xn = 0.0, yn = 0.0;
                if (base + 32 + (int)lane < total) fetch(base + 32 + (int)lane, ln, xn, yn);
                if (act) {
                    px[lane] = xv;
                    py[lane] = yv;
                }
                const unsigned am = __ballot_sync(0xffffffffu, act);
                __syncwarp();
                if (act) {
                    const unsigned grp = __match_any_sync(am, l);
                    if ((int)lane == __ffs(grp) - 1) hash_group_fma(keys, vals, mask, l, grp, px, py);
                }
                __syncwarp();
                l = ln;
                xv = xn;
                yv = yn;
            }
        }
        __syncwarp();
        const int o = g.off[a];
        int cnt = compact_table(keys, vals, cap, lane);
        constexpr int RMAX = CAP >= 1024 ? 16 : CAP / 64;
        if (FUSE) {
            // rows reach this kernel with cnt <= CAP / 2 <= 32 * RMAX only (the host fuses when every row does)
            if (cnt <= 32) cnt = fused_p_tail<1>(g, keys, vals, cap, cnt, px, py, g.tcol + o, g.tval + o, lane);
            else if (cnt <= 64) cnt = fused_p_tail<(RMAX >= 2 ? 2 : 1)>(g, keys, vals, cap, cnt, px, py, g.tcol + o, g.tval + o, lane);
            else if (cnt <= 128) cnt = fused_p_tail<(RMAX >= 4 ? 4 : 1)>(g, keys, vals, cap, cnt, px, py, g.tcol + o, g.tval + o, lane);
            else if (cnt <= 256) cnt = fused_p_tail<(RMAX >= 8 ? 8 : 1)>(g, keys, vals, cap, cnt, px, py, g.tcol + o, g.tval + o, lane);
            else cnt = fused_p_tail<(RMAX >= 16 ? 16 : 1)>(g, keys, vals, cap, cnt, px, py, g.tcol + o, g.tval + o, lane);
        } else if (cnt <= 32 * RMAX) {
            write_ordered<RMAX>(keys, vals, cnt, cap, g.tcol + o, g.tval + o, lane);
        } else {
            // rank counting: the position of a key is the number of smaller keys (keys are unique)
            for (int e = lane; e < cnt; e += 32) {
                const int key = keys[e];
                int r = 0;
                for (int f = 0; f < cnt; ++f) r += keys[f] < key;
                g.tcol[o + r] = key;
                g.tval[o + r] = vals[e];
            }
        }
        if (lane == 0) g.cnt[a] = cnt;
        __syncwarp();
    }
}

// long rows: one CTA per row, hash table and staging area in global scratch
__global__ void __launch_bounds__(256) k_spgemm_cta(SpgemmArgs g, const int *__restrict__ list, const int *__restrict__ count,
                                                   int *__restrict__ skeys, double *__restrict__ svals, unsigned cap) {
    __shared__ int cnt;
    const int n = *count;
    int *keys = skeys + (size_t)2 * cap * blockIdx.x;
    int *stk = keys + cap;
    double *vals = svals + (size_t)2 * cap * blockIdx.x;
    double *stv = vals + cap;
    const unsigned mask = cap - 1;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int a = list[t];
        for (unsigned e = threadIdx.x; e < cap; e += blockDim.x) keys[e] = -1;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        for (int p = g.xrp[a]; p < g.xrp[a + 1]; ++p) {
            const int k = g.xcol[p];
            const double x = g.xval[p];
            for (int q = g.yrp[k] + threadIdx.x; q < g.yrp[k + 1]; q += blockDim.x) {
                const int l = g.ycol[q];
                const double y = g.yval[q];
                unsigned h = hash_slot(l, mask);
                for (;;) {
                    int prev = atomicCAS(&keys[h], -1, l);
                    if (prev == -1) { vals[h] = __fma_rn(x, y, 0.0); break; }
                    if (prev == l) { vals[h] = __fma_rn(x, y, vals[h]); break; }
                    h = (h + 1) & mask;
                }
            }
            __syncthreads();
        }
        for (unsigned e = threadIdx.x; e < cap; e += blockDim.x) {
            int key = keys[e];
            if (key != -1) {
                int pos = atomicAdd(&cnt, 1);
                stk[pos] = key;
                stv[pos] = vals[e];
            }
        }
        __syncthreads();
        const int c = cnt;
        unsigned np2 = 1;
        while ((int)np2 < c) np2 <<= 1;
        for (unsigned e = c + threadIdx.x; e < np2; e += blockDim.x) stk[e] = 0x7fffffff;
        __syncthreads();
        for (unsigned kk = 2; kk <= np2; kk <<= 1)
            for (unsigned j = kk >> 1; j > 0; j >>= 1) {
                for (unsigned i = threadIdx.x; i < np2; i += blockDim.x) {
                    unsigned ixj = i ^ j;
                    if (ixj > i) {
                        bool up = (i & kk) == 0;
                        int ki = stk[i], kj = stk[ixj];
                        if ((ki > kj) == up) {
                            stk[i] = kj; stk[ixj] = ki;
                            double tv = stv[i]; stv[i] = stv[ixj]; stv[ixj] = tv;
                        }
                    }
                }
                __syncthreads();
            }
        const int o = g.off[a];
        for (int e = threadIdx.x; e < c; e += blockDim.x) {
            g.tcol[o + e] = stk[e];
            g.tval[o + e] = stv[e];
        }
        if (threadIdx.x == 0) g.cnt[a] = c;
        __syncthreads();
    }
}

__global__ void k_copy_rows(int nr, const int *__restrict__ off, const int *__restrict__ tcol, const double *__restrict__ tval,
                            const int *__restrict__ rp, int *__restrict__ col, double *__restrict__ val) {
    // one warp per row
    int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int a = wid; a < nr; a += nw) {
        int b = rp[a], e = rp[a + 1], o = off[a];
        for (int k = b + lane; k < e; k += 32) {
            col[k] = tcol[o + k - b];
            val[k] = tval[o + k - b];
        }
    }
}

void launch_spgemm_ub(int nr, const int *xrp, const int *xcol, const int *yrp, int *ub, cudaStream_t s) {
    k_spgemm_ub<<<grid_for(nr, 256), 256, 0, s>>>(nr, xrp, xcol, yrp, ub);
    count_launch();
}

void launch_spgemm_classify(int nr, const int *off, const int *xrp, bool merge, bool merge2, int merge_ub_max,
                            int *lists, int *counts, int *ubmax, cudaStream_t s) {
    k_spgemm_classify<<<grid_for(nr, 256), 256, 0, s>>>(nr, off, xrp, merge, merge2, merge_ub_max, lists, counts,
                                                        ubmax);
    count_launch();
}

template <int CAP, int WARPS, bool FUSE>
static void launch_spgemm_bin(const SpgemmArgs &g, const int *list, const int *count_dev, int count, cudaStream_t s) {
    const size_t bytes = (size_t)WARPS * spgemm_warp_bytes<CAP>();
    cudaFuncSetAttribute(k_spgemm_warp<CAP, WARPS, FUSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    int grid = grid_for(count, WARPS, device_sms() * 16);
    k_spgemm_warp<CAP, WARPS, FUSE><<<grid, 32 * WARPS, bytes, s>>>(g, list, count_dev);
    count_launch();
}

bool spgemm_can_fuse(const int counts_host[SPGEMM_BINS]) {
    return counts_host[2] == 0 && counts_host[SPGEMM_BIN_CTA] == 0 && counts_host[SPGEMM_BIN_MERGE2] == 0;
}

cudaError_t launch_spgemm_rows(const SpgemmArgs &g, int nr, const int *lists, const int *counts_dev,
                               const int counts_host[SPGEMM_BINS], int ubmax, int *skeys, double *svals, cudaStream_t s) {
    if (g.prp) {
        // fused one-point P: rows of the two short bins only (checked by spgemm_can_fuse)
        if (!spgemm_can_fuse(counts_host)) return cudaErrorInvalidValue;
        if (counts_host[0] > 0) launch_spgemm_bin<256, 8, true>(g, lists, counts_dev, counts_host[0], s);
        if (counts_host[1] > 0) launch_spgemm_bin<1024, 4, true>(g, lists + nr, counts_dev + 1, counts_host[1], s);
        if (counts_host[SPGEMM_BIN_MERGE] > 0) {
            if (!g.pmap_col || !g.pmap_val) return cudaErrorInvalidValue;
            k_p1_map<<<grid_for(g.pn, 256), 256, 0, s>>>(g.pn, g.prp, g.pcol, g.pval, g.pmap_col, g.pmap_val);
            k_spgemm_merge_p1<SPGEMM_MERGE_K>
                <<<grid_for(counts_host[SPGEMM_BIN_MERGE], SPGEMM_P1_THREADS, device_sms() * 8), SPGEMM_P1_THREADS, 0, s>>>(
                    g, lists + SPGEMM_BIN_MERGE * (size_t)nr, counts_dev + SPGEMM_BIN_MERGE, g.pmap_col, g.pmap_val);
            count_launch(2);
        }
        return cudaGetLastError();
    }
    if (counts_host[0] > 0) launch_spgemm_bin<256, 8, false>(g, lists, counts_dev, counts_host[0], s);
    if (counts_host[1] > 0) launch_spgemm_bin<1024, 4, false>(g, lists + nr, counts_dev + 1, counts_host[1], s);
    if (counts_host[2] > 0) launch_spgemm_bin<2048, 2, false>(g, lists + 2 * (size_t)nr, counts_dev + 2, counts_host[2], s);
    if (counts_host[SPGEMM_BIN_CTA] > 0) {
        unsigned cap = spgemm_big_cap(ubmax);
        int grid = counts_host[SPGEMM_BIN_CTA] < SPGEMM_CTA_GRID ? counts_host[SPGEMM_BIN_CTA] : SPGEMM_CTA_GRID;
        k_spgemm_cta<<<grid, 256, 0, s>>>(g, lists + SPGEMM_BIN_CTA * (size_t)nr, counts_dev + SPGEMM_BIN_CTA, skeys,
                                          svals, cap);
        count_launch();
    }
    if (counts_host[SPGEMM_BIN_MERGE] > 0) {
        k_spgemm_merge<SPGEMM_MERGE_K><<<grid_for(counts_host[SPGEMM_BIN_MERGE], 256, device_sms() * 16), 256, 0, s>>>(
            g, lists + SPGEMM_BIN_MERGE * (size_t)nr, counts_dev + SPGEMM_BIN_MERGE);
        count_launch();
    }
    if (counts_host[SPGEMM_BIN_MERGE2] > 0) {
        k_spgemm_merge<SPGEMM_MERGE_K2><<<grid_for(counts_host[SPGEMM_BIN_MERGE2], 128, device_sms() * 32), 128, 0, s>>>(
            g, lists + SPGEMM_BIN_MERGE2 * (size_t)nr, counts_dev + SPGEMM_BIN_MERGE2);
        count_launch();
    }
    return cudaGetLastError();
}

unsigned spgemm_big_cap(int ubmax) {
    unsigned cap = 32;
    while ((long long)cap < 2LL * ubmax) cap <<= 1;
    return cap;
}

void launch_copy_rows(int nr, const int *off, const int *tcol, const double *tval, DCsr &Z, cudaStream_t s) {
    k_copy_rows<<<grid_for((long long)nr * 32, 256), 256, 0, s>>>(nr, off, tcol, tval, Z.rp, Z.col, Z.val);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// lumping (Sec. 3.3): in row i drop every off-diagonal with |k_ij| < theta_D * max_j |k_ij|
// (max over the whole row) and add it to k_ii, in ascending j, starting from k_ii.
// ---------------------------------------------------------------------------------------
// Row i of K is col/val[rp[i], rp[i + 1]) or, when len is given, col/val[rp[i], rp[i] + len[i]) (the
// staging area of a product that was not compacted).
// Lumping (Sec. 3.3): entries with |k_ij| < tol * max_k |k_ik| off the diagonal are added to the diagonal in
// ascending column order starting from k_ii. Count: the row's maximum and diagonal in one pass, then the
// dropped sum and the kept count; the lumped diagonal and the threshold are kept per row (rowst[2 i], [2 i + 1])
// so that the fill reads the row once.
__global__ void k_lump_count(int n, const int *__restrict__ rp, const int *__restrict__ len, const int *__restrict__ col,
                             const double *__restrict__ val, double tol, int *__restrict__ cnt,
                             double2 *__restrict__ rowst, int *status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = rp[i], e = len ? b + len[i] : rp[i + 1];
        double m = 0.0, d = 0.0;
        bool has = false;
        for (int k0 = b; k0 < e; k0 += ROW_CHUNK) {
            int cc[ROW_CHUNK];
            double v[ROW_CHUNK];
#pragma unroll
            for (int u = 0; u < ROW_CHUNK; ++u) {
                cc[u] = k0 + u < e ? col[k0 + u] : -1;
                v[u] = k0 + u < e ? val[k0 + u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < ROW_CHUNK; ++u) {
                m = fmax(m, fabs(v[u]));
                if (cc[u] == i) {
                    d = v[u];
                    has = true;
                }
            }
        }
        if (!has) set_status(status, LAIR_ERR_ZERO_DIAGONAL);
        const double thr = __dmul_rn(tol, m);
        int c = 0;
        for (int k0 = b; k0 < e; k0 += ROW_CHUNK) {
            int cc[ROW_CHUNK];
            double v[ROW_CHUNK];
#pragma unroll
            for (int u = 0; u < ROW_CHUNK; ++u) {
                cc[u] = k0 + u < e ? col[k0 + u] : i;
                v[u] = k0 + u < e ? val[k0 + u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < ROW_CHUNK; ++u) {
                if (k0 + u >= e) break;
                if (cc[u] != i && fabs(v[u]) < thr) d = __dadd_rn(d, v[u]);
                else ++c;
            }
        }
        cnt[i] = c;
        rowst[i] = make_double2(d, thr);
    }
}

__global__ void k_lump_fill(int n, const int *__restrict__ rp, const int *__restrict__ len, const int *__restrict__ col,
                            const double *__restrict__ val, const double2 *__restrict__ rowst,
                            const int *__restrict__ orp, int *__restrict__ ocol, double *__restrict__ oval) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = rp[i], e = len ? b + len[i] : rp[i + 1];
        const double2 st = rowst[i];
        int p = orp[i];
        for (int k0 = b; k0 < e; k0 += ROW_CHUNK) {
            int cc[ROW_CHUNK];
            double v[ROW_CHUNK];
#pragma unroll
            for (int u = 0; u < ROW_CHUNK; ++u) {
                cc[u] = k0 + u < e ? col[k0 + u] : i;
                v[u] = k0 + u < e ? val[k0 + u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < ROW_CHUNK; ++u) {
                if (k0 + u >= e) break;
                if (cc[u] != i && fabs(v[u]) < st.y) continue;
                ocol[p] = cc[u];
                oval[p] = cc[u] == i ? st.x : v[u];
                ++p;
            }
        }
    }
}

void launch_lump(int phase, const DCsr &K, const int *len, double tol, int *cnt, double *rowst, const DCsr *out,
                 int *status, cudaStream_t s) {
    double2 *st = reinterpret_cast<double2 *>(rowst);
    if (phase == 0)
        k_lump_count<<<grid_for(K.nr, 256), 256, 0, s>>>(K.nr, K.rp, len, K.col, K.val, tol, cnt, st, status);
    else
        k_lump_fill<<<grid_for(K.nr, 256), 256, 0, s>>>(K.nr, K.rp, len, K.col, K.val, st, out->rp, out->col,
                                                         out->val);
    count_launch();
}

// Lumping onto a kept pattern (hierarchy refresh, Sec. 3.3): row i of the output keeps exactly its
// columns; every other entry of row i of K is added to the diagonal in ascending column order from
// k_ii (the order of k_lump_count when the dropped set is the same); kept entries take K's value.
// Both rows ascending; the kept row must be a subset of K's row that holds the diagonal.
__global__ void k_lump_kept(int n, const int *__restrict__ rp, const int *__restrict__ len, const int *__restrict__ col,
                            const double *__restrict__ val, const int *__restrict__ orp, const int *__restrict__ ocol,
                            double *__restrict__ oval, int *status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = rp[i], e = len ? b + len[i] : rp[i + 1];
        const int t0 = orp[i], t1 = orp[i + 1];
        double d = 0.0;
        for (int k = b; k < e; ++k)
            if (col[k] == i) d = val[k];
        int t = t0, dpos = -1;
        for (int k = b; k < e; ++k) {
            const int j = col[k];
            const bool kept = t < t1 && ocol[t] == j;
            if (kept) {
                if (j == i) dpos = t;
                else oval[t] = val[k];
                ++t;
            } else if (j != i) {
                d = __dadd_rn(d, val[k]);
            }
        }
        if (t != t1 || dpos < 0) set_status(status, t != t1 ? LAIR_ERR_INVALID_ARG : LAIR_ERR_ZERO_DIAGONAL);
        else oval[dpos] = d;
    }
}

void launch_lump_kept(const DCsr &K, const int *len, const DCsr &out, int *status, cudaStream_t s) {
    if (K.nr <= 0) return;
    k_lump_kept<<<grid_for(K.nr, 256), 256, 0, s>>>(K.nr, K.rp, len, K.col, K.val, out.rp, out.col, out.val, status);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// Jacobi diagonal inverse (1 / a_ii, IEEE division) and FP32 copies
// ---------------------------------------------------------------------------------------
__global__ void k_dinv(int n, const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val,
                       double *__restrict__ dinv, float *__restrict__ dinv32, int *status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] == i) d = val[k];
        if (d == 0.0) set_status(status, LAIR_ERR_ZERO_DIAGONAL);
        double r = __ddiv_rn(1.0, d);
        dinv[i] = r;
        if (dinv32) dinv32[i] = (float)r;
    }
}

__global__ void k_to_f32(long long n, const double *__restrict__ a, float *__restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

void launch_dinv(const DCsr &A, double *dinv, float *dinv32, int *status, cudaStream_t s) {
    k_dinv<<<grid_for(A.nr, 256), 256, 0, s>>>(A.nr, A.rp, A.col, A.val, dinv, dinv32, status);
    count_launch();
}

void launch_to_f32(long long n, const double *a, float *b, cudaStream_t s) {
    if (n <= 0) return;
    k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// coarsest level: dense LU with partial pivoting in one CTA, then the explicit inverse
// (one thread per column), so that the per-cycle coarse solve is a dense product.
// ---------------------------------------------------------------------------------------
__global__ void k_dense_build(int n, const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val,
                              double *__restrict__ D) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x)
        D[e] = 0.0;
}

__global__ void k_dense_scatter(int n, const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val,
                                double *__restrict__ D) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) D[(size_t)i * n + col[k]] = val[k];
}

__global__ void __launch_bounds__(1024) k_dense_lu(int n, double *__restrict__ D, int *__restrict__ perm, int *status) {
    __shared__ double bv[32];
    __shared__ int bi[32];
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int piv = -1;
        for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
            double v = fabs(D[(size_t)r * n + k]);
            if (piv < 0 || v > best) { best = v; piv = r; }
        }
        for (int o = 16; o >= 1; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, piv, o);
            if (oi >= 0 && (piv < 0 || ov > best || (ov == best && oi < piv))) { best = ov; piv = oi; }
        }
        if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = piv; }
        __syncthreads();
        best = bv[0];
        piv = bi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (bi[w] >= 0 && (piv < 0 || bv[w] > best || (bv[w] == best && bi[w] < piv))) { best = bv[w]; piv = bi[w]; }
        __syncthreads();
        if (best == 0.0) {
            if (threadIdx.x == 0) set_status(status, LAIR_ERR_ZERO_DIAGONAL);
            return;
        }
        if (piv != k) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                double t = D[(size_t)k * n + c];
                D[(size_t)k * n + c] = D[(size_t)piv * n + c];
                D[(size_t)piv * n + c] = t;
            }
            if (threadIdx.x == 0) { int t = perm[k]; perm[k] = perm[piv]; perm[piv] = t; }
        }
        __syncthreads();
        const double pk = D[(size_t)k * n + k];
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) D[(size_t)r * n + k] = D[(size_t)r * n + k] / pk;
        __syncthreads();
        const int w = n - k - 1;
        for (long long e = threadIdx.x; e < (long long)w * w; e += blockDim.x) {
            int r = k + 1 + (int)(e / w), c = k + 1 + (int)(e % w);
            D[(size_t)r * n + c] = fma(-D[(size_t)r * n + k], D[(size_t)k * n + c], D[(size_t)r * n + c]);
        }
        __syncthreads();
    }
}

// Ainv[:, t] = U^{-1} L^{-1} P e_t
__global__ void k_dense_inverse(int n, const double *__restrict__ LU, const int *__restrict__ perm, double *__restrict__ Ainv) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        for (int r = 0; r < n; ++r) Ainv[(size_t)r * n + t] = perm[r] == t ? 1.0 : 0.0;
        for (int k = 0; k < n; ++k) {
            double xk = Ainv[(size_t)k * n + t];
            if (xk == 0.0) continue;
            for (int r = k + 1; r < n; ++r) Ainv[(size_t)r * n + t] = fma(-LU[(size_t)r * n + k], xk, Ainv[(size_t)r * n + t]);
        }
        for (int c = n - 1; c >= 0; --c) {
            double xc = Ainv[(size_t)c * n + t] / LU[(size_t)c * n + c];
            Ainv[(size_t)c * n + t] = xc;
            for (int r = 0; r < c; ++r) Ainv[(size_t)r * n + t] = fma(-LU[(size_t)r * n + c], xc, Ainv[(size_t)r * n + t]);
        }
    }
}

// small coarsest levels (n <= DENSE_SMEM_N): the LU factorisation entirely in shared memory, one CTA, written
// out with its row permutation for k_dense_inv_cols
constexpr int DENSE_SMEM_N = 160;   // n^2 doubles + n ints: 205 KB of the 227 KB a CTA may have

__global__ void __launch_bounds__(256) k_dense_small(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                                      const double *__restrict__ val, double *__restrict__ LU,
                                                      int *__restrict__ perm_out, int *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *D = reinterpret_cast<double *>(smem);  // n x n
    int *perm = reinterpret_cast<int *>(D + (size_t)n * n);
    __shared__ double bv[32];
    __shared__ int bi[32];
    __shared__ int bad;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) D[e] = 0.0;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        perm[i] = i;
        for (int k = rp[i]; k < rp[i + 1]; ++k) D[i * n + col[k]] = val[k];
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int piv = -1;
        for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
            double v = fabs(D[r * n + k]);
            if (piv < 0 || v > best) { best = v; piv = r; }
        }
        for (int o = 16; o >= 1; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, piv, o);
            if (oi >= 0 && (piv < 0 || ov > best || (ov == best && oi < piv))) { best = ov; piv = oi; }
        }
        if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = piv; }
        __syncthreads();
        best = bv[0];
        piv = bi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (bi[w] >= 0 && (piv < 0 || bv[w] > best || (bv[w] == best && bi[w] < piv))) { best = bv[w]; piv = bi[w]; }
        if (best == 0.0) {
            if (threadIdx.x == 0) { set_status(status, LAIR_ERR_ZERO_DIAGONAL); bad = 1; }
            break;
        }
        if (piv != k) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                double t = D[k * n + c];
                D[k * n + c] = D[piv * n + c];
                D[piv * n + c] = t;
            }
            if (threadIdx.x == 0) { int t = perm[k]; perm[k] = perm[piv]; perm[piv] = t; }
        }
        __syncthreads();
        const double pk = D[k * n + k];
        for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) D[r * n + k] = D[r * n + k] / pk;
        __syncthreads();
        const int w = n - k - 1;
        for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
            int r = k + 1 + e / w, c = k + 1 + e % w;
            D[r * n + c] = fma(-D[r * n + k], D[k * n + c], D[r * n + c]);
        }
        __syncthreads();
    }
    __syncthreads();
    // a singular matrix leaves perm_out at -1, which k_dense_inv_cols reads as "skip"
    if (threadIdx.x == 0 && bad) perm_out[0] = -1;
    if (bad) return;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) LU[e] = D[e];
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm_out[i] = perm[i];
}

// columns of the inverse from the factors P A = L U: each warp owns DINV_COLS columns, DINV_ROWS lanes per
// column take the rows of every substitution step. The device's FP64 pipe serves whole warps, so this keeps
// the lanes full (a warp per column left most of them idle in the short steps, and a lane per division left 31
// of 32 idle) and spreads the columns over n / DINV_COLS SMs. Per element the operations and their order are
// those of the LU solve with e_t as right-hand side: forward x_r -= l_rk x_k, then x_c /= u_cc and
// x_r -= u_rc x_c for r < c.
constexpr int DINV_COLS = 4, DINV_ROWS = 32 / DINV_COLS;

__global__ void __launch_bounds__(32) k_dense_inv_cols(int n, const double *__restrict__ LU,
                                                       const int *__restrict__ perm, double *__restrict__ Ainv) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *x = reinterpret_cast<double *>(smem);  // n x DINV_COLS, row-major
    if (perm[0] < 0) return;
    const int lane = threadIdx.x, cg = lane / DINV_ROWS, rl = lane % DINV_ROWS;
    const int t = blockIdx.x * DINV_COLS + cg;
    for (int r = rl; r < n; r += DINV_ROWS) x[r * DINV_COLS + cg] = perm[r] == t ? 1.0 : 0.0;
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const double xk = x[k * DINV_COLS + cg];
        for (int r = k + 1 + rl; r < n; r += DINV_ROWS)
            x[r * DINV_COLS + cg] = fma(-LU[(size_t)r * n + k], xk, x[r * DINV_COLS + cg]);
        __syncwarp();
    }
    for (int c = n - 1; c >= 0; --c) {
        const double xc = x[c * DINV_COLS + cg] / LU[(size_t)c * n + c];
        __syncwarp();
        if (rl == 0) x[c * DINV_COLS + cg] = xc;
        for (int r = rl; r < c; r += DINV_ROWS) x[r * DINV_COLS + cg] = fma(-LU[(size_t)r * n + c], xc, x[r * DINV_COLS + cg]);
        __syncwarp();
    }
    if (t < n)
        for (int r = rl; r < n; r += DINV_ROWS) Ainv[(size_t)r * n + t] = x[r * DINV_COLS + cg];
}

bool dense_small(int n) { return n <= DENSE_SMEM_N; }

void launch_dense_setup(const DCsr &A, double *D, int *perm, double *Ainv, int *status, cudaStream_t s) {
    int n = A.nr;
    if (n <= 0) return;
    if (n <= DENSE_SMEM_N) {
        size_t bytes = sizeof(double) * (size_t)n * n + sizeof(int) * (size_t)n;
        cudaFuncSetAttribute(k_dense_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        // every column of the elimination costs a few block barriers: fewer warps make them cheaper, and a
        // coarsest level of a hundred unknowns has little work per column
        const int tb = n <= 64 ? 128 : 256;
        k_dense_small<<<1, tb, bytes, s>>>(n, A.rp, A.col, A.val, D, perm, status);
        k_dense_inv_cols<<<(n + DINV_COLS - 1) / DINV_COLS, 32, sizeof(double) * (size_t)n * DINV_COLS, s>>>(
            n, D, perm, Ainv);
        count_launch(2);
        return;
    }
    k_dense_build<<<grid_for((long long)n * n, 256), 256, 0, s>>>(n, A.rp, A.col, A.val, D);
    k_dense_scatter<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.col, A.val, D);
    k_dense_lu<<<1, 1024, 0, s>>>(n, D, perm, status);
    // the columns of the inverse over n / 4 CTAs (lanes full, as for small levels); a column per thread in the
    // fallback when the four columns' vectors do not fit in shared memory
    const size_t xb = sizeof(double) * (size_t)n * DINV_COLS;
    if (xb <= (size_t)200 * 1024 &&
        cudaFuncSetAttribute(k_dense_inv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xb) == cudaSuccess) {
        k_dense_inv_cols<<<(n + DINV_COLS - 1) / DINV_COLS, 32, xb, s>>>(n, D, perm, Ainv);
    } else {
        cudaGetLastError();
        k_dense_inverse<<<grid_for(n, 64), 64, 0, s>>>(n, D, perm, Ainv);
    }
    count_launch(4);
}

}  // namespace lair
