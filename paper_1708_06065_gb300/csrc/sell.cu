// sell.cu -- sliced-ELL copies of the cycle's matrices and the kernels that stream them.
//
// A view holds a subset of a matrix's rows (all rows, or only the F rows or only the C rows of
// a level) in slices of 32 rows. Inside a slice, entry j of the slice's r-th row sits at
// slice_ptr[s] + 32 j + r, so one thread owns one row and the 32 threads of a warp read 32
// consecutive values and column indices per step: every load is coalesced and a thread keeps
// several independent loads in flight. Rows are ordered by decreasing length inside windows of
// 256 rows to keep the padding of a slice small; row[] maps a view row back to its matrix row.
// The sweeps of a level then read only the rows they update (F rows, or C rows).
#include "setup_kernels.cuh"

#include <climits>

namespace lair {

constexpr int SELL_WINDOW = 256;

// F rows in ascending order from the exclusive scan of the C flags: F point i has F index i - scan[i]
__global__ void k_frows(int n, const int8_t *__restrict__ cf, const int *__restrict__ cscan, int *__restrict__ frows) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (cf[i] != CF_C) frows[i - cscan[i]] = i;
}

// ---------------------------------------------------------------------------------------
// Building many views at once. Views are described by SellDesc entries; view p owns windows
// [win0, win0 + its windows), linear slices [lin0, lin0 + its slices) and, in the slice-length
// array cnt, positions [sl0, sl0 + its slices). Every kernel finds the view of its window or
// slice by binary search over the descriptors.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int find_desc(const SellDesc *__restrict__ d, int nd, int key, int which) {
    int lo = 0, hi = nd - 1;     // last descriptor whose start <= key
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int st = which == 0 ? d[mid].win0 : d[mid].lin0;
        if (st <= key) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Ascending bitonic sort of 32 R distinct keys held by a warp, element e = 32 r + lane in key[r]: exchanges at
// distance < 32 through shuffles, the others inside a lane's registers (compile-time indices only).
template <int R>
__device__ __forceinline__ void warp_sort_keys(unsigned (&key)[R], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int r2 = r ^ (j >> 5);
                    if (r2 > r) {
                        const bool up = ((32 * r + lane) & k) == 0;
                        if (up ? key[r] > key[r2] : key[r] < key[r2]) {
                            const unsigned t = key[r];
                            key[r] = key[r2];
                            key[r2] = t;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const unsigned pk = __shfl_xor_sync(0xffffffffu, key[r], j);
                    const bool up = ((32 * r + lane) & k) == 0, lower = (lane & j) == 0;
                    if (lower == up ? pk < key[r] : pk > key[r]) key[r] = pk;
                }
            }
        }
    }
}

constexpr int SORT_WARPS = 8;                 // windows in flight per CTA (one per warp)
constexpr int SELL_RPL = SELL_WINDOW / 32;    // rows of a window per lane
constexpr int SELL_COUNT_SORT = 16;           // windows with fewer distinct lengths than this: counting sort

// Order the rows of every window by decreasing length (ties: window position), one warp per window: row t of
// the window is lane t % 32's entry t / 32, so the loads of a window are coalesced and every lane has eight
// independent row lengths in flight. A window already in non-increasing order (the interior of a stencil)
// is written as it is, one with a narrow range of lengths goes through a counting sort by length, the others
// through a register bitonic sort of (length, position) keys.
__global__ void __launch_bounds__(32 * SORT_WARPS) k_sell_sort_multi(const SellDesc *__restrict__ d, int nd,
                                                                     int nwin) {
    __shared__ int stage[SORT_WARPS][SELL_WINDOW];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    for (int w = blockIdx.x * SORT_WARPS + wq; w < nwin; w += gridDim.x * SORT_WARPS) {
        const int p = find_desc(d, nd, w, 0);
        const int *rows_in = d[p].rows_in, *rp = d[p].rp;
        int *row_out = d[p].row_out;
        const int w0 = (w - d[p].win0) * SELL_WINDOW;
        const int cnt = min(SELL_WINDOW, d[p].nrows - w0);
        int rid[SELL_RPL], len[SELL_RPL];
#pragma unroll
        for (int k = 0; k < SELL_RPL; ++k) {
            const int t = 32 * k + lane;
            rid[k] = t < cnt ? (rows_in ? rows_in[w0 + t] : w0 + t) : -1;
        }
#pragma unroll
        for (int k = 0; k < SELL_RPL; ++k) len[k] = rid[k] >= 0 ? rp[rid[k] + 1] - rp[rid[k]] : -1;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < SELL_RPL; ++k) {
            const int down = __shfl_down_sync(0xffffffffu, len[k], 1);
            const int wrap = __shfl_sync(0xffffffffu, k + 1 < SELL_RPL ? len[k + 1 < SELL_RPL ? k + 1 : k] : 0, 0);
            const int next = lane < 31 ? down : (k + 1 < SELL_RPL ? wrap : -1);
            if (32 * k + lane + 1 < cnt && len[k] < next) ok = false;
        }
        if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
            for (int k = 0; k < SELL_RPL; ++k)
                if (32 * k + lane < cnt) row_out[w0 + 32 * k + lane] = rid[k];
            continue;
        }
        // few distinct lengths (a stencil's boundary rows): a counting sort, longest first, window order inside
        // a length -- the same order as the stable sort, at one ballot per length and row register
        int lo = INT_MAX, hi = -1;
#pragma unroll
        for (int k = 0; k < SELL_RPL; ++k)
            if (len[k] >= 0) {
                lo = min(lo, len[k]);
                hi = max(hi, len[k]);
            }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (hi - lo < SELL_COUNT_SORT) {
            const unsigned below = (1u << lane) - 1u;
            int pos[SELL_RPL];
            int base = 0;
            for (int v = hi; v >= lo; --v) {
#pragma unroll
                for (int k = 0; k < SELL_RPL; ++k) {
                    const unsigned m = __ballot_sync(0xffffffffu, len[k] == v);
                    if (len[k] == v) pos[k] = base + __popc(m & below);
                    base += __popc(m);
                }
            }
#pragma unroll
            for (int k = 0; k < SELL_RPL; ++k)
                if (len[k] >= 0) row_out[w0 + pos[k]] = rid[k];
            continue;
        }
        // keys: (2^23 - 1 - length) in the high bits, the window position in the low 8; padding last
        unsigned key[SELL_RPL];
#pragma unroll
        for (int k = 0; k < SELL_RPL; ++k) {
            const int t = 32 * k + lane;
            stage[wq][t] = rid[k];
            key[k] = t < cnt ? ((unsigned)(0x7fffff - min(len[k], 0x7fffff)) << 8) | (unsigned)t : 0xffffffffu;
        }
        __syncwarp();
        warp_sort_keys<SELL_RPL>(key, lane);
#pragma unroll
        for (int k = 0; k < SELL_RPL; ++k)
            if (32 * k + lane < cnt) row_out[w0 + 32 * k + lane] = stage[wq][key[k] & 0xffu];
        __syncwarp();
    }
}

// batched systems: the system of row i (the last q with seg[q] <= i)
__device__ __forceinline__ int system_of(const int *__restrict__ seg, int nseg, int i) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// slice lengths in entries (32 x longest row of the slice), one warp per slice; also their
// 64-bit sum per group (two groups: FP32 and FP64 views), so that an int overflow of the offsets is caught on
// the host. Each warp adds its own sums once at the end.
__global__ void k_sell_len_multi(const SellDesc *__restrict__ d, int nd, int nlin, int *__restrict__ cnt,
                                 unsigned long long *__restrict__ gsum) {
    const int lane = threadIdx.x & 31;
    unsigned long long s0 = 0, s1 = 0;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nlin; q += (gridDim.x * blockDim.x) >> 5) {
        const int p = find_desc(d, nd, q, 1);
        const SellDesc &v = d[p];
        const int sl = q - v.lin0;
        const int r = sl * 32 + lane;
        int l = 0, sy = -2;
        if (r < v.nrows) {
            const int i = v.row_out[r];
            l = v.rp[i + 1] - v.rp[i];
            if (v.nseg > 0) sy = system_of(v.seg, v.nseg, i);
        }
        l = __reduce_max_sync(0xffffffffu, l);
        if (v.nseg > 0) {
            // the slice's system when all its rows share one (lane 0 always holds a row)
            const int sy0 = __shfl_sync(0xffffffffu, sy, 0);
            const bool one = __all_sync(0xffffffffu, sy == -2 || sy == sy0);
            if (lane == 0) v.slice_sys[sl] = one ? sy0 : -1;
        }
        if (lane == 0) {
            cnt[v.sl0 + sl] = 32 * l;
            if (v.group == 0) s0 += 32ull * (unsigned long long)l;
            else s1 += 32ull * (unsigned long long)l;
        }
    }
    if (lane == 0) {
        if (s0) atomicAdd(&gsum[0], s0);
        if (s1) atomicAdd(&gsum[1], s1);
    }
}

// entries of the views [p0, p1) (one element type), one thread per row slot of a slice
template <class T>
__global__ void k_sell_fill_multi(const SellDesc *__restrict__ d, int p0, int p1, int lin_end) {
    const int lin_beg = d[p0].lin0;
    const long long nslot = 32ll * (lin_end - lin_beg);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nslot; e += (long long)gridDim.x * blockDim.x) {
        const int q = lin_beg + (int)(e >> 5), lane = (int)(e & 31);
        const int p = p0 + find_desc(d + p0, p1 - p0, q, 1);
        const SellDesc &v = d[p];
        const int sl = q - v.lin0;
        const int *sptr = v.slice_ptr;
        const int base = sptr[sl] + lane, len = (sptr[sl + 1] - sptr[sl]) >> 5;
        const int r = sl * 32 + lane;
        // padding entries carry value 0 and a column that is valid for x: the row's last column
        // (a row index is not one when the matrix is rectangular, as P and R are)
        int b = 0, en = 0, pad = 0;
        if (r < v.nrows) {
            const int i = v.row_out[r];
            b = v.rp[i];
            en = v.rp[i + 1];
            pad = en > b ? v.col[en - 1] : 0;
            if (v.sdinv) static_cast<T *>(v.sdinv)[r] = (T)v.dinv[i];
        }
        int *scol = v.scol;
        T *sval = static_cast<T *>(v.sval);
        for (int j = 0; j < len; ++j) {
            const bool in = b + j < en;
            scol[base + 32 * j] = in ? v.col[b + j] : pad;
            sval[base + 32 * j] = in ? (T)v.val[b + j] : T(0);
        }
    }
}

// The matrix entries, the Jacobi diagonal and b are read once per launch: they are loaded with the
// streaming (evict-first) policy, so that they pass through L2 without pushing out x, which every row
// gathers from and which stays in L2 from one kernel of the cycle to the next.
//
// y[row[r]] = (view row r) . x. RPT rows per thread: the thread of lane l in group g takes row l of each of
// the slices g RPT, ..., g RPT + RPT - 1, so every load of a warp stays coalesced and a thread keeps RPT
// independent sums in flight; each row is still summed alone in column order.
template <class T, int RPT>
__global__ void __launch_bounds__(256) k_sell_spmv(SellView v, const T *__restrict__ x, T *__restrict__ y) {
    pdl_enter();
    const int *__restrict__ sptr = v.slice_ptr;
    const int *__restrict__ scol = v.col;
    const T *__restrict__ sval = static_cast<const T *>(v.val);
    const int nsl = (v.nrows + 31) >> 5;
    const long long nthr = (long long)((nsl + RPT - 1) / RPT) * 32;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nthr; u += (long long)gridDim.x * blockDim.x) {
        const int lane = (int)(u & 31), s0 = (int)(u >> 5) * RPT;
        int base[RPT], len[RPT], r[RPT];
        int lmax = 0;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            bool on = s0 + k < nsl, zero = false;
            if (on && v.run) {
                const int q = v.slice_sys[s0 + k];
                on = q < 0 || v.run[q];
                zero = !on && v.zero_stopped;   // no entries: the row's sum stays 0 and is written
            }
            r[k] = on || zero ? (s0 + k) * 32 + lane : v.nrows;
            base[k] = 0;
            len[k] = 0;
            if (on) {
                const int a = __ldg(sptr + s0 + k);
                base[k] = a + lane;
                len[k] = (__ldg(sptr + s0 + k + 1) - a) >> 5;
            }
            lmax = max(lmax, len[k]);
        }
        T acc[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) acc[k] = T(0);
#pragma unroll 4
        for (int j = 0; j < lmax; ++j)
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (j < len[k])
                    acc[k] = fma(__ldcs(sval + base[k] + 32 * j), __ldg(x + __ldcs(scol + base[k] + 32 * j)), acc[k]);
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (r[k] < v.nrows) y[v.row[r[k]]] = acc[k];
    }
}

// one Jacobi sweep over the view's rows (x_i + d_i (b_i - A_i x)), RPT rows per thread as above; then the
// entries of the other rows (copy[], ncopy of them) are copied from x to xo, one per thread
template <class T, int RPT>
__global__ void __launch_bounds__(256) k_sell_sweep(SellView v, const int *__restrict__ copy, int ncopy,
                                                    const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ xo) {
    pdl_enter();
    const int *__restrict__ sptr = v.slice_ptr;
    const int *__restrict__ scol = v.col;
    const T *__restrict__ sval = static_cast<const T *>(v.val);
    const T *__restrict__ sd = static_cast<const T *>(v.dinv);
    const int nsl = (v.nrows + 31) >> 5;
    const long long nthr = (long long)((nsl + RPT - 1) / RPT) * 32;
    const long long total = nthr + ncopy;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total; u += (long long)gridDim.x * blockDim.x) {
        if (u < nthr) {
            const int lane = (int)(u & 31), s0 = (int)(u >> 5) * RPT;
            int base[RPT], len[RPT], r[RPT];
            int lmax = 0;
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                bool on = s0 + k < nsl;
                if (on && v.run) {
                    const int q = v.slice_sys[s0 + k];
                    on = q < 0 || v.run[q];
                }
                r[k] = on ? (s0 + k) * 32 + lane : v.nrows;
                base[k] = 0;
                len[k] = 0;
                if (on) {
                    const int a = __ldg(sptr + s0 + k);
                    base[k] = a + lane;
                    len[k] = (__ldg(sptr + s0 + k + 1) - a) >> 5;
                }
                lmax = max(lmax, len[k]);
            }
            T acc[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) acc[k] = T(0);
#pragma unroll 4
            for (int j = 0; j < lmax; ++j)
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                    if (j < len[k])
                        acc[k] = fma(__ldcs(sval + base[k] + 32 * j), __ldg(x + __ldcs(scol + base[k] + 32 * j)), acc[k]);
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (r[k] < v.nrows) {
                    const int i = v.row[r[k]];
                    xo[i] = fma(__ldcs(sd + r[k]), __ldcs(b + i) - acc[k], x[i]);
                }
        } else {
            const int j = copy[u - nthr];
            xo[j] = x[j];
        }
    }
}

// One-point interpolation (one-point P, or the identity blocks of the nodal hierarchy: at most one entry per
// row, every entry 1): x_i = x_c[col_i] + 0, or 0 for a row without an entry -- the bits of fma(1, x_c[col_i], 0)
// that the sliced-ELL product gives (a -0 becomes +0). One column per row from the dense column array, one
// gather, one write: coalesced everywhere but the gather.
template <class T>
__global__ void __launch_bounds__(256) k_p1_interp(int n, const int *__restrict__ p1col, const int *__restrict__ blk_sys,
                                                   const uint8_t *run, const T *__restrict__ xc, T *__restrict__ x) {
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (run) {
            const int q = blk_sys[i >> 5];
            if (q >= 0 && !run[q]) continue;
        }
        const int c = __ldcs(p1col + i);
        x[i] = c >= 0 ? __ldg(xc + c) + T(0) : T(0);
    }
}

template <class T>
void p1_interp(int n, const int *p1col, const int *blk_sys, const uint8_t *run, const T *xc, T *x, cudaStream_t s) {
    if (n <= 0) return;
    launch_pdl(k_p1_interp<T>, grid_for(n, 256, device_sms() * 16), 256, 0, s, n, p1col, blk_sys, run, xc, x);
    count_launch();
}
template void p1_interp<float>(int, const int *, const int *, const uint8_t *, const float *, float *, cudaStream_t);
template void p1_interp<double>(int, const int *, const int *, const uint8_t *, const double *, double *,
                                cudaStream_t);

// ---------------------------------------------------------------------------------------
// The bottom of the V-cycle in one CTA: the restrictions of the smallest levels, the coarsest solve, and on the
// way up their interpolations and F/C sweeps, with a block barrier between phases instead of a kernel boundary.
// Every row is computed by one thread with the arithmetic of k_sell_spmv, k_sell_sweep, k_p1_interp and
// k_dense_apply (same entries, same order), so the cycle's result is the same bits either way. Vectors written
// in one phase and read in a later one are read with plain loads (the block's own writes, ordered by
// __syncthreads); matrices do not change during the launch. Stopped batched systems are not skipped here.
// ---------------------------------------------------------------------------------------
namespace {

template <class T>
__device__ __forceinline__ void bottom_spmv(const SellView &v, const T *x, T *y) {
    const T *__restrict__ sval = static_cast<const T *>(v.val);
    const long long nthr = (long long)((v.nrows + 31) >> 5) * 32;
    for (long long u = threadIdx.x; u < nthr; u += blockDim.x) {
        const int lane = (int)(u & 31), sl = (int)(u >> 5), r = sl * 32 + lane;
        const int a = __ldg(v.slice_ptr + sl);
        const int base = a + lane, len = (__ldg(v.slice_ptr + sl + 1) - a) >> 5;
        T acc = T(0);
        for (int j = 0; j < len; ++j) acc = fma(__ldg(sval + base + 32 * j), x[__ldg(v.col + base + 32 * j)], acc);
        if (r < v.nrows) y[__ldg(v.row + r)] = acc;
    }
}

template <class T>
__device__ __forceinline__ void bottom_sweep(const SellView &v, const int *copy, int ncopy, const T *b, const T *x,
                                             T *xo) {
    const T *__restrict__ sval = static_cast<const T *>(v.val);
    const T *__restrict__ sd = static_cast<const T *>(v.dinv);
    const long long nthr = (long long)((v.nrows + 31) >> 5) * 32;
    for (long long u = threadIdx.x; u < nthr + ncopy; u += blockDim.x) {
        if (u < nthr) {
            const int lane = (int)(u & 31), sl = (int)(u >> 5), r = sl * 32 + lane;
            const int a = __ldg(v.slice_ptr + sl);
            const int base = a + lane, len = (__ldg(v.slice_ptr + sl + 1) - a) >> 5;
            T acc = T(0);
            for (int j = 0; j < len; ++j) acc = fma(__ldg(sval + base + 32 * j), x[__ldg(v.col + base + 32 * j)], acc);
            if (r < v.nrows) {
                const int i = __ldg(v.row + r);
                xo[i] = fma(__ldg(sd + r), b[i] - acc, x[i]);
            }
        } else {
            const int j = __ldg(copy + (u - nthr));
            xo[j] = x[j];
        }
    }
}

}  // namespace

template <class T>
__global__ void __launch_bounds__(BOTTOM_THREADS) k_cycle_bottom(const BottomLevel<T> *__restrict__ lv, int nl,
                                                                 BottomCoarse<T> cz, int4 seq) {
    pdl_enter();
    const int sq[3] = {seq.x, seq.y, seq.z};
    for (int l = 0; l < nl; ++l) {
        bottom_spmv<T>(lv[l].R, lv[l].b, l + 1 < nl ? lv[l + 1].b : cz.b);
        __syncthreads();
    }
    {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r = threadIdx.x >> 5; r < cz.n; r += nw) {
            double acc = 0.0;
            for (int c = lane; c < cz.n; c += 32) acc = fma(__ldg(cz.Ainv + (size_t)r * cz.n + c), (double)cz.b[c], acc);
            acc = warp_sum(acc);
            if (lane == 0) cz.x[r] = (T)acc;
        }
    }
    for (int l = nl - 1; l >= 0; --l) {
        const BottomLevel<T> &L = lv[l];
        __syncthreads();
        const T *xc = l + 1 < nl ? lv[l + 1].x[seq.w] : cz.x;
        if (L.p1col) {
            for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
                const int c = __ldg(L.p1col + i);
                L.x[0][i] = c >= 0 ? xc[c] + T(0) : T(0);
            }
        } else {
            bottom_spmv<T>(L.P, xc, L.x[0]);
        }
        int cur = 0;
        for (int k = 0; k < 3 && sq[k] >= 0; ++k) {
            __syncthreads();
            if (sq[k] == CF_F) bottom_sweep<T>(L.AF, L.crows, L.nc, L.b, L.x[cur], L.x[1 - cur]);
            else bottom_sweep<T>(L.AC, L.frows, L.n - L.nc, L.b, L.x[cur], L.x[1 - cur]);
            cur ^= 1;
        }
    }
}

template <class T>
void cycle_bottom(const BottomLevel<T> *lv, int nl, const BottomCoarse<T> &cz, const int *seq3, cudaStream_t s) {
    int nsw = 0;
    while (nsw < 3 && seq3[nsw] >= 0) ++nsw;
    const int4 seq = make_int4(seq3[0], seq3[1], seq3[2], nsw & 1);
    launch_pdl(k_cycle_bottom<T>, 1, BOTTOM_THREADS, 0, s, lv, nl, cz, seq);
    count_launch();
}
template void cycle_bottom<float>(const BottomLevel<float> *, int, const BottomCoarse<float> &, const int *,
                                  cudaStream_t);
template void cycle_bottom<double>(const BottomLevel<double> *, int, const BottomCoarse<double> &, const int *,
                                   cudaStream_t);

// the system of every 32-row block: that of its first row when its last row has the same one, else -1
__global__ void k_blk_sys(int n, const int *__restrict__ seg, int nseg, int *__restrict__ blk_sys) {
    const int nb = (n + 31) >> 5;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int q0 = system_of(seg, nseg, 32 * b), q1 = system_of(seg, nseg, min(32 * b + 31, n - 1));
        blk_sys[b] = q0 == q1 ? q0 : -1;
    }
}

void launch_blk_sys(int n, const int *seg, int nseg, int *blk_sys, cudaStream_t s) {
    if (n <= 0) return;
    k_blk_sys<<<grid_for((n + 31) / 32, 256), 256, 0, s>>>(n, seg, nseg, blk_sys);
    count_launch();
}

// the dense column array of a P with at most one entry per row
__global__ void k_p1_cols(int n, const int *__restrict__ rp, const int *__restrict__ col, int *__restrict__ p1col) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p1col[i] = rp[i + 1] > rp[i] ? col[rp[i]] : -1;
}

void launch_p1_cols(int n, const int *rp, const int *col, int *p1col, cudaStream_t s) {
    if (n <= 0) return;
    k_p1_cols<<<grid_for(n, 256), 256, 0, s>>>(n, rp, col, p1col);
    count_launch();
}

// r = b - A x over all rows of an FP64 view of A (r and its FP32 copy each optional), and the block partial
// of |r|^2 in part[blockIdx.x] (gridDim.x = RED_PARTS blocks, summed by finish_partials)
constexpr int RES_THREADS = 512;

__global__ void __launch_bounds__(RES_THREADS) k_sell_residual(SellView v, const double *__restrict__ b,
                                                               const double *__restrict__ x, double *__restrict__ r,
                                                               float *__restrict__ r32, double *__restrict__ part) {
    __shared__ double red[RES_THREADS / 32];
    const int *__restrict__ sptr = v.slice_ptr;
    const int *__restrict__ scol = v.col;
    const double *__restrict__ sval = static_cast<const double *>(v.val);
    double ss = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < v.nrows; q += gridDim.x * blockDim.x) {
        const int sl = q >> 5;
        const int base = __ldg(sptr + sl) + (q & 31);
        const int len = (__ldg(sptr + sl + 1) - __ldg(sptr + sl)) >> 5;
        double acc = 0.0;
#pragma unroll 4
        for (int j = 0; j < len; ++j) acc = fma(__ldcs(sval + base + 32 * j), __ldg(x + __ldcs(scol + base + 32 * j)), acc);
        const int i = v.row[q];
        const double ri = b[i] - acc;
        if (r) r[i] = ri;
        if (r32) r32[i] = (float)ri;
        ss = fma(ri, ri, ss);
    }
    for (int o = 16; o >= 1; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RES_THREADS / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

void sell_residual(const SellView &v, const double *b, const double *x, double *r, float *r32, double *part,
                   cudaStream_t s) {
    k_sell_residual<<<RED_PARTS, RES_THREADS, 0, s>>>(v, b, x, r, r32, part);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
void launch_frows(int n, const int8_t *cf, const int *cscan, int *frows, cudaStream_t s) {
    k_frows<<<grid_for(n, 256), 256, 0, s>>>(n, cf, cscan, frows);
    count_launch();
}

void launch_sell_prepare_multi(const SellDesc *d, int nd, int nwin, int nlin, int *cnt, unsigned long long *gsum,
                               cudaStream_t s) {
    if (nwin <= 0) return;
    k_sell_sort_multi<<<grid_for((long long)nwin, SORT_WARPS, device_sms() * 16), 32 * SORT_WARPS, 0, s>>>(d, nd, nwin);
    k_sell_len_multi<<<grid_for((long long)nlin * 32, 256), 256, 0, s>>>(d, nd, nlin, cnt, gsum);
    count_launch(2);
}

void launch_sell_fill_multi(const SellDesc *d, int p0, int p1, int lin_beg, int lin_end, bool fp32, cudaStream_t s) {
    if (p1 <= p0 || lin_end <= lin_beg) return;
    const int grid = grid_for(32ll * (lin_end - lin_beg), 256);
    if (fp32) k_sell_fill_multi<float><<<grid, 256, 0, s>>>(d, p0, p1, lin_end);
    else k_sell_fill_multi<double><<<grid, 256, 0, s>>>(d, p0, p1, lin_end);
    count_launch();
}

template <class T>
void sell_spmv(const SellView &v, const T *x, T *y, cudaStream_t s) {
    if (v.nrows <= 0) return;
    // every row is summed alone by one thread, so the schedule (block size, grid cap, rows per thread) never
    // changes the result
    const int tb = v.tb > 0 ? v.tb : 256;
    const int cap = v.grid > 0 ? v.grid : device_sms() * 16;
    const long long nsl = (v.nrows + 31) / 32;
    if (v.rpt == 2) launch_pdl(k_sell_spmv<T, 2>, grid_for((nsl + 1) / 2 * 32, tb, cap), tb, 0, s, v, x, y);
    else launch_pdl(k_sell_spmv<T, 1>, grid_for(nsl * 32, tb, cap), tb, 0, s, v, x, y);
    count_launch();
}

template <class T>
void sell_sweep(const SellView &v, const int *copy, int ncopy, const T *b, const T *x, T *xo, cudaStream_t s) {
    if (v.nrows + ncopy <= 0) return;
    const int tb = v.tb > 0 ? v.tb : 256;
    const int cap = v.grid > 0 ? v.grid : device_sms() * 16;
    const long long nsl = (v.nrows + 31) / 32;
    if (v.rpt == 2)
        launch_pdl(k_sell_sweep<T, 2>, grid_for((nsl + 1) / 2 * 32 + ncopy, tb, cap), tb, 0, s, v, copy, ncopy, b, x, xo);
    else
        launch_pdl(k_sell_sweep<T, 1>, grid_for(nsl * 32 + ncopy, tb, cap), tb, 0, s, v, copy, ncopy, b, x, xo);
    count_launch();
}

template void sell_spmv<float>(const SellView &, const float *, float *, cudaStream_t);
template void sell_spmv<double>(const SellView &, const double *, double *, cudaStream_t);
template void sell_sweep<float>(const SellView &, const int *, int, const float *, const float *, float *, cudaStream_t);
template void sell_sweep<double>(const SellView &, const int *, int, const double *, const double *, double *,
                                 cudaStream_t);

}  // namespace lair
