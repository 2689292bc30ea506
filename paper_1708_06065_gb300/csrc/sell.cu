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

namespace lair {

constexpr int SELL_WINDOW = 256;

// F rows in ascending order from the exclusive scan of the C flags: F point i has F index i - scan[i]
__global__ void k_frows(int n, const int8_t *__restrict__ cf, const int *__restrict__ cscan, int *__restrict__ frows) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (cf[i] != CF_C) frows[i - cscan[i]] = i;
}

// one CTA per window: order the window's rows by decreasing length (stable)
__global__ void __launch_bounds__(SELL_WINDOW) k_sell_sort(int nrows, const int *__restrict__ rows_in,
                                                          const int *__restrict__ rp, int *__restrict__ rows_out) {
    __shared__ int len[SELL_WINDOW];
    __shared__ int rid[SELL_WINDOW];
    const int w0 = blockIdx.x * SELL_WINDOW;
    const int t = threadIdx.x;
    const int cnt = min(SELL_WINDOW, nrows - w0);
    if (t < cnt) {
        const int i = rows_in ? rows_in[w0 + t] : w0 + t;
        rid[t] = i;
        len[t] = rp[i + 1] - rp[i];
    }
    __syncthreads();
    if (t < cnt) {
        const int lt = len[t];
        int r = 0;
        for (int u = 0; u < cnt; ++u) r += (len[u] > lt) || (len[u] == lt && u < t);
        rows_out[w0 + r] = rid[t];
    }
}

// slice lengths (in entries: 32 x longest row of the slice); cnt has nslices + 1 entries
__global__ void k_sell_len(int nrows, const int *__restrict__ rows, const int *__restrict__ rp, int *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int nsl = (nrows + 31) / 32;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nsl; s += (gridDim.x * blockDim.x) >> 5) {
        const int r = s * 32 + lane;
        int l = 0;
        if (r < nrows) {
            const int i = rows[r];
            l = rp[i + 1] - rp[i];
        }
        l = __reduce_max_sync(0xffffffffu, l);
        if (lane == 0) cnt[s] = 32 * l;
    }
}

template <class T>
__global__ void k_sell_fill(int nrows, const int *__restrict__ rows, const int *__restrict__ rp, const int *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ dinv, const int *__restrict__ sptr,
                            int *__restrict__ scol, T *__restrict__ sval, T *__restrict__ sdinv) {
    const int nsl = (nrows + 31) / 32;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nsl * 32; r += gridDim.x * blockDim.x) {
        const int s = r >> 5, lane = r & 31;
        const int base = sptr[s] + lane, len = (sptr[s + 1] - sptr[s]) >> 5;
        // padding entries carry value 0 and a column that is valid for x: the row's last column
        // (a row index is not one when the matrix is rectangular, as P and R are)
        int b = 0, e = 0, pad = 0;
        if (r < nrows) {
            const int i = rows[r];
            b = rp[i];
            e = rp[i + 1];
            pad = e > b ? col[e - 1] : 0;
            if (sdinv) sdinv[r] = (T)dinv[i];
        }
        for (int j = 0; j < len; ++j) {
            const bool in = b + j < e;
            scol[base + 32 * j] = in ? col[b + j] : pad;
            sval[base + 32 * j] = in ? (T)val[b + j] : T(0);
        }
    }
}

// y[row[r]] = (view row r) . x
template <class T>
__global__ void __launch_bounds__(256) k_sell_spmv(SellView v, const T *__restrict__ x, T *__restrict__ y) {
    const int *__restrict__ sptr = v.slice_ptr;
    const int *__restrict__ scol = v.col;
    const T *__restrict__ sval = static_cast<const T *>(v.val);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < v.nrows; r += gridDim.x * blockDim.x) {
        const int s = r >> 5;
        const int base = __ldg(sptr + s) + (r & 31);
        const int len = (__ldg(sptr + s + 1) - __ldg(sptr + s)) >> 5;
        T acc = T(0);
#pragma unroll 4
        for (int j = 0; j < len; ++j) acc = fma(__ldg(sval + base + 32 * j), __ldg(x + __ldg(scol + base + 32 * j)), acc);
        y[v.row[r]] = acc;
    }
}

// one Jacobi sweep over the view's rows (x_i + d_i (b_i - A_i x)); threads beyond the view copy
// the entries of the other rows (copy[], ncopy of them) from x to xo
template <class T>
__global__ void __launch_bounds__(256) k_sell_sweep(SellView v, const int *__restrict__ copy, int ncopy,
                                                    const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ xo) {
    const int *__restrict__ sptr = v.slice_ptr;
    const int *__restrict__ scol = v.col;
    const T *__restrict__ sval = static_cast<const T *>(v.val);
    const T *__restrict__ sd = static_cast<const T *>(v.dinv);
    const int total = v.nrows + ncopy;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < total; r += gridDim.x * blockDim.x) {
        if (r < v.nrows) {
            const int s = r >> 5;
            const int base = __ldg(sptr + s) + (r & 31);
            const int len = (__ldg(sptr + s + 1) - __ldg(sptr + s)) >> 5;
            T acc = T(0);
#pragma unroll 4
            for (int j = 0; j < len; ++j) acc = fma(__ldg(sval + base + 32 * j), __ldg(x + __ldg(scol + base + 32 * j)), acc);
            const int i = v.row[r];
            xo[i] = fma(sd[r], b[i] - acc, x[i]);
        } else {
            const int j = copy[r - v.nrows];
            xo[j] = x[j];
        }
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
void launch_frows(int n, const int8_t *cf, const int *cscan, int *frows, cudaStream_t s) {
    k_frows<<<grid_for(n, 256), 256, 0, s>>>(n, cf, cscan, frows);
    count_launch();
}

void launch_sell_prepare(int nrows, const int *rows_in, const int *rp, int *rows_sorted, int *cnt, cudaStream_t s) {
    if (nrows <= 0) return;
    k_sell_sort<<<(nrows + SELL_WINDOW - 1) / SELL_WINDOW, SELL_WINDOW, 0, s>>>(nrows, rows_in, rp, rows_sorted);
    const int nsl = (nrows + 31) / 32;
    k_sell_len<<<grid_for((long long)nsl * 32, 256), 256, 0, s>>>(nrows, rows_sorted, rp, cnt);
    count_launch(2);
}

void launch_sell_fill(const SellView &v, const DCsr &M, const double *dinv, bool fp32, cudaStream_t s) {
    if (v.nrows <= 0) return;
    const int nsl = (v.nrows + 31) / 32;
    const int grid = grid_for((long long)nsl * 32, 256);
    if (fp32)
        k_sell_fill<float><<<grid, 256, 0, s>>>(v.nrows, v.row, M.rp, M.col, M.val, dinv, v.slice_ptr, v.col,
                                                static_cast<float *>(v.val), static_cast<float *>(v.dinv));
    else
        k_sell_fill<double><<<grid, 256, 0, s>>>(v.nrows, v.row, M.rp, M.col, M.val, dinv, v.slice_ptr, v.col,
                                                 static_cast<double *>(v.val), static_cast<double *>(v.dinv));
    count_launch();
}

template <class T>
void sell_spmv(const SellView &v, const T *x, T *y, cudaStream_t s) {
    if (v.nrows <= 0) return;
    k_sell_spmv<T><<<grid_for(v.nrows, 256, 152 * 16), 256, 0, s>>>(v, x, y);
    count_launch();
}

template <class T>
void sell_sweep(const SellView &v, const int *copy, int ncopy, const T *b, const T *x, T *xo, cudaStream_t s) {
    if (v.nrows + ncopy <= 0) return;
    k_sell_sweep<T><<<grid_for((long long)v.nrows + ncopy, 256, 152 * 16), 256, 0, s>>>(v, copy, ncopy, b, x, xo);
    count_launch();
}

template void sell_spmv<float>(const SellView &, const float *, float *, cudaStream_t);
template void sell_spmv<double>(const SellView &, const double *, double *, cudaStream_t);
template void sell_sweep<float>(const SellView &, const int *, int, const float *, const float *, float *, cudaStream_t);
template void sell_sweep<double>(const SellView &, const int *, int, const double *, const double *, double *,
                                 cudaStream_t);

}  // namespace lair
