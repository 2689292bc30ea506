// solve_kernels.cu -- the cycle (Sec. 4): restriction b_c = R r, interpolation
// x = P x_c, Jacobi F/C sweeps x_i <- x_i + d_i (b_i - A_i x) (Eq. (2.4)), the dense
// coarsest solve, and the FP64 outer-iteration kernels (residual, norms, block dots
// for classical Gram-Schmidt, updates).
//
// Sparse rows are processed by groups of G consecutive lanes (G = 1, 2, 4, 8, 16 or
// 32, picked from the average row length); group lanes stride over the row so that
// consecutive lanes load consecutive column indices and values, and the partial sums
// are combined by xor-shuffles inside the group. All of these kernels are bound by
// HBM bandwidth on the large levels.
#include "setup_kernels.cuh"

namespace lair {

template <int G, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// y = A x  (also R b and P x_c)
template <int G, class T>
__global__ void __launch_bounds__(256) k_spmv(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                                             const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y) {
    const int gl = threadIdx.x & (G - 1);
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long lane = threadIdx.x & 31;
    for (long long base = tid; base - lane < (long long)nr * G; base += stride) {  // warp-uniform trip count
        int i = (int)(base / G);
        T acc = T(0);
        if (i < nr) {
            int b = __ldg(rp + i), e = __ldg(rp + i + 1);
            for (int k = b + gl; k < e; k += G) acc = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), acc);
        }
        acc = group_sum<G>(acc);
        if (i < nr && gl == 0) y[i] = acc;
    }
}

// one Jacobi sweep over the points with cf == target; all other points are copied
template <int G, class T>
__global__ void __launch_bounds__(256) k_sweep(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                                              const T *__restrict__ val, const int8_t *__restrict__ cf, int target,
                                              const T *__restrict__ dinv, const T *__restrict__ b,
                                              const T *__restrict__ x, T *__restrict__ xo) {
    const int gl = threadIdx.x & (G - 1);
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long lane = threadIdx.x & 31;
    for (long long base = tid; base - lane < (long long)nr * G; base += stride) {  // warp-uniform trip count
        int i = (int)(base / G);
        bool act = i < nr && cf[i] == target;
        T acc = T(0);
        if (act) {
            int bb = __ldg(rp + i), e = __ldg(rp + i + 1);
            for (int k = bb + gl; k < e; k += G) acc = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), acc);
        }
        acc = group_sum<G>(acc);
        if (i < nr && gl == 0) xo[i] = act ? fma(dinv[i], b[i] - acc, x[i]) : x[i];
    }
}

template <class T>
static int pick_group(const DCsr &A) {
    double avg = A.nr > 0 ? (double)A.nnz / A.nr : 1.0;
    if (avg <= 1.5) return 1;
    if (avg <= 3.0) return 2;
    if (avg <= 10.0) return 4;
    if (avg <= 24.0) return 8;
    if (avg <= 48.0) return 16;
    return 32;
}

template <class T>
static const T *vals_of(const DCsr &A);
template <> const double *vals_of<double>(const DCsr &A) { return A.val; }
template <> const float *vals_of<float>(const DCsr &A) { return A.val32; }

template <class T>
void spmv(const DCsr &A, const T *x, T *y, cudaStream_t s) {
    if (A.nr == 0) return;
    int G = pick_group<T>(A);
    int grid = grid_for((long long)A.nr * G, 256, device_sms() * 16);
    const T *v = vals_of<T>(A);
    switch (G) {
        case 1: k_spmv<1, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, x, y); break;
        case 2: k_spmv<2, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, x, y); break;
        case 4: k_spmv<4, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, x, y); break;
        case 8: k_spmv<8, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, x, y); break;
        case 16: k_spmv<16, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, x, y); break;
        default: k_spmv<32, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, x, y); break;
    }
    count_launch();
}

template <class T>
void sweep(const DCsr &A, const int8_t *cf, int target, const T *dinv, const T *b, const T *x, T *xo, cudaStream_t s) {
    if (A.nr == 0) return;
    int G = pick_group<T>(A);
    int grid = grid_for((long long)A.nr * G, 256, device_sms() * 16);
    const T *v = vals_of<T>(A);
    switch (G) {
        case 1: k_sweep<1, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, cf, target, dinv, b, x, xo); break;
        case 2: k_sweep<2, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, cf, target, dinv, b, x, xo); break;
        case 4: k_sweep<4, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, cf, target, dinv, b, x, xo); break;
        case 8: k_sweep<8, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, cf, target, dinv, b, x, xo); break;
        case 16: k_sweep<16, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, cf, target, dinv, b, x, xo); break;
        default: k_sweep<32, T><<<grid, 256, 0, s>>>(A.nr, A.rp, A.col, v, cf, target, dinv, b, x, xo); break;
    }
    count_launch();
}

template void spmv<double>(const DCsr &, const double *, double *, cudaStream_t);
template void spmv<float>(const DCsr &, const float *, float *, cudaStream_t);
template void sweep<double>(const DCsr &, const int8_t *, int, const double *, const double *, const double *, double *,
                            cudaStream_t);
template void sweep<float>(const DCsr &, const int8_t *, int, const float *, const float *, const float *, float *,
                           cudaStream_t);

// coarsest level: y = Ainv b (dense, FP64), with the input/output in T
template <class T>
__global__ void k_dense_apply(int n, const double *__restrict__ Ainv, const T *__restrict__ b, T *__restrict__ y) {
    pdl_enter();
    int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = wid; r < n; r += nw) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) acc = fma(Ainv[(size_t)r * n + c], (double)b[c], acc);
        acc = warp_sum(acc);
        if (lane == 0) y[r] = (T)acc;
    }
}

template <class T>
void dense_apply(int n, const double *Ainv, const T *b, T *y, cudaStream_t s) {
    launch_pdl(k_dense_apply<T>, grid_for((long long)n * 32, 256), 256, 0, s, n, Ainv, b, y);
    count_launch();
}
template void dense_apply<double>(int, const double *, const double *, double *, cudaStream_t);
template void dense_apply<float>(int, const double *, const float *, float *, cudaStream_t);

// ---------------------------------------------------------------------------------------
// FP64 outer iteration
// ---------------------------------------------------------------------------------------
constexpr int RED_BLOCKS = 152 * 4;
constexpr int RED_THREADS = 256;

// r = b - A x (FP64, one thread per row... group of G lanes), optional float copy, block partials of |r|^2
template <int G>
__global__ void __launch_bounds__(RED_THREADS) k_residual(int nr, const int *__restrict__ rp, const int *__restrict__ col,
                                                          const double *__restrict__ val, const double *__restrict__ b,
                                                          const double *__restrict__ x, double *__restrict__ r,
                                                          float *__restrict__ r32, double *__restrict__ part) {
    __shared__ double red[RED_THREADS / 32];
    const int gl = threadIdx.x & (G - 1);
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double ss = 0.0;
    const long long lane = threadIdx.x & 31;
    for (long long base = tid; base - lane < (long long)nr * G; base += stride) {  // warp-uniform trip count
        int i = (int)(base / G);
        double acc = 0.0;
        if (i < nr)
            for (int k = __ldg(rp + i) + gl; k < __ldg(rp + i + 1); k += G) acc = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), acc);
        acc = group_sum<G>(acc);
        if (i < nr && gl == 0) {
            double ri = b[i] - acc;
            r[i] = ri;
            if (r32) r32[i] = (float)ri;
            ss = fma(ri, ri, ss);
        }
    }
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

void residual(const DCsr &A, const double *b, const double *x, double *r, float *r32, double *part, cudaStream_t s) {
    int G = pick_group<double>(A);
    switch (G) {
        case 1: k_residual<1><<<RED_BLOCKS, RED_THREADS, 0, s>>>(A.nr, A.rp, A.col, A.val, b, x, r, r32, part); break;
        case 2: k_residual<2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(A.nr, A.rp, A.col, A.val, b, x, r, r32, part); break;
        case 4: k_residual<4><<<RED_BLOCKS, RED_THREADS, 0, s>>>(A.nr, A.rp, A.col, A.val, b, x, r, r32, part); break;
        case 8: k_residual<8><<<RED_BLOCKS, RED_THREADS, 0, s>>>(A.nr, A.rp, A.col, A.val, b, x, r, r32, part); break;
        case 16: k_residual<16><<<RED_BLOCKS, RED_THREADS, 0, s>>>(A.nr, A.rp, A.col, A.val, b, x, r, r32, part); break;
        default: k_residual<32><<<RED_BLOCKS, RED_THREADS, 0, s>>>(A.nr, A.rp, A.col, A.val, b, x, r, r32, part); break;
    }
    count_launch();
}

// block partials of sum_i x_i y_i for vectors x_k (stride ldx) against y, MD vectors per launch:
// part[k * RED_BLOCKS + block] for k = k0 .. k0 + m - 1
constexpr int MD = 8;
__global__ void __launch_bounds__(RED_THREADS) k_multidot(int n, int k0, int m, const double *__restrict__ X, long long ldx,
                                                          const double *__restrict__ y, double *__restrict__ part) {
    __shared__ double red[RED_THREADS / 32][MD];
    double acc[MD];
#pragma unroll
    for (int k = 0; k < MD; ++k) acc[k] = 0.0;
    const double *Xk = X + (long long)k0 * ldx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double yi = y[i];
#pragma unroll
        for (int k = 0; k < MD; ++k)
            if (k < m) acc[k] = fma(Xk[k * ldx + i], yi, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < MD; ++k) {
        if (k < m) {
            double v = warp_sum(acc[k]);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double t = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) t += red[w][threadIdx.x];
        part[(k0 + threadIdx.x) * RED_BLOCKS + blockIdx.x] = t;
    }
}

// out[k] = sum of the RED_BLOCKS partials of vector k (fixed order); if acc != NULL, acc[k] += out[k]
__global__ void k_finish(int m, const double *__restrict__ part, double *__restrict__ out, double *__restrict__ acc) {
    int k = blockIdx.x;
    if (k >= m) return;
    __shared__ double red[32];
    double t = 0.0;
    for (int b = threadIdx.x; b < RED_BLOCKS; b += blockDim.x) t += part[k * RED_BLOCKS + b];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
        out[k] = u;
        if (acc) acc[k] += u;
    }
}

void multidot(int n, int m, const double *X, long long ldx, const double *y, double *part, double *out, double *acc,
              cudaStream_t s) {
    for (int k0 = 0; k0 < m; k0 += MD) {
        int mm = m - k0 < MD ? m - k0 : MD;
        k_multidot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, k0, mm, X, ldx, y, part);
        count_launch();
    }
    k_finish<<<m, 256, 0, s>>>(m, part, out, acc);
    count_launch();
}

void finish_partials(int m, const double *part, double *out, cudaStream_t s) {
    k_finish<<<m, 256, 0, s>>>(m, part, out, nullptr);
    count_launch();
}

void finish_partials_acc(int m, const double *part, double *out, double *acc, cudaStream_t s) {
    k_finish<<<m, 256, 0, s>>>(m, part, out, acc);
    count_launch();
}

// w -= sum_k h_k X_k (h on the device)
__global__ void k_sub_combo(int n, int m, const double *__restrict__ X, long long ldx, const double *__restrict__ h,
                            double *__restrict__ w) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = w[i];
        for (int k = 0; k < m; ++k) v = fma(-h[k], X[k * ldx + i], v);
        w[i] = v;
    }
}

void sub_combo(int n, int m, const double *X, long long ldx, const double *h, double *w, cudaStream_t s) {
    k_sub_combo<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, m, X, ldx, h, w);
    count_launch();
}

// x += sum_k y_k Z_k (y on the device)
__global__ void k_add_combo(int n, int m, const double *__restrict__ Z, long long ldz, const double *__restrict__ y,
                            double *__restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = x[i];
        for (int k = 0; k < m; ++k) v = fma(y[k], Z[k * ldz + i], v);
        x[i] = v;
    }
}

void add_combo(int n, int m, const double *Z, long long ldz, const double *y, double *x, cudaStream_t s) {
    k_add_combo<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, m, Z, ldz, y, x);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// One classical Gram-Schmidt step with re-orthogonalisation (CGS2) of w against the m <= 32
// columns of X in three streaming passes over X instead of four:
//   pass 1: part_k = X_k . w
//   pass 2: w <- w - sum_k h1_k X_k, then part_k = X_k . w (the new w)
//   pass 3: w <- w - sum_k h2_k X_k, then part_0 = w . w
// Each thread loads X_k[i] once per pass and keeps it in registers for both of its uses.
// The w update accumulates fma(-h_k, X_k[i], .) in ascending k.
// ---------------------------------------------------------------------------------------
template <int MM>
__device__ __forceinline__ void block_partials(const double (&acc)[MM], int m, double *part) {
    __shared__ double red[RED_THREADS / 32][MM];
#pragma unroll
    for (int k = 0; k < MM; ++k)
        if (k < m) {
            const double v = warp_sum(acc[k]);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
        }
    __syncthreads();
    if ((int)threadIdx.x < m) {
        double t = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) t += red[w][threadIdx.x];
        part[threadIdx.x * RED_BLOCKS + blockIdx.x] = t;
    }
}

template <int MM, int PASS>
__global__ void __launch_bounds__(RED_THREADS, MM <= 8 ? RED_BLOCKS / 152 : 1) k_cgs_pass(int n, int m, const double *__restrict__ X, long long ldx,
                                                          const double *__restrict__ h, double *__restrict__ w,
                                                          double *__restrict__ part) {
    double acc[MM];
    double hk[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) {
        acc[k] = 0.0;
        hk[k] = (PASS > 1 && k < m) ? h[k] : 0.0;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double x[MM];
#pragma unroll
        for (int k = 0; k < MM; ++k) x[k] = k < m ? X[k * ldx + i] : 0.0;
        double v = w[i];
        if (PASS > 1) {
#pragma unroll
            for (int k = 0; k < MM; ++k)
                if (k < m) v = fma(-hk[k], x[k], v);
            w[i] = v;
        }
        if (PASS < 3) {
#pragma unroll
            for (int k = 0; k < MM; ++k)
                if (k < m) acc[k] = fma(x[k], v, acc[k]);
        } else {
            acc[0] = fma(v, v, acc[0]);
        }
    }
    block_partials<MM>(acc, PASS < 3 ? m : 1, part);
}

template <int MM>
static void cgs_pass_mm(int pass, int n, int m, const double *X, long long ldx, const double *h, double *w, double *part,
                        cudaStream_t s) {
    if (pass == 1) k_cgs_pass<MM, 1><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m, X, ldx, h, w, part);
    else if (pass == 2) k_cgs_pass<MM, 2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m, X, ldx, h, w, part);
    else k_cgs_pass<MM, 3><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, m, X, ldx, h, w, part);
}

void cgs_pass(int pass, int n, int m, const double *X, long long ldx, const double *h, double *w, double *part,
              cudaStream_t s) {
    if (m <= 8) cgs_pass_mm<8>(pass, n, m, X, ldx, h, w, part, s);
    else if (m <= 16) cgs_pass_mm<16>(pass, n, m, X, ldx, h, w, part, s);
    else cgs_pass_mm<32>(pass, n, m, X, ldx, h, w, part, s);
    count_launch();
}

// v_out = v_in / *nrm (nrm = sqrt of a device scalar of squared norm)
__global__ void k_scale_by_norm(int n, const double *__restrict__ v, const double *__restrict__ nrm2, double *__restrict__ out) {
    const double n2 = *nrm2;
    const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = v[i] * inv;
}

void scale_by_norm(int n, const double *v, const double *nrm2, double *out, cudaStream_t s) {
    k_scale_by_norm<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, v, nrm2, out);
    count_launch();
}

// precision conversions and plain vector updates
__global__ void k_d2f(int n, const double *__restrict__ a, float *__restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
__global__ void k_f2d(int n, const float *__restrict__ a, double *__restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}
__global__ void k_axpy_f(int n, const float *__restrict__ e, double *__restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += (double)e[i];
}
__global__ void k_axpy_d(int n, const double *__restrict__ e, double *__restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += e[i];
}

void d2f(int n, const double *a, float *b, cudaStream_t s) { k_d2f<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, a, b); count_launch(); }
void f2d(int n, const float *a, double *b, cudaStream_t s) { k_f2d<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, a, b); count_launch(); }
void axpy_f(int n, const float *e, double *x, cudaStream_t s) { k_axpy_f<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, e, x); count_launch(); }
void axpy_d(int n, const double *e, double *x, cudaStream_t s) { k_axpy_d<<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, e, x); count_launch(); }

// adjoint gradient on the pattern of A: g[k] = -lambda_i x_j
__global__ void k_grad_A(int n, const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ lam,
                         const double *__restrict__ x, double *__restrict__ g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double li = lam[i];
        for (int k = rp[i]; k < rp[i + 1]; ++k) g[k] = -li * x[col[k]];
    }
}

void grad_A(const DCsr &A, const double *lam, const double *x, double *g, cudaStream_t s) {
    k_grad_A<<<grid_for(A.nr, 256), 256, 0, s>>>(A.nr, A.rp, A.col, lam, x, g);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// batched systems: per-system residuals, norms, dots and updates over row tiles. The rows of
// every system are cut into tiles of at most SEG_TILE rows (tile t: system tile[t].x, rows
// [tile[t].y, tile[t].z)); a CTA works on one tile at a time, so a large system is spread over
// many SMs. Reductions write one partial per tile; seg_reduce then sums the partials of each
// system in tile order (one warp per system), so the result does not depend on scheduling.
// ---------------------------------------------------------------------------------------
constexpr int SEG_GRID = 152 * 8;

__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) k_tile_residual(SegTiles st, const int *__restrict__ rp, const int *__restrict__ col,
                                                       const double *__restrict__ val, const double *__restrict__ b,
                                                       const double *__restrict__ x, double *__restrict__ r,
                                                       float *__restrict__ r32) {
    __shared__ double red[8];
    for (int t = blockIdx.x; t < st.ntiles; t += gridDim.x) {
        const int4 tl = st.tile[t];
        if (st.active && !st.active[tl.x]) continue;
        double ss = 0.0;
        for (int i = tl.y + threadIdx.x; i < tl.z; i += blockDim.x) {
            double acc = 0.0;
            for (int k = rp[i]; k < rp[i + 1]; ++k) acc = fma(val[k], x[col[k]], acc);
            const double ri = b[i] - acc;
            r[i] = ri;
            if (r32) r32[i] = (float)ri;
            ss = fma(ri, ri, ss);
        }
        const double tsum = block_sum(ss, red);
        if (threadIdx.x == 0) st.part[t] = tsum;
    }
}

__global__ void __launch_bounds__(256) k_tile_norm2(SegTiles st, const double *__restrict__ v) {
    __shared__ double red[8];
    for (int t = blockIdx.x; t < st.ntiles; t += gridDim.x) {
        const int4 tl = st.tile[t];
        if (st.active && !st.active[tl.x]) continue;
        double ss = 0.0;
        for (int i = tl.y + threadIdx.x; i < tl.z; i += blockDim.x) ss = fma(v[i], v[i], ss);
        const double tsum = block_sum(ss, red);
        if (threadIdx.x == 0) st.part[t] = tsum;
    }
}

// One pass of the batched CGS2 step over the tiles of the running systems (m <= 31 and m <= MM <= SEG_TILE_PARTS
// columns of X, h per system at h[q * hs]), each thread loading X_k[i] once for both of its uses:
//   PASS 1: part[t][k] = X_k . w over the tile
//   PASS 2: w <- w - sum_k h_k X_k, then part[t][k] = X_k . w (the new w)
//   PASS 3: w <- w - sum_k h_k X_k, then part[t][0] = w . w
// The update accumulates fma(-h_k, X_k[i], .) in ascending k and every partial is a warp sum followed by the
// sum over the warps in order, as in k_tile_norm2.
template <int MM, int PASS>
__global__ void __launch_bounds__(256) k_tile_cgs(SegTiles st, int m, const double *__restrict__ X, long long ldx,
                                                  int hs, const double *__restrict__ h, double *__restrict__ w) {
    __shared__ double red[8][MM];
    __shared__ double hsh[MM];
    for (int t = blockIdx.x; t < st.ntiles; t += gridDim.x) {
        const int4 tl = st.tile[t];
        if (st.active && !st.active[tl.x]) continue;
        if (PASS > 1 && (int)threadIdx.x < MM) hsh[threadIdx.x] = (int)threadIdx.x < m ? h[(size_t)tl.x * hs + threadIdx.x] : 0.0;
        __syncthreads();
        double acc[PASS < 3 ? MM : 1];
#pragma unroll
        for (int k = 0; k < (PASS < 3 ? MM : 1); ++k) acc[k] = 0.0;
        for (int i = tl.y + threadIdx.x; i < tl.z; i += blockDim.x) {
            double x[MM];
#pragma unroll
            for (int k = 0; k < MM; ++k) x[k] = k < m ? X[k * ldx + i] : 0.0;
            double v = w[i];
            if (PASS > 1) {
#pragma unroll
                for (int k = 0; k < MM; ++k)
                    if (k < m) v = fma(-hsh[k], x[k], v);
                w[i] = v;
            }
            if (PASS < 3) {
#pragma unroll
                for (int k = 0; k < (PASS < 3 ? MM : 1); ++k)
                    if (k < m) acc[k] = fma(x[k], v, acc[k]);
            } else {
                acc[0] = fma(v, v, acc[0]);
            }
        }
        const int nout = PASS < 3 ? m : 1;
#pragma unroll
        for (int k = 0; k < (PASS < 3 ? MM : 1); ++k)
            if (k < nout) {
                const double v = warp_sum(acc[k]);
                if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
            }
        __syncthreads();
        if ((int)threadIdx.x < nout) {
            double s2 = 0.0;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s2 += red[ww][threadIdx.x];
            st.part[(size_t)t * SEG_TILE_PARTS + threadIdx.x] = s2;
        }
        __syncthreads();
    }
}

// out[q * hs + k0 + k] = sum of the system's tile partials part[t * pw + k] in tile order (k < m);
// acc_out[...] += the same when given. One warp per system.
__global__ void __launch_bounds__(256) k_seg_reduce(SegTiles st, int pw, int m, int hs, int k0, double *__restrict__ out,
                                                    double *__restrict__ acc_out) {
    const int lane = threadIdx.x & 31;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < st.nseg; q += (gridDim.x * blockDim.x) >> 5) {
        if (st.active && !st.active[q]) continue;
        const int t0 = st.first[q], t1 = st.first[q + 1];
        for (int k = 0; k < m; ++k) {
            double v = 0.0;
            for (int t = t0 + lane; t < t1; t += 32) v += st.part[(size_t)t * pw + k];
            v = warp_sum(v);
            if (lane == 0) {
                out[(size_t)q * hs + k0 + k] = v;
                if (acc_out) acc_out[(size_t)q * hs + k0 + k] += v;
            }
        }
    }
}

// x_i += sum_{k < cnt[q]} y[q * hs + k] Z_k[i] for the rows of system q
__global__ void __launch_bounds__(256) k_tile_add_combo(SegTiles st, const int *__restrict__ cnt, const double *__restrict__ Z,
                                                        long long ldz, int hs, const double *__restrict__ y,
                                                        double *__restrict__ x) {
    for (int t = blockIdx.x; t < st.ntiles; t += gridDim.x) {
        const int4 tl = st.tile[t];
        if (st.active && !st.active[tl.x]) continue;
        const int m = cnt[tl.x];
        if (m == 0) continue;
        const double *yq = y + (size_t)tl.x * hs;
        for (int i = tl.y + threadIdx.x; i < tl.z; i += blockDim.x) {
            double v = x[i];
            for (int k = 0; k < m; ++k) v = fma(yq[k], Z[k * ldz + i], v);
            x[i] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_tile_scale(SegTiles st, const double *__restrict__ v,
                                                    const double *__restrict__ nrm2, double *__restrict__ out) {
    for (int t = blockIdx.x; t < st.ntiles; t += gridDim.x) {
        const int4 tl = st.tile[t];
        if (st.active && !st.active[tl.x]) continue;
        const double n2 = nrm2[tl.x];
        const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
        for (int i = tl.y + threadIdx.x; i < tl.z; i += blockDim.x) out[i] = v[i] * inv;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_tile_axpy(SegTiles st, const uint8_t *__restrict__ active, const T *__restrict__ e,
                                                   double *__restrict__ x) {
    for (int t = blockIdx.x; t < st.ntiles; t += gridDim.x) {
        const int4 tl = st.tile[t];
        if (st.active && !st.active[tl.x]) continue;
        if (!active[tl.x]) continue;
        for (int i = tl.y + threadIdx.x; i < tl.z; i += blockDim.x) x[i] += (double)e[i];
    }
}

// ---------------------------------------------------------------------------------------
// device-side control of the batched outer loops: one thread per system decides, from the
// per-system norms the tile kernels reduced, whether the system goes on, and keeps its Krylov
// state; the flags feed the tile kernels (SegTiles.active) of the next step directly, so the
// host never has to read a norm to continue. count (zero on entry) receives the number of
// systems still running. The arithmetic of the stopping tests and Givens rotations is the
// oracle's (separate roundings, no fused operations).
// ---------------------------------------------------------------------------------------
__global__ void k_bat_bnorm(int nseg, const double *__restrict__ nrm2, double *__restrict__ bn) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nseg) bn[q] = nrm2[q] > 0.0 ? sqrt(nrm2[q]) : 1.0;
}

// stationary refinement, iteration it: from ||r_q||^2, deactivate converged systems; count the running ones
// (each running system then receives one more cycle)
__global__ void k_bat_stat_check(BatchCtl c, const double *__restrict__ nrm2, int it, int *count) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= c.nseg || !c.run[q]) return;
    const double r = __ddiv_rn(sqrt(nrm2[q]), c.bn[q]);
    c.rl[q] = r;
    if (!isfinite(r)) {
        *c.nan = 1;
        c.run[q] = 0;
        return;
    }
    if (r <= c.tol || it >= c.max_iter) {
        c.run[q] = 0;
        return;
    }
    c.its[q] += 1;
    atomicAdd(count, 1);
}

// FGMRES restart: beta = ||r_q||, the stopping test on it, g = beta e_1 for the systems that go on
__global__ void k_bat_fg_restart(BatchCtl c, const double *__restrict__ nrm2, int *count) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= c.nseg) return;
    c.jd[q] = 0;
    const double beta = sqrt(nrm2[q]);
    const double r = __ddiv_rn(beta, c.bn[q]);
    c.rl[q] = r;
    if (!isfinite(r)) {
        *c.nan = 1;
        c.done[q] = 1;
    }
    if (r <= c.tol || c.its[q] >= c.max_iter) c.done[q] = 1;
    c.run[q] = c.done[q] ? 0 : 1;
    if (!c.run[q]) return;
    double *g = c.g + (size_t)q * (c.m + 1);
    for (int k = 0; k <= c.m; ++k) g[k] = 0.0;
    g[0] = beta;
    atomicAdd(count, 1);
}

// FGMRES step j of every running system: the new Hessenberg column (the Gram-Schmidt sums h[q * hs + k],
// k <= j, and ||w||), the earlier rotations applied to it, a new rotation, the residual estimate and the
// stopping test; a system that stops keeps its step count in jd
__global__ void k_bat_fg_givens(BatchCtl c, int j, const double *__restrict__ hsum, const double *__restrict__ nrm2w,
                                int *count) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= c.nseg || !c.run[q]) return;
    const int m = c.m;
    double hc[BATCH_HS + 1];
    for (int k = 0; k <= j; ++k) hc[k] = hsum[(size_t)q * c.hs + k];
    const double hn = sqrt(nrm2w[q]);
    hc[j + 1] = hn;
    double *cs = c.cs + (size_t)q * m, *sn = c.sn + (size_t)q * m, *g = c.g + (size_t)q * (m + 1);
    double *Hq = c.Hm + (size_t)q * (m + 1) * m;
    for (int k = 0; k < j; ++k) {
        const double t = __dadd_rn(__dmul_rn(cs[k], hc[k]), __dmul_rn(sn[k], hc[k + 1]));
        hc[k + 1] = __dadd_rn(__dmul_rn(-sn[k], hc[k]), __dmul_rn(cs[k], hc[k + 1]));
        hc[k] = t;
    }
    const double den = sqrt(__dadd_rn(__dmul_rn(hc[j], hc[j]), __dmul_rn(hc[j + 1], hc[j + 1])));
    cs[j] = den > 0.0 ? __ddiv_rn(hc[j], den) : 1.0;
    sn[j] = den > 0.0 ? __ddiv_rn(hc[j + 1], den) : 0.0;
    hc[j] = den;
    g[j + 1] = __dmul_rn(-sn[j], g[j]);
    g[j] = __dmul_rn(cs[j], g[j]);
    for (int k = 0; k <= j; ++k) Hq[(size_t)k * m + j] = hc[k];
    c.its[q] += 1;
    const double est = __ddiv_rn(fabs(g[j + 1]), c.bn[q]);
    if (est <= c.tol || hn == 0.0 || !isfinite(est) || c.its[q] >= c.max_iter || j == m - 1) {
        c.run[q] = 0;
        c.jd[q] = j + 1;
    } else {
        atomicAdd(count, 1);
    }
}

// y_q = H_q^{-1} g_q (upper triangular, jd_q x jd_q) for the update x += Z y
__global__ void k_bat_fg_solve_y(BatchCtl c, double *__restrict__ y) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= c.nseg) return;
    const int jd = c.jd[q], m = c.m;
    const double *Hq = c.Hm + (size_t)q * (m + 1) * m, *g = c.g + (size_t)q * (m + 1);
    double *yq = y + (size_t)q * c.hs;
    for (int k = jd - 1; k >= 0; --k) {
        double acc = g[k];
        for (int cc = k + 1; cc < jd; ++cc) acc = __dsub_rn(acc, __dmul_rn(Hq[(size_t)k * m + cc], yq[cc]));
        yq[k] = __ddiv_rn(acc, Hq[(size_t)k * m + k]);
    }
}

void bat_bnorm(int nseg, const double *nrm2, double *bn, cudaStream_t s) {
    k_bat_bnorm<<<(nseg + 127) / 128, 128, 0, s>>>(nseg, nrm2, bn);
    count_launch();
}
void bat_stat_check(const BatchCtl &c, const double *nrm2, int it, int *count, cudaStream_t s) {
    k_bat_stat_check<<<(c.nseg + 127) / 128, 128, 0, s>>>(c, nrm2, it, count);
    count_launch();
}
void bat_fg_restart(const BatchCtl &c, const double *nrm2, int *count, cudaStream_t s) {
    k_bat_fg_restart<<<(c.nseg + 127) / 128, 128, 0, s>>>(c, nrm2, count);
    count_launch();
}
void bat_fg_givens(const BatchCtl &c, int j, const double *hsum, const double *nrm2w, int *count, cudaStream_t s) {
    k_bat_fg_givens<<<(c.nseg + 127) / 128, 128, 0, s>>>(c, j, hsum, nrm2w, count);
    count_launch();
}
void bat_fg_solve_y(const BatchCtl &c, double *y, cudaStream_t s) {
    k_bat_fg_solve_y<<<(c.nseg + 127) / 128, 128, 0, s>>>(c, y);
    count_launch();
}

static int seg_grid(const SegTiles &st) { return st.ntiles < SEG_GRID ? (st.ntiles > 0 ? st.ntiles : 1) : SEG_GRID; }

static void seg_reduce(const SegTiles &st, int pw, int m, int hs, int k0, double *out, double *acc, cudaStream_t s) {
    k_seg_reduce<<<(st.nseg + 7) / 8, 256, 0, s>>>(st, pw, m, hs, k0, out, acc);
    count_launch();
}

template <int MM>
static void seg_cgs_mm(const SegTiles &st, int pass, int m, const double *X, long long ldx, int hs, const double *h,
                       double *w, cudaStream_t s) {
    if (pass == 1) k_tile_cgs<MM, 1><<<seg_grid(st), 256, 0, s>>>(st, m, X, ldx, hs, h, w);
    else if (pass == 2) k_tile_cgs<MM, 2><<<seg_grid(st), 256, 0, s>>>(st, m, X, ldx, hs, h, w);
    else k_tile_cgs<MM, 3><<<seg_grid(st), 256, 0, s>>>(st, m, X, ldx, hs, h, w);
    count_launch();
}

void seg_cgs_pass(const SegTiles &st, int pass, int m, const double *X, long long ldx, int hs, const double *h, double *w,
                  double *out, double *acc, cudaStream_t s) {
    if (m <= 8) seg_cgs_mm<8>(st, pass, m, X, ldx, hs, h, w, s);
    else if (m <= 16) seg_cgs_mm<16>(st, pass, m, X, ldx, hs, h, w, s);
    else seg_cgs_mm<32>(st, pass, m, X, ldx, hs, h, w, s);
    if (pass < 3) seg_reduce(st, SEG_TILE_PARTS, m, hs, 0, out, acc, s);
    else seg_reduce(st, SEG_TILE_PARTS, 1, 1, 0, out, nullptr, s);
}

void seg_add_combo(const SegTiles &st, const int *cnt, const double *Z, long long ldz, int hs, const double *y, double *x,
                   cudaStream_t s) {
    k_tile_add_combo<<<seg_grid(st), 256, 0, s>>>(st, cnt, Z, ldz, hs, y, x);
    count_launch();
}
void seg_scale(const SegTiles &st, const double *v, const double *nrm2, double *out, cudaStream_t s) {
    k_tile_scale<<<seg_grid(st), 256, 0, s>>>(st, v, nrm2, out);
    count_launch();
}
void seg_residual(const DCsr &A, const SegTiles &st, const double *b, const double *x, double *r, float *r32,
                  double *norm2, cudaStream_t s) {
    k_tile_residual<<<seg_grid(st), 256, 0, s>>>(st, A.rp, A.col, A.val, b, x, r, r32);
    count_launch();
    seg_reduce(st, 1, 1, 1, 0, norm2, nullptr, s);
}
void seg_norm2(const SegTiles &st, const double *v, double *norm2, cudaStream_t s) {
    k_tile_norm2<<<seg_grid(st), 256, 0, s>>>(st, v);
    count_launch();
    seg_reduce(st, 1, 1, 1, 0, norm2, nullptr, s);
}
template <class T>
void seg_axpy(const SegTiles &st, const uint8_t *active, const T *e, double *x, cudaStream_t s) {
    k_tile_axpy<T><<<seg_grid(st), 256, 0, s>>>(st, active, e, x);
    count_launch();
}
template void seg_axpy<float>(const SegTiles &, const uint8_t *, const float *, double *, cudaStream_t);
template void seg_axpy<double>(const SegTiles &, const uint8_t *, const double *, double *, cudaStream_t);

__global__ void k_gather_int(int m, const int *__restrict__ idx, const int *__restrict__ src, int *__restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) out[t] = src[idx[t]];
}

void gather_int(int m, const int *idx, const int *src, int *out, cudaStream_t s) {
    k_gather_int<<<grid_for(m, 256), 256, 0, s>>>(m, idx, src, out);
    count_launch();
}

// rows and entries of F and C rows: out = {n_F, nnz_F, n_C, nnz_C}
__global__ void k_cf_stats(int n, const int *__restrict__ rp, const int8_t *__restrict__ cf,
                           unsigned long long *__restrict__ out) {
    unsigned long long a = 0, b = 0, c = 0, d = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long len = (unsigned long long)(rp[i + 1] - rp[i]);
        if (cf[i] == CF_F) { a += 1; b += len; } else { c += 1; d += len; }
    }
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c); d = warp_sum(d);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out + 0, a); atomicAdd(out + 1, b); atomicAdd(out + 2, c); atomicAdd(out + 3, d);
    }
}

void cf_stats(const DCsr &A, const int8_t *cf, unsigned long long *out4, cudaStream_t s) {
    k_cf_stats<<<grid_for(A.nr, 256), 256, 0, s>>>(A.nr, A.rp, cf, out4);
    count_launch();
}

}  // namespace lair
