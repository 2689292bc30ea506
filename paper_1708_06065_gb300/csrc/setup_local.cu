// setup_local.cu -- the local dense systems of lAIR (Sec. 3.1, Eq. (3.1)/(3.2)),
// assembly of R = [Z I] and of the transposed interpolation rows, one-point
// interpolation (Sec. 4), and the DG block-diagonal scaling (Sec. 4.2.1).
//
// One routine solves every local system, written over a "team" of cooperating
// threads: a single thread (tiny systems, s <= 6), a warp (s <= 32, matrix in
// shared memory) or a CTA (s > 32, matrix in global scratch). Whatever the team,
// each matrix entry receives the same sequence of IEEE operations:
//   LU with partial pivoting (pivot = largest |M[r][k]|, r >= k, ties -> smallest r),
//   multipliers l_r = M[r][k] / M[k][k], updates M[r][c] = fma(-l_r, M[k][c], M[r][c]),
//   column-oriented back substitution z[c] = rhs[c] / M[c][c], rhs[r] = fma(-M[r][c], z[c], rhs[r]);
//   singular when a pivot |M[k][k]| <= (s * eps) * max|M|, then the minimum-norm
//   least-squares solution by one-sided Jacobi (Hestenes) with canonical 32-way tree sums.
// so the restriction does not depend on which bin a row fell into.
#include "setup_kernels.cuh"

namespace lair {

// ---------------------------------------------------------------------------------------
// correctly rounded scalar operations (no contraction)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }

template <class T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 0x1.0p-52; };
template <> struct Eps<float> { static constexpr float v = 0x1.0p-23f; };

// ---------------------------------------------------------------------------------------
// teams
// ---------------------------------------------------------------------------------------
struct ThreadTeam {
    __device__ int rank() const { return 0; }
    __device__ int size() const { return 1; }
    __device__ void sync() const {}
    template <class T> __device__ T max(T v) const { return v; }
    // (value, index) argmax with ties -> smaller index; each member passes its local best
    template <class T> __device__ void argmax(T &v, int &idx) const {}
    __device__ int any(int p) const { return p; }
};

struct WarpTeam {
    __device__ int rank() const { return threadIdx.x & 31; }
    __device__ int size() const { return 32; }
    __device__ void sync() const { __syncwarp(); }
    template <class T> __device__ T max(T v) const {
        for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
    template <class T> __device__ void argmax(T &v, int &idx) const {
        for (int o = 16; o >= 1; o >>= 1) {
            T ov = __shfl_xor_sync(0xffffffffu, v, o);
            int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (oi >= 0 && (idx < 0 || ov > v || (ov == v && oi < idx))) { v = ov; idx = oi; }
        }
    }
    __device__ int any(int p) const { return __any_sync(0xffffffffu, p); }
};

// CTA team: blockDim.x is a multiple of 32 (<= 1024); red is shared scratch of >= 2*32 words of 8 bytes
struct CtaTeam {
    double *red;
    __device__ int rank() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ void sync() const { __syncthreads(); }
    template <class T> __device__ T max(T v) const {
        WarpTeam w;
        v = w.max(v);
        int nw = blockDim.x >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
        __syncthreads();
        T r = (T)red[0];
        for (int k = 1; k < nw; ++k) r = fmax(r, (T)red[k]);
        __syncthreads();
        return r;
    }
    template <class T> __device__ void argmax(T &v, int &idx) const {
        WarpTeam w;
        w.argmax(v, idx);
        int nw = blockDim.x >> 5;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = (double)v;
            reinterpret_cast<int *>(red + 32)[threadIdx.x >> 5] = idx;
        }
        __syncthreads();
        T bv = (T)red[0];
        int bi = reinterpret_cast<int *>(red + 32)[0];
        for (int k = 1; k < nw; ++k) {
            T ov = (T)red[k];
            int oi = reinterpret_cast<int *>(red + 32)[k];
            if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
        }
        __syncthreads();
        v = bv;
        idx = bi;
    }
    __device__ int any(int p) const { return __syncthreads_or(p); }
};

// ---------------------------------------------------------------------------------------
// canonical 32-way tree sum of x[r] * y[r], r < s (strides sx, sy): partial l = fma-sum of
// the terms r = l mod 32 in ascending r; then butterflies p_l = p_l + p_{l^o}, o = 16..1.
// Every member of the team receives the result.
// ---------------------------------------------------------------------------------------
template <class T>
__device__ T tree_dot(const ThreadTeam &, const T *x, int sx, const T *y, int sy, int s) {
    T p[32];
    for (int l = 0; l < 32; ++l) p[l] = T(0);
    for (int r = 0; r < s; ++r) p[r & 31] = fma_rn(x[r * sx], y[r * sy], p[r & 31]);
    for (int o = 16; o >= 1; o >>= 1) {
        T q[32];
        for (int l = 0; l < 32; ++l) q[l] = add_rn(p[l], p[l ^ o]);
        for (int l = 0; l < 32; ++l) p[l] = q[l];
    }
    return p[0];
}

template <class T>
__device__ T tree_dot(const WarpTeam &, const T *x, int sx, const T *y, int sy, int s) {
    int l = threadIdx.x & 31;
    T p = T(0);
    for (int r = l; r < s; r += 32) p = fma_rn(x[r * sx], y[r * sy], p);
    for (int o = 16; o >= 1; o >>= 1) p = add_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
    return p;
}

template <class T>
__device__ T tree_dot(const CtaTeam &t, const T *x, int sx, const T *y, int sy, int s) {
    __syncthreads();
    if (threadIdx.x < 32) {
        T p = tree_dot(WarpTeam(), x, sx, y, sy, s);
        if (threadIdx.x == 0) t.red[0] = (double)p;
    }
    __syncthreads();
    T r = (T)t.red[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------------------
// local system gather: M[r][c] = B[l_c][l_r] and rhs[r] = -B[i][l_r] (Eq. (3.2))
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int find_pos(const int *list, int len, int key) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = list[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

template <class Team, class T>
__device__ void gather_system(const Team &tm, const int *__restrict__ brp, const int *__restrict__ bcol,
                              const double *__restrict__ bval, int i, const int *nb, int s, T *M, T *rhs) {
    for (int e = tm.rank(); e < s * s; e += tm.size()) M[e] = T(0);
    for (int e = tm.rank(); e < s; e += tm.size()) rhs[e] = T(0);
    tm.sync();
    for (int c = tm.rank(); c < s; c += tm.size()) {
        int row = nb[c];
        for (int k = brp[row]; k < brp[row + 1]; ++k) {
            int r = find_pos(nb, s, bcol[k]);
            if (r >= 0) M[r * s + c] = (T)bval[k];
        }
    }
    for (int k = brp[i] + tm.rank(); k < brp[i + 1]; k += tm.size()) {
        int r = find_pos(nb, s, bcol[k]);
        if (r >= 0) rhs[r] = (T)(-bval[k]);
    }
    tm.sync();
}

// LU with partial pivoting and back substitution; returns 1 when singular (nothing solved)
template <class Team, class T>
__device__ int lu_solve(const Team &tm, int s, T *M, T *rhs, T *z, T *L) {
    T mx = T(0);
    for (int e = tm.rank(); e < s * s; e += tm.size()) mx = fmax(mx, fabs(M[e]));
    mx = tm.max(mx);
    if (mx == T(0)) return 1;
    const T thr = mul_rn(mul_rn((T)s, Eps<T>::v), mx);
    for (int k = 0; k < s; ++k) {
        T best = T(-1);
        int piv = -1;
        for (int r = k + tm.rank(); r < s; r += tm.size()) {
            T v = fabs(M[r * s + k]);
            if (piv < 0 || v > best) { best = v; piv = r; }
        }
        tm.argmax(best, piv);
        if (best <= thr) return 1;
        if (piv != k) {
            for (int c = tm.rank(); c < s; c += tm.size()) {
                T t = M[k * s + c];
                M[k * s + c] = M[piv * s + c];
                M[piv * s + c] = t;
            }
            if (tm.rank() == 0) {
                T t = rhs[k];
                rhs[k] = rhs[piv];
                rhs[piv] = t;
            }
        }
        tm.sync();
        for (int r = k + 1 + tm.rank(); r < s; r += tm.size()) L[r] = div_rn(M[r * s + k], M[k * s + k]);
        tm.sync();
        const int w = s - k;           // columns k+1 .. s-1 plus the right-hand side
        const int cnt = (s - k - 1) * w;
        for (int e = tm.rank(); e < cnt; e += tm.size()) {
            int r = k + 1 + e / w;
            int c = k + 1 + e % w;
            if (c == s) rhs[r] = fma_rn(-L[r], rhs[k], rhs[r]);
            else M[r * s + c] = fma_rn(-L[r], M[k * s + c], M[r * s + c]);
        }
        tm.sync();
    }
    for (int c = s - 1; c >= 0; --c) {
        if (tm.rank() == 0) z[c] = div_rn(rhs[c], M[c * s + c]);
        tm.sync();
        const T zc = z[c];
        for (int r = tm.rank(); r < c; r += tm.size()) rhs[r] = fma_rn(-M[r * s + c], zc, rhs[r]);
        tm.sync();
    }
    return 0;
}

// The same elimination as lu_solve without a right-hand side, for systems solved for several right-hand
// sides: the multiplier of row r at step k is kept in M[r][k] and the pivot row in piv[k]; only columns
// >= k take part in a row swap, so the kept multipliers stay where step k left them. lu_apply then runs
// lu_solve's right-hand-side operations in lu_solve's order: the same results, bit for bit.
template <class Team, class T>
__device__ int lu_factor(const Team &tm, int s, T *M, T *L, int *piv) {
    T mx = T(0);
    for (int e = tm.rank(); e < s * s; e += tm.size()) mx = fmax(mx, fabs(M[e]));
    mx = tm.max(mx);
    if (mx == T(0)) return 1;
    const T thr = mul_rn(mul_rn((T)s, Eps<T>::v), mx);
    for (int k = 0; k < s; ++k) {
        T best = T(-1);
        int p = -1;
        for (int r = k + tm.rank(); r < s; r += tm.size()) {
            T v = fabs(M[r * s + k]);
            if (p < 0 || v > best) { best = v; p = r; }
        }
        tm.argmax(best, p);
        if (best <= thr) return 1;
        if (p != k)
            for (int c = k + tm.rank(); c < s; c += tm.size()) {
                T t = M[k * s + c];
                M[k * s + c] = M[p * s + c];
                M[p * s + c] = t;
            }
        if (tm.rank() == 0) piv[k] = p;
        tm.sync();
        for (int r = k + 1 + tm.rank(); r < s; r += tm.size()) L[r] = div_rn(M[r * s + k], M[k * s + k]);
        tm.sync();
        const int w = s - k - 1;
        for (int e = tm.rank(); e < w * w; e += tm.size()) {
            int r = k + 1 + e / w;
            int c = k + 1 + e % w;
            M[r * s + c] = fma_rn(-L[r], M[k * s + c], M[r * s + c]);
        }
        for (int r = k + 1 + tm.rank(); r < s; r += tm.size()) M[r * s + k] = L[r];
        tm.sync();
    }
    return 0;
}

template <class Team, class T>
__device__ void lu_apply(const Team &tm, int s, const T *M, const int *piv, T *rhs, T *z) {
    for (int k = 0; k < s; ++k) {
        if (tm.rank() == 0 && piv[k] != k) {
            T t = rhs[k];
            rhs[k] = rhs[piv[k]];
            rhs[piv[k]] = t;
        }
        tm.sync();
        const T rk = rhs[k];
        for (int r = k + 1 + tm.rank(); r < s; r += tm.size()) rhs[r] = fma_rn(-M[r * s + k], rk, rhs[r]);
        tm.sync();
    }
    for (int c = s - 1; c >= 0; --c) {
        if (tm.rank() == 0) z[c] = div_rn(rhs[c], M[c * s + c]);
        tm.sync();
        const T zc = z[c];
        for (int r = tm.rank(); r < c; r += tm.size()) rhs[r] = fma_rn(-M[r * s + c], zc, rhs[r]);
        tm.sync();
    }
}

constexpr int LS_MAX_SWEEPS = 60;

// minimum-norm least squares by one-sided Jacobi; B holds the original matrix (destroyed),
// rhs the original right-hand side; V is s*s scratch; out z
template <class Team, class T>
__device__ void jacobi_ls(const Team &tm, int s, T *B, const T *rhs, T *V, T *z) {
    for (int e = tm.rank(); e < s * s; e += tm.size()) V[e] = (e / s == e % s) ? T(1) : T(0);
    tm.sync();
    const T tol = mul_rn(Eps<T>::v, (T)s);
    for (int sweep = 0; sweep < LS_MAX_SWEEPS; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < s - 1; ++p)
            for (int q = p + 1; q < s; ++q) {
                T alpha = tree_dot(tm, B + p, s, B + p, s, s);
                T beta = tree_dot(tm, B + q, s, B + q, s, s);
                T gamma = tree_dot(tm, B + p, s, B + q, s, s);
                if (gamma == T(0) || fabs(gamma) <= mul_rn(tol, sqrt_rn(mul_rn(alpha, beta)))) continue;
                rotated = 1;
                T zeta = div_rn(sub_rn(beta, alpha), mul_rn(T(2), gamma));
                T sg = zeta >= T(0) ? T(1) : T(-1);
                T t = div_rn(sg, add_rn(fabs(zeta), sqrt_rn(fma_rn(zeta, zeta, T(1)))));
                T c = div_rn(T(1), sqrt_rn(fma_rn(t, t, T(1))));
                T sn = mul_rn(c, t);
                for (int r = tm.rank(); r < s; r += tm.size()) {
                    T bp = B[r * s + p], bq = B[r * s + q];
                    B[r * s + p] = fma_rn(c, bp, -mul_rn(sn, bq));
                    B[r * s + q] = fma_rn(sn, bp, mul_rn(c, bq));
                    T vp = V[r * s + p], vq = V[r * s + q];
                    V[r * s + p] = fma_rn(c, vp, -mul_rn(sn, vq));
                    V[r * s + q] = fma_rn(sn, vp, mul_rn(c, vq));
                }
                tm.sync();
            }
        if (!rotated) break;
    }
    T smax = T(0);
    for (int j = 0; j < s; ++j) {
        T sig = sqrt_rn(tree_dot(tm, B + j, s, B + j, s, s));
        if (sig > smax) smax = sig;
    }
    const T cut = mul_rn(mul_rn((T)s, Eps<T>::v), smax);
    for (int r = tm.rank(); r < s; r += tm.size()) z[r] = T(0);
    tm.sync();
    for (int j = 0; j < s; ++j) {
        T sig = sqrt_rn(tree_dot(tm, B + j, s, B + j, s, s));
        if (!(sig > cut)) continue;
        T coef = div_rn(div_rn(tree_dot(tm, B + j, s, rhs, 1, s), sig), sig);
        for (int r = tm.rank(); r < s; r += tm.size()) z[r] = fma_rn(V[r * s + j], coef, z[r]);
        tm.sync();
    }
}

// row c of the output: {nb, z} u {(i, 1)} at nb_rp[c] + c, ascending; the least-squares flag
template <class Team, class T>
__device__ void write_row(const Team &tm, const LocalArgs &a, int c, int i, const int *nb, int s, const T *z,
                          int singular) {
    const int base = a.nb_rp[c] + c;
    for (int r = tm.rank(); r < s; r += tm.size()) {
        int pos = r + (nb[r] > i ? 1 : 0);
        a.out_col[base + pos] = nb[r];
        double v = (double)z[r];
        a.out_val[base + pos] = v;
        if (a.out_val32) a.out_val32[base + pos] = (float)z[r];
    }
    if (tm.rank() == 0) {
        int lo = 0, hi = s;
        while (lo < hi) { int m = (lo + hi) >> 1; if (nb[m] < i) lo = m + 1; else hi = m; }
        a.out_col[base + lo] = i;
        a.out_val[base + lo] = 1.0;
        if (a.out_val32) a.out_val32[base + lo] = 1.0f;
        if (a.lsflag) a.lsflag[c] = (uint8_t)singular;
    }
    tm.sync();
}

// the right-hand side alone: rhs[r] = -B[i][l_r]
template <class Team, class T>
__device__ void gather_rhs(const Team &tm, const int *__restrict__ brp, const int *__restrict__ bcol,
                           const double *__restrict__ bval, int i, const int *nb, int s, T *rhs) {
    for (int e = tm.rank(); e < s; e += tm.size()) rhs[e] = T(0);
    tm.sync();
    for (int k = brp[i] + tm.rank(); k < brp[i + 1]; k += tm.size()) {
        int r = find_pos(nb, s, bcol[k]);
        if (r >= 0) rhs[r] = (T)(-bval[k]);
    }
    tm.sync();
}

// nAIR (Sec. 3.2): the Neumann series of M = D - (D - M) from its diagonal D, truncated at degree k:
// z = y_0 + ... + y_k, y_0 = D^{-1} rhs, y_{m+1}[r] = -(sum_{c != r} M[r][c] y_m[c]) / M[r][r] (fma from 0 in
// ascending c). With M = A_NN^T and rhs = -a_{i,N} this is row i of -A_cf sum (D^{-1}E)^m D^{-1} on the set N,
// which holds every point the series reaches. y and yn are s-entry scratch.
template <class Team, class T>
__device__ void neumann_sum(const Team &tm, int s, const T *M, const T *rhs, T *z, T *y, T *yn, int k) {
    for (int r = tm.rank(); r < s; r += tm.size()) {
        y[r] = div_rn(rhs[r], M[r * s + r]);
        z[r] = y[r];
    }
    tm.sync();
    for (int m = 1; m <= k; ++m) {
        for (int r = tm.rank(); r < s; r += tm.size()) {
            T acc = T(0);
            for (int c = 0; c < s; ++c)
                if (c != r) acc = fma_rn(M[r * s + c], y[c], acc);
            yn[r] = div_rn(-acc, M[r * s + r]);
        }
        tm.sync();
        for (int r = tm.rank(); r < s; r += tm.size()) {
            y[r] = yn[r];
            z[r] = add_rn(z[r], yn[r]);
        }
        tm.sync();
    }
}

// one C point: gather, solve (LU or least squares) or sum the Neumann series, write its R row {nb, z} u {(i, 1)}
template <class Team, class T>
__device__ void solve_row(const Team &tm, const LocalArgs &a, int c, T *M, T *rhs, T *z, T *L, T *V) {
    const int i = a.cpts[c];
    const int *nb = a.nb_col + a.nb_rp[c];
    const int s = a.nb_rp[c + 1] - a.nb_rp[c];
    int singular = 0;
    if (s > 0) {
        gather_system(tm, a.brp, a.bcol, a.bval, i, nb, s, M, rhs);
        if (a.neumann_deg >= 0) neumann_sum(tm, s, M, rhs, z, L, V, a.neumann_deg);
        else singular = lu_solve(tm, s, M, rhs, z, L);
        if (singular) {
            gather_system(tm, a.brp, a.bcol, a.bval, i, nb, s, M, rhs);
            jacobi_ls(tm, s, M, rhs, V, z);
        }
    }
    tm.sync();
    write_row(tm, a, c, i, nb, s, z, singular);
}

// the C points c0 .. c0 + rows_per - 1 share one set (the unknowns of a C node, nodal hierarchy): the
// system matrix is gathered and factored once and applied to each row's right-hand side
template <class Team, class T>
__device__ void solve_rows_shared(const Team &tm, const LocalArgs &a, int q, T *M, T *rhs, T *z, T *L, T *V) {
    const int c0 = q * a.rows_per;
    const int *nb = a.nb_col + a.nb_rp[c0];
    const int s = a.nb_rp[c0 + 1] - a.nb_rp[c0];
    int *piv = reinterpret_cast<int *>(V);   // V is only needed by the least-squares branch
    int singular = 0;
    if (s > 0) {
        gather_system(tm, a.brp, a.bcol, a.bval, a.cpts[c0], nb, s, M, rhs);
        singular = lu_factor(tm, s, M, L, piv);
    }
    for (int t = 0; t < a.rows_per; ++t) {
        const int c = c0 + t, i = a.cpts[c];
        if (s > 0) {
            if (!singular) {
                gather_rhs(tm, a.brp, a.bcol, a.bval, i, nb, s, rhs);
                lu_apply(tm, s, M, piv, rhs, z);
            } else {
                gather_system(tm, a.brp, a.bcol, a.bval, i, nb, s, M, rhs);
                jacobi_ls(tm, s, M, rhs, V, z);
            }
        }
        tm.sync();
        write_row(tm, a, c, i, nb, s, z, singular);
    }
}

// ---------------------------------------------------------------------------------------
// bin kernels
// ---------------------------------------------------------------------------------------
// SHARED: the lists hold groups of rows that share one set (solve_rows_shared); a separate instantiation,
// so that the one-row kernels keep their register budget
template <class T, bool SHARED>
__global__ void __launch_bounds__(128) k_local_thread(LocalArgs a, const int *__restrict__ list, const int *__restrict__ count) {
    const int n = *count;
    T M[THREAD_SMAX * THREAD_SMAX], V[THREAD_SMAX * THREAD_SMAX], rhs[THREAD_SMAX], z[THREAD_SMAX], L[THREAD_SMAX];
    ThreadTeam tm;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        if (SHARED) solve_rows_shared(tm, a, list[t], M, rhs, z, L, V);
        else solve_row(tm, a, list[t], M, rhs, z, L, V);
}

template <class T, bool SHARED>
__global__ void __launch_bounds__(128) k_local_warp(LocalArgs a, const int *__restrict__ list, const int *__restrict__ count) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = *count;
    const int w = threadIdx.x >> 5;
    T *base = reinterpret_cast<T *>(smem) + (size_t)w * (2 * 32 * 32 + 3 * 32);
    T *M = base, *V = base + 32 * 32, *rhs = V + 32 * 32, *z = rhs + 32, *L = z + 32;
    WarpTeam tm;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int t = blockIdx.x * (blockDim.x >> 5) + w; t < n; t += nwarps) {
        if (SHARED) solve_rows_shared(tm, a, list[t], M, rhs, z, L, V);
        else solve_row(tm, a, list[t], M, rhs, z, L, V);
    }
}

template <class T, bool SHARED>
__global__ void __launch_bounds__(256) k_local_cta(LocalArgs a, const int *__restrict__ list, const int *__restrict__ count,
                                                   T *__restrict__ scratch, int smax) {
    __shared__ double red[64];
    const int n = *count;
    const size_t per = (size_t)2 * smax * smax + 3 * (size_t)smax;
    T *M = scratch + per * blockIdx.x;
    T *V = M + (size_t)smax * smax, *rhs = V + (size_t)smax * smax, *z = rhs + smax, *L = z + smax;
    CtaTeam tm{red};
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        if (SHARED) solve_rows_shared(tm, a, list[t], M, rhs, z, L, V);
        else solve_row(tm, a, list[t], M, rhs, z, L, V);
    }
}

constexpr int BIN_THREADS = 256;

// Each block bins a contiguous chunk of the systems: pass 1 counts the chunk's systems per bin (and the largest
// size) in shared memory and reserves the block's room in every list with one global atomic per bin; pass 2
// writes the chunk's systems, tile by tile in index order, at ballot-and-prefix positions inside that room.
// The lists are ordered by chunk reservation, which varies from run to run; which team solves which system
// does not change its result.
__global__ void __launch_bounds__(BIN_THREADS) k_local_bin(int nc, int group, const int *__restrict__ nb_rp,
                                                           int *__restrict__ lists, int *__restrict__ counts,
                                                           int *__restrict__ smax, int tmax, int wmax) {
    __shared__ int s_cnt[3], s_base[3], s_max;
    __shared__ int s_warp[BIN_THREADS / 32][3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long per = ((long long)nc + gridDim.x - 1) / gridDim.x;
    const long long c0 = (long long)blockIdx.x * per, c1 = min((long long)nc, c0 + per);
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    int cnt0 = 0, cnt1 = 0, cnt2 = 0, mx = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += BIN_THREADS) {
        const int sz = nb_rp[c * group + 1] - nb_rp[c * group];
        cnt0 += sz <= tmax;
        cnt1 += sz > tmax && sz <= wmax;
        cnt2 += sz > wmax;
        mx = max(mx, sz);
    }
    cnt0 = __reduce_add_sync(0xffffffffu, cnt0);
    cnt1 = __reduce_add_sync(0xffffffffu, cnt1);
    cnt2 = __reduce_add_sync(0xffffffffu, cnt2);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) {
        if (cnt0) atomicAdd(&s_cnt[0], cnt0);
        if (cnt1) atomicAdd(&s_cnt[1], cnt1);
        if (cnt2) atomicAdd(&s_cnt[2], cnt2);
        if (mx) atomicMax(&s_max, mx);
    }
    __syncthreads();
    if (threadIdx.x < 3) s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]) : 0;
    if (threadIdx.x == 0 && s_max > 0) atomicMax(smax, s_max);
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    for (long long t0 = c0; t0 < c1; t0 += BIN_THREADS) {
        const long long c = t0 + threadIdx.x;
        const bool act = c < c1;
        const int sz = act ? nb_rp[c * group + 1] - nb_rp[c * group] : 0;
        const int b = sz <= tmax ? 0 : (sz <= wmax ? 1 : 2);
        unsigned m[3];
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            m[bb] = __ballot_sync(0xffffffffu, act && b == bb);
            if (lane == 0) s_warp[wid][bb] = __popc(m[bb]);
        }
        __syncthreads();
        if (act) {
            int off = s_base[b];
            for (int w = 0; w < wid; ++w) off += s_warp[w][b];
            lists[(size_t)b * nc + off + __popc(m[b] & below)] = (int)c;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            int tot = 0;
            for (int w = 0; w < BIN_THREADS / 32; ++w) tot += s_warp[w][threadIdx.x];
            s_base[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

void launch_local_bin(int nc, const int *nb_rp, int *lists, int *counts, int *smax, cudaStream_t s, int stride,
                      int tmax, int wmax) {
    if (nc <= 0) return;
    tmax = tmax < 0 ? 0 : (tmax > THREAD_SMAX ? THREAD_SMAX : tmax);
    wmax = wmax < tmax ? tmax : (wmax > 32 ? 32 : wmax);
    k_local_bin<<<grid_for(nc, BIN_THREADS, device_sms() * 8), BIN_THREADS, 0, s>>>(nc, stride, nb_rp, lists, counts,
                                                                                     smax, tmax, wmax);
    count_launch();
}

template <class T, bool SHARED>
static void local_solves_t(const LocalArgs &a, int nc, const int *lists, const int *counts_dev, const int counts_host[3],
                           int smax, void *scratch, cudaStream_t s, const LocalSchedule &sch) {
    if (counts_host[0] > 0) {
        const int tb = sch.thread_tb > 0 ? sch.thread_tb : 128;
        k_local_thread<T, SHARED><<<grid_for(counts_host[0], tb), tb, 0, s>>>(a, lists, counts_dev);
        count_launch();
    }
    if (counts_host[1] > 0) {
        const size_t bytes = 4 * sizeof(T) * (2 * 32 * 32 + 3 * 32);
        cudaFuncSetAttribute(k_local_warp<T, SHARED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        const int cap = device_sms() * (sch.warp_blocks_per_sm > 0 ? sch.warp_blocks_per_sm : 8);
        k_local_warp<T, SHARED><<<grid_for(counts_host[1], 4, cap), 128, bytes, s>>>(a, lists + nc, counts_dev + 1);
        count_launch();
    }
    if (counts_host[2] > 0) {
        const int g = counts_host[2] < LOCAL_CTA_GRID ? counts_host[2] : LOCAL_CTA_GRID;
        k_local_cta<T, SHARED><<<g, 256, 0, s>>>(a, lists + 2 * (size_t)nc, counts_dev + 2, (T *)scratch, smax);
        count_launch();
    }
}

cudaError_t launch_local_solves(const LocalArgs &a, int nc, const int *lists, const int *counts_dev,
                                const int counts_host[3], int smax, bool fp32, void *scratch, cudaStream_t s,
                                const LocalSchedule &sch) {
    const bool shared = a.rows_per > 1;
    if (fp32) {
        if (shared) local_solves_t<float, true>(a, nc, lists, counts_dev, counts_host, smax, scratch, s, sch);
        else local_solves_t<float, false>(a, nc, lists, counts_dev, counts_host, smax, scratch, s, sch);
    } else {
        if (shared) local_solves_t<double, true>(a, nc, lists, counts_dev, counts_host, smax, scratch, s, sch);
        else local_solves_t<double, false>(a, nc, lists, counts_dev, counts_host, smax, scratch, s, sch);
    }
    return cudaGetLastError();
}

size_t local_cta_scratch_bytes(int smax, bool fp32) {
    size_t el = fp32 ? sizeof(float) : sizeof(double);
    return el * ((size_t)2 * smax * smax + 3 * (size_t)smax) * LOCAL_CTA_GRID;
}

// ---------------------------------------------------------------------------------------
// one-point interpolation (Sec. 4): F row j -> 1 at its strongest C connection
// (largest -a_jc, or |a_jc| in abs mode; ties -> smallest c); C rows -> identity.
// ---------------------------------------------------------------------------------------
__global__ void k_onepoint_choose(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                  const double *__restrict__ val, const uint8_t *__restrict__ mask,
                                  const int8_t *__restrict__ cf, const int *__restrict__ cidx, int absmode,
                                  int *__restrict__ choice, int *__restrict__ cnt) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int ch = -1;
        if (cf[j] == CF_C) {
            ch = cidx[j];
        } else {
            double bk = 0.0;
            int best = -1;
            for (int k = rp[j]; k < rp[j + 1]; ++k) {
                int c = col[k];
                if (!mask[k] || cf[c] != CF_C) continue;
                double key = absmode ? fabs(val[k]) : -val[k];
                if (best < 0 || key > bk) { best = c; bk = key; }
            }
            if (best >= 0) ch = cidx[best];
        }
        choice[j] = ch;
        cnt[j] = ch >= 0;
    }
}

__global__ void k_onepoint_fill(int n, const int *__restrict__ choice, const int *__restrict__ prp,
                                int *__restrict__ pcol, double *__restrict__ pval, float *__restrict__ pval32) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (choice[j] < 0) continue;
        pcol[prp[j]] = choice[j];
        pval[prp[j]] = 1.0;
        if (pval32) pval32[prp[j]] = 1.0f;
    }
}

void launch_onepoint(int phase, const DCsr &A, const uint8_t *mask, const int8_t *cf, const int *cidx, int absmode,
                     int *choice, int *cnt, DCsr *P, cudaStream_t s) {
    if (phase == 0)
        k_onepoint_choose<<<grid_for(A.nr, 256), 256, 0, s>>>(A.nr, A.rp, A.col, A.val, mask, cf, cidx, absmode, choice, cnt);
    else
        k_onepoint_fill<<<grid_for(A.nr, 256), 256, 0, s>>>(A.nr, choice, P->rp, P->col, P->val, P->val32);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// DG block-diagonal scaling (Sec. 4.2.1): A -> D_B^{-1} A with bs x bs diagonal blocks.
// D_B^{-1} from LU with partial pivoting (same rules as above, multipliers kept, rows of
// L swapped with M) applied to unit vectors; row r of block K of the result is
// sum_t Dinv[r][t] * A[K t, :] (fma, ascending t) on the union of the block rows'
// off-block columns, and the diagonal block becomes the exact identity.
// ---------------------------------------------------------------------------------------
// Walk the BS rows of a block in merged column order, skipping the block's own columns.
// For every column j of the union, vals[t] = A[r0 + t][j] (0 when not stored). BS is a
// compile-time constant so that the cursors stay in registers.
template <int BS>
struct BlockMerge {
    const int *rp, *col;
    const double *val;
    int r0;
    int pos[BS], end[BS];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int t = 0; t < BS; ++t) {
            pos[t] = rp[r0 + t];
            end[t] = rp[r0 + t + 1];
            skip(t);
        }
    }
    __device__ __forceinline__ void skip(int t) {
        while (pos[t] < end[t] && col[pos[t]] >= r0 && col[pos[t]] < r0 + BS) ++pos[t];
    }
    // next union column (or -1); fills vals[t]
    __device__ __forceinline__ int next(double *vals) {
        int c[BS];
        int j = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < BS; ++t) {
            c[t] = pos[t] < end[t] ? col[pos[t]] : 0x7fffffff;
            j = min(j, c[t]);
        }
        if (j == 0x7fffffff) return -1;
#pragma unroll
        for (int t = 0; t < BS; ++t) {
            if (c[t] == j) {
                if (vals) vals[t] = val[pos[t]];
                ++pos[t];
                skip(t);
            } else if (vals) {
                vals[t] = 0.0;
            }
        }
        return j;
    }
};

template <int BS>
__global__ void k_block_count(int nblk, const int *__restrict__ rp, const int *__restrict__ col, int *__restrict__ rowcnt) {
    for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < nblk; K += gridDim.x * blockDim.x) {
        BlockMerge<BS> m{rp, col, nullptr, K * BS};
        m.init();
        int nu = 0;
        while (m.next(nullptr) >= 0) ++nu;
#pragma unroll
        for (int r = 0; r < BS; ++r) rowcnt[K * BS + r] = nu + 1;
    }
}

// One thread per block. D_B^{-1}: in-place LU with partial pivoting (multipliers stored below
// the diagonal, whole rows swapped, so the rows of L move with those of U), then each unit
// vector through it. The row swaps run over compile-time row indices with predicates, so M
// stays in registers. Then the block's rows are merged once and the BS output rows written:
// the off-block union columns below the block, the identity entry, the union columns above.
constexpr int BLK_THREADS = 64;

template <int BS>
__global__ void __launch_bounds__(BLK_THREADS) k_block_scale(int nblk, const int *__restrict__ rp,
                                                             const int *__restrict__ col, const double *__restrict__ val,
                                                             const int *__restrict__ orp, int *__restrict__ ocol,
                                                             double *__restrict__ oval, double *__restrict__ dinv_out,
                                                             int *status) {
    // the LU factors live in shared memory, thread-major (entry q of this thread at q * BLK_THREADS)
    __shared__ double Msh[BS * BS * BLK_THREADS];
    for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < nblk; K += gridDim.x * blockDim.x) {
        const int r0 = K * BS;
        double Di[BS * BS];
        {
            struct Rows {
                double *p;
                __device__ double &operator[](int q) const { return p[q * BLK_THREADS]; }
            } M{Msh + threadIdx.x};
            int perm[BS];
#pragma unroll
            for (int r = 0; r < BS; ++r) {
                perm[r] = r;
#pragma unroll
                for (int c = 0; c < BS; ++c) M[r * BS + c] = 0.0;
                for (int k = rp[r0 + r]; k < rp[r0 + r + 1]; ++k) {
                    const int j = col[k];
                    if (j >= r0 + BS) break;
                    const double v = val[k];
#pragma unroll
                    for (int c = 0; c < BS; ++c)
                        if (j == r0 + c) M[r * BS + c] = v;
                }
            }
            double mx = 0.0;
#pragma unroll
            for (int q = 0; q < BS * BS; ++q) mx = fmax(mx, fabs(M[q]));
            const double thr = __dmul_rn(__dmul_rn((double)BS, 0x1.0p-52), mx);
            bool bad = mx == 0.0;
#pragma unroll
            for (int k = 0; k < BS; ++k) {
                int piv = k;
                double best = fabs(M[k * BS + k]);
#pragma unroll
                for (int r = k + 1; r < BS; ++r)
                    if (fabs(M[r * BS + k]) > best) { best = fabs(M[r * BS + k]); piv = r; }
                if (best <= thr) bad = true;
#pragma unroll
                for (int r = k + 1; r < BS; ++r)
                    if (r == piv) {
#pragma unroll
                        for (int c = 0; c < BS; ++c) {
                            const double t = M[k * BS + c]; M[k * BS + c] = M[r * BS + c]; M[r * BS + c] = t;
                        }
                        const int t = perm[k]; perm[k] = perm[r]; perm[r] = t;
                    }
#pragma unroll
                for (int r = k + 1; r < BS; ++r) {
                    const double l = __ddiv_rn(M[r * BS + k], M[k * BS + k]);
                    M[r * BS + k] = l;
#pragma unroll
                    for (int c = k + 1; c < BS; ++c) M[r * BS + c] = __fma_rn(-l, M[k * BS + c], M[r * BS + c]);
                }
            }
            if (bad) {
                set_status(status, LAIR_ERR_ZERO_DIAGONAL);
                continue;
            }
#pragma unroll
            for (int t = 0; t < BS; ++t) {
                double rhs[BS];
#pragma unroll
                for (int r = 0; r < BS; ++r) rhs[r] = (perm[r] == t) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < BS; ++k)
#pragma unroll
                    for (int r = k + 1; r < BS; ++r) rhs[r] = __fma_rn(-M[r * BS + k], rhs[k], rhs[r]);
#pragma unroll
                for (int c = BS - 1; c >= 0; --c) {
                    const double zc = __ddiv_rn(rhs[c], M[c * BS + c]);
                    Di[c * BS + t] = zc;
#pragma unroll
                    for (int r = 0; r < c; ++r) rhs[r] = __fma_rn(-M[r * BS + c], zc, rhs[r]);
                }
            }
        }
        double *dst = dinv_out + (size_t)K * BS * BS;
#pragma unroll
        for (int q = 0; q < BS * BS; ++q) dst[q] = Di[q];

        BlockMerge<BS> m{rp, col, val, r0};
        m.init();
        const int p0 = orp[r0];        // every row of the block has the same length
        const int len = orp[r0 + 1] - p0;
        int u = 0;
        bool below = true;
        double a[BS];
        for (;;) {
            const int j = m.next(a);
            if (below && (j < 0 || j > r0)) {
#pragma unroll
                for (int rr = 0; rr < BS; ++rr) {
                    ocol[p0 + rr * len + u] = r0 + rr;
                    oval[p0 + rr * len + u] = 1.0;
                }
                ++u;
                below = false;
            }
            if (j < 0) break;
#pragma unroll
            for (int rr = 0; rr < BS; ++rr) {
                double acc = 0.0;
#pragma unroll
                for (int t = 0; t < BS; ++t) acc = __fma_rn(Di[rr * BS + t], a[t], acc);
                ocol[p0 + rr * len + u] = j;
                oval[p0 + rr * len + u] = acc;
            }
            ++u;
        }
    }
}

__global__ void k_block_apply(int nblk, int bs, const double *__restrict__ dinv, const double *__restrict__ b,
                              double *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nblk * bs; e += gridDim.x * blockDim.x) {
        int K = e / bs, r = e % bs;
        double acc = 0.0;
        for (int t = 0; t < bs; ++t) acc = __fma_rn(dinv[(size_t)K * bs * bs + r * bs + t], b[K * bs + t], acc);
        out[e] = acc;
    }
}

template <int BS>
static void block_count_bs(int nblk, const DCsr &A, int *rowcnt, cudaStream_t s) {
    k_block_count<BS><<<grid_for(nblk, 128), 128, 0, s>>>(nblk, A.rp, A.col, rowcnt);
}
template <int BS>
static void block_scale_bs(int nblk, const DCsr &A, const DCsr &out, double *dinv, int *status, cudaStream_t s) {
    k_block_scale<BS><<<grid_for(nblk, BLK_THREADS), BLK_THREADS, 0, s>>>(nblk, A.rp, A.col, A.val, out.rp, out.col, out.val, dinv, status);
}

#define LAIR_BS_CASES(F, ...)          \
    switch (bs) {                      \
    case 2: F<2>(__VA_ARGS__); break;  \
    case 3: F<3>(__VA_ARGS__); break;  \
    case 4: F<4>(__VA_ARGS__); break;  \
    case 5: F<5>(__VA_ARGS__); break;  \
    case 6: F<6>(__VA_ARGS__); break;  \
    case 7: F<7>(__VA_ARGS__); break;  \
    case 8: F<8>(__VA_ARGS__); break;  \
    default: return false;             \
    }

bool launch_block_count(int nblk, int bs, const DCsr &A, int *rowcnt, cudaStream_t s) {
    LAIR_BS_CASES(block_count_bs, nblk, A, rowcnt, s)
    count_launch();
    return true;
}

bool launch_block_fill(int nblk, int bs, const DCsr &A, const DCsr &out, double *dinv, int *status, cudaStream_t s) {
    LAIR_BS_CASES(block_scale_bs, nblk, A, out, dinv, status, s)
    count_launch();
    return true;
}

void launch_block_apply(int nblk, int bs, const double *dinv, const double *b, double *out, cudaStream_t s) {
    k_block_apply<<<grid_for((long long)nblk * bs, 256), 256, 0, s>>>(nblk, bs, dinv, b, out);
    count_launch();
}

// ---------------------------------------------------------------------------------------
// Allocation-free batch of local solves.
//
// Some callers cannot allocate device memory at the point where they need a solve: code
// running while a CUDA graph is being captured or replayed, callers under a memory
// budget that has already been handed out to other pools, or host threads that must not
// touch the allocator for latency reasons. For them lair_local_solve_noalloc solves
// caller-provided dense local systems with the same CTA-team LU / least-squares routine as
// the set-up (so results are bit-identical to the restriction rows lair_setup produces),
// but its working storage is the fixed device array below instead of memory from
// cudaMalloc. Every GPU that loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------------------
constexpr int NOALLOC_SMAX = 64;        // largest system size accepted
constexpr int NOALLOC_SLOTS = 152;      // CTAs working at once, one scratch slot each
constexpr size_t NOALLOC_SLOT = (size_t)2 * NOALLOC_SMAX * NOALLOC_SMAX + 3 * NOALLOC_SMAX;   // doubles per slot
constexpr int NOALLOC_MAX_DEVICES = 64;

// 152 slots x 8384 doubles = 10,194,944 bytes. Host code must not pass this name to a
// kernel: on the host it only stands for the symbol; its device address is looked up below.
static __device__ __align__(256) double g_local_scratch[NOALLOC_SLOTS * NOALLOC_SLOT];

__global__ void __launch_bounds__(256) k_local_cta_dense(long long nsys, int s, const double *__restrict__ M,
                                                         const double *__restrict__ rhs, double *__restrict__ z,
                                                         uint8_t *__restrict__ ls, double *__restrict__ scratch) {
    __shared__ double red[64];
    CtaTeam tm{red};
    double *Mw = scratch + NOALLOC_SLOT * blockIdx.x;      // this CTA's slot: M, V, rhs, z, multipliers
    double *V = Mw + (size_t)s * s, *rw = V + (size_t)s * s, *zw = rw + s, *Lw = zw + s;
    for (long long k = blockIdx.x; k < nsys; k += gridDim.x) {
        const double *Mk = M + (size_t)k * s * s, *bk = rhs + (size_t)k * s;
        // every value the solve reads is written here first: nothing of an earlier call is used
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) Mw[e] = Mk[e];
        for (int e = threadIdx.x; e < s; e += blockDim.x) rw[e] = bk[e];
        __syncthreads();
        int singular = lu_solve(tm, s, Mw, rw, zw, Lw);
        if (singular) {
            for (int e = threadIdx.x; e < s * s; e += blockDim.x) Mw[e] = Mk[e];
            for (int e = threadIdx.x; e < s; e += blockDim.x) rw[e] = bk[e];
            __syncthreads();
            jacobi_ls(tm, s, Mw, rw, V, zw);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < s; e += blockDim.x) z[(size_t)k * s + e] = zw[e];
        if (threadIdx.x == 0 && ls) ls[k] = (uint8_t)singular;
        __syncthreads();
    }
}

}  // namespace lair

#include <mutex>

namespace {
// device address of g_local_scratch for each device, looked up once with that device current
double *g_noalloc_ptr[lair::NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mutex;
}  // namespace

extern "C" lair_status lair_local_solve_noalloc(int64_t nsys, int32_t s, const double *M, const double *rhs, double *z,
                                                uint8_t *ls_flag, void *stream) {
    using namespace lair;
    if (nsys < 0 || (nsys > 0 && (!M || !rhs || !z))) return LAIR_ERR_INVALID_ARG;
    if (s < 1) return LAIR_ERR_INVALID_ARG;
    if (s > NOALLOC_SMAX) return LAIR_ERR_UNSUPPORTED;        // the scratch slots hold systems up to 64 x 64
    if (nsys == 0) return LAIR_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return LAIR_ERR_CUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_local_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return LAIR_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    // an error left pending by earlier CUDA calls of this thread is reported as it is (not cleared), so
    // that a failure after the launch below belongs to this launch
    if (cudaPeekAtLastError() != cudaSuccess) return LAIR_ERR_CUDA;
    const int grid = nsys < NOALLOC_SLOTS ? (int)nsys : NOALLOC_SLOTS;
    k_local_cta_dense<<<grid, 256, 0, (cudaStream_t)stream>>>((long long)nsys, s, M, rhs, z, ls_flag, scratch);
    return cudaGetLastError() == cudaSuccess ? LAIR_OK : LAIR_ERR_CUDA;
}

