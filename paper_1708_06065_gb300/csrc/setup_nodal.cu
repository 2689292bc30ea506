// setup_nodal.cu -- the nodal (block) hierarchy: Sec. 3.1 forms the local system with k x k blocks,
// Sec. 4.2.1 names approach (iii), strength, C/F splitting and transfer operators computed by block.
// Node I holds the k consecutive unknowns kI .. kI + k - 1 (k <= 8). The kernels here build the matrix
// of block Frobenius norms (on which the scalar strength, splitting, neighbourhood and one-point kernels
// then run), expand node labels and node sets to unknowns, write block one-point interpolation, lump
// whole blocks, and apply the inverse diagonal blocks to the cycle's right-hand sides (block Jacobi).
#include "setup_kernels.cuh"

namespace lair {

// the k rows of node I (row r spans [rp[r], rp[r] + len[r]) with len, else [rp[r], rp[r + 1])), walked in
// ascending block column col / k
struct NodeRows {
    int pos[NODAL_MAX], end[NODAL_MAX];
    int k;
    __device__ void init(const int *rp, const int *len, int I, int kk) {
        k = kk;
#pragma unroll
        for (int t = 0; t < NODAL_MAX; ++t) {
            const int r = I * kk + t;
            pos[t] = t < kk ? rp[r] : 0;
            end[t] = t < kk ? (len ? rp[r] + len[r] : rp[r + 1]) : 0;
        }
    }
    __device__ int next_block(const int *col) const {
        int J = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < NODAL_MAX; ++t)
            if (pos[t] < end[t]) J = min(J, col[pos[t]] / k);
        return J == 0x7fffffff ? -1 : J;
    }
    // ||block J||_F: fma(a, a, .) from 0 in ascending row, then ascending column; advances past the block
    // and records each row's first entry of the block in st and its entry count in nt
    __device__ double block_norm(const int *col, const double *val, int J, int *st, int *nt) {
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < NODAL_MAX; ++t) {
            if (st) st[t] = pos[t];
            int c = 0;
            while (pos[t] < end[t] && col[pos[t]] / k == J) {
                acc = __fma_rn(val[pos[t]], val[pos[t]], acc);
                ++pos[t];
                ++c;
            }
            if (nt) nt[t] = c;
        }
        return __dsqrt_rn(acc);
    }
};

// ---- node matrix: b_IJ = ||A_IJ||_F --------------------------------------------------------------
__global__ void k_node_matrix(int phase, int N, int k, const int *__restrict__ rp, const int *__restrict__ col,
                              const double *__restrict__ val, int *__restrict__ cnt, const int *__restrict__ brp,
                              int *__restrict__ bcol, double *__restrict__ bval) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
        NodeRows w;
        w.init(rp, nullptr, I, k);
        int p = phase ? brp[I] : 0, c = 0;
        for (int J; (J = w.next_block(col)) >= 0;) {
            const double nb = w.block_norm(col, val, J, nullptr, nullptr);
            if (phase) {
                bcol[p] = J;
                bval[p] = nb;
                ++p;
            }
            ++c;
        }
        if (!phase) cnt[I] = c;
    }
}

void launch_node_matrix(int phase, int N, int k, const DCsr &A, int *cnt, const DCsr *B, cudaStream_t s) {
    if (N <= 0) return;
    k_node_matrix<<<grid_for(N, 128), 128, 0, s>>>(phase, N, k, A.rp, A.col, A.val, cnt, B ? B->rp : nullptr,
                                                   B ? B->col : nullptr, B ? B->val : nullptr);
    count_launch();
}

// ---- node labels and masks to unknowns ----------------------------------------------------------------
// mask[q] for entry q of A = the node mask of its block; cf[i] = cfB[i / k]
__global__ void k_node_expand(int n, int k, const int *__restrict__ rp, const int *__restrict__ col,
                              const int *__restrict__ brp, const int *__restrict__ bcol,
                              const uint8_t *__restrict__ bmask, uint8_t *__restrict__ mask,
                              const int8_t *__restrict__ cfB, int8_t *__restrict__ cf) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int I = i / k, b0 = brp[I], nb = brp[I + 1] - b0;
        if (cf) cf[i] = cfB[I];
        if (!mask) continue;
        for (int q = rp[i]; q < rp[i + 1]; ++q) {
            const int J = col[q] / k;
            int lo = 0, hi = nb - 1, at = -1;
            while (lo <= hi) {
                const int m = (lo + hi) >> 1, v = bcol[b0 + m];
                if (v == J) { at = m; break; }
                if (v < J) lo = m + 1; else hi = m - 1;
            }
            mask[q] = at >= 0 ? bmask[b0 + at] : 0;
        }
    }
}

void launch_node_expand(int n, int k, const DCsr &A, const DCsr &B, const uint8_t *bmask, uint8_t *mask,
                        const int8_t *cfB, int8_t *cf, cudaStream_t s) {
    if (n <= 0) return;
    k_node_expand<<<grid_for(n, 256), 256, 0, s>>>(n, k, A.rp, A.col, B.rp, B.col, bmask, mask, cfB, cf);
    count_launch();
}

// ---- node sets to rows of unknowns ------------------------------------------------------------------------
// coarse node q with node set N_q gives the rows c = kq + t: every unknown of N_q plus the unknown
// k * cptsB[q] + t itself, ascending (phase 0: lengths; phase 1: the rows at orp)
__global__ void k_node_rows(int phase, int NC, int k, const int *__restrict__ nrp, const int *__restrict__ ncol,
                            const int *__restrict__ cptsB, int *__restrict__ len, const int *__restrict__ orp,
                            int *__restrict__ ocol) {
    const int nc = NC * k;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int q = c / k, t = c % k;
        if (!phase) {
            len[c] = k * (nrp[q + 1] - nrp[q]) + 1;
            continue;
        }
        const int self = k * cptsB[q] + t;
        int p = orp[c];
        bool placed = false;
        for (int a = nrp[q]; a < nrp[q + 1]; ++a)
            for (int u = 0; u < k; ++u) {
                const int v = k * ncol[a] + u;
                if (!placed && self < v) {
                    ocol[p++] = self;
                    placed = true;
                }
                ocol[p++] = v;
            }
        if (!placed) ocol[p] = self;
    }
}

void launch_node_rows(int phase, int NC, int k, const int *nrp, const int *ncol, const int *cptsB, int *len,
                      const int *orp, int *ocol, cudaStream_t s) {
    if (NC <= 0) return;
    k_node_rows<<<grid_for((long long)NC * k, 256), 256, 0, s>>>(phase, NC, k, nrp, ncol, cptsB, len, orp, ocol);
    count_launch();
}

// ---- block one-point interpolation: the k x k identity at the node's chosen coarse node -------------------
__global__ void k_onepoint_nodal(int phase, int n, int k, const int *__restrict__ choiceB, int *__restrict__ cnt,
                                 const int *__restrict__ prp, int *__restrict__ pcol, double *__restrict__ pval,
                                 float *__restrict__ pval32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ch = choiceB[i / k];
        if (!phase) {
            cnt[i] = ch >= 0;
            continue;
        }
        if (ch < 0) continue;
        pcol[prp[i]] = k * ch + i % k;
        pval[prp[i]] = 1.0;
        if (pval32) pval32[prp[i]] = 1.0f;
    }
}

void launch_onepoint_nodal(int phase, int n, int k, const int *choiceB, int *cnt, const DCsr *P, cudaStream_t s) {
    if (n <= 0) return;
    k_onepoint_nodal<<<grid_for(n, 256), 256, 0, s>>>(phase, n, k, choiceB, cnt, P ? P->rp : nullptr,
                                                      P ? P->col : nullptr, P ? P->val : nullptr,
                                                      P ? P->val32 : nullptr);
    count_launch();
}

// ---- lumping by block (Sec. 3.3 with k x k blocks) -----------------------------------------------------------
// Node row I: every block J != I with ||K_IJ||_F < theta_D max_J ||K_IJ||_F (diagonal block included) is
// removed and added entrywise to the diagonal block, k_{i, kI+u} += k_{i, kJ+u}, in ascending J from
// k_{i, kI+u}. phase 0: kept entries per row into cnt; phase 1: the kept rows at orp.
__global__ void k_lump_nodal(int phase, int N, int k, const int *__restrict__ rp, const int *__restrict__ len,
                             const int *__restrict__ col, const double *__restrict__ val, double tol,
                             int *__restrict__ cnt, const int *__restrict__ orp, int *__restrict__ ocol,
                             double *__restrict__ oval, int *status) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
        NodeRows w;
        w.init(rp, len, I, k);
        double m = 0.0;
        for (int J; (J = w.next_block(col)) >= 0;) m = fmax(m, w.block_norm(col, val, J, nullptr, nullptr));
        const double thr = __dmul_rn(tol, m);
        int st[NODAL_MAX], nt[NODAL_MAX];
        if (!phase) {
            int c[NODAL_MAX];
#pragma unroll
            for (int t = 0; t < NODAL_MAX; ++t) c[t] = 0;
            w.init(rp, len, I, k);
            for (int J; (J = w.next_block(col)) >= 0;) {
                const double nb = w.block_norm(col, val, J, nullptr, nt);
                if (J == I || !(nb < thr)) {
#pragma unroll
                    for (int t = 0; t < NODAL_MAX; ++t) c[t] += nt[t];
                }
            }
            for (int t = 0; t < k; ++t) cnt[I * k + t] = c[t];
            continue;
        }
        // the diagonal block's values and which of them are stored
        double d[NODAL_MAX * NODAL_MAX];
        unsigned has[NODAL_MAX];
        int o[NODAL_MAX];
        for (int t = 0; t < k; ++t) {
            has[t] = 0u;
            o[t] = orp[I * k + t];
        }
        w.init(rp, len, I, k);
        for (int t = 0; t < k; ++t)
            for (int q = w.pos[t]; q < w.end[t]; ++q)
                if (col[q] / k == I) {
                    d[t * NODAL_MAX + col[q] % k] = val[q];
                    has[t] |= 1u << (col[q] % k);
                }
        for (int J; (J = w.next_block(col)) >= 0;) {
            const double nb = w.block_norm(col, val, J, st, nt);
            const bool kept = J == I || !(nb < thr);
            for (int t = 0; t < k; ++t)
                for (int q = st[t]; q < st[t] + nt[t]; ++q) {
                    if (kept) {
                        ocol[o[t]] = col[q];
                        oval[o[t]] = val[q];
                        ++o[t];
                    } else {
                        const int u = col[q] % k;
                        if (!((has[t] >> u) & 1u)) set_status(status, LAIR_ERR_INVALID_ARG);
                        else d[t * NODAL_MAX + u] = __dadd_rn(d[t * NODAL_MAX + u], val[q]);
                    }
                }
        }
        for (int t = 0; t < k; ++t)
            for (int p = orp[I * k + t]; p < o[t]; ++p)
                if (ocol[p] / k == I) oval[p] = d[t * NODAL_MAX + ocol[p] % k];
    }
}

void launch_lump_nodal(int phase, int k, const DCsr &K, const int *len, double tol, int *cnt, const DCsr *out,
                       int *status, cudaStream_t s) {
    const int N = K.nr / k;
    if (N <= 0) return;
    k_lump_nodal<<<grid_for(N, 64), 64, 0, s>>>(phase, N, k, K.rp, len, K.col, K.val, tol, cnt,
                                                out ? out->rp : nullptr, out ? out->col : nullptr,
                                                out ? out->val : nullptr, status);
    count_launch();
}

// Lumping onto a kept block pattern (hierarchy refresh): row i of out keeps its columns; every other entry
// k_{i, kJ+u} of K is added to k_{i, kI+u}, in ascending column order.
__global__ void k_lump_nodal_kept(int n, int k, const int *__restrict__ rp, const int *__restrict__ len,
                                  const int *__restrict__ col, const double *__restrict__ val,
                                  const int *__restrict__ orp, const int *__restrict__ ocol, double *__restrict__ oval,
                                  int *status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int I = i / k, b = rp[i], e = len ? b + len[i] : rp[i + 1];
        const int t0 = orp[i], t1 = orp[i + 1];
        double d[NODAL_MAX];
        unsigned has = 0u;
        for (int q = b; q < e; ++q)
            if (col[q] / k == I) {
                d[col[q] % k] = val[q];
                has |= 1u << (col[q] % k);
            }
        int t = t0;
        for (int q = b; q < e; ++q) {
            const int j = col[q];
            if (t < t1 && ocol[t] == j) {
                if (j / k != I) oval[t] = val[q];
                ++t;
            } else {
                const int u = j % k;
                if (!((has >> u) & 1u)) set_status(status, LAIR_ERR_INVALID_ARG);
                else d[u] = __dadd_rn(d[u], val[q]);
            }
        }
        if (t != t1) set_status(status, LAIR_ERR_INVALID_ARG);
        for (int p = t0; p < t1; ++p)
            if (ocol[p] / k == I && ((has >> (ocol[p] % k)) & 1u)) oval[p] = d[ocol[p] % k];
    }
}

void launch_lump_nodal_kept(int k, const DCsr &K, const int *len, const DCsr &out, int *status, cudaStream_t s) {
    if (K.nr <= 0) return;
    k_lump_nodal_kept<<<grid_for(K.nr, 256), 256, 0, s>>>(K.nr, k, K.rp, len, K.col, K.val, out.rp, out.col, out.val,
                                                          status);
    count_launch();
}

// ---- block Jacobi right-hand side: out_I = D_I^{-1} b_I (fma from 0, ascending t) -----------------------------
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <class T>
__global__ void k_block_apply_t(int n, int k, const T *__restrict__ inv, const T *__restrict__ b, T *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int I = e / k, r = e % k;
        const T *row = inv + ((size_t)I * k + r) * k;
        T acc = T(0);
        for (int t = 0; t < k; ++t) acc = fma_t(row[t], b[I * k + t], acc);
        out[e] = acc;
    }
}

template <class T>
void block_apply_t(int n, int k, const T *inv, const T *b, T *out, cudaStream_t s) {
    if (n <= 0) return;
    k_block_apply_t<T><<<grid_for(n, 256, device_sms() * 8), 256, 0, s>>>(n, k, inv, b, out);
    count_launch();
}

template void block_apply_t<float>(int, int, const float *, const float *, float *, cudaStream_t);
template void block_apply_t<double>(int, int, const double *, const double *, double *, cudaStream_t);

}  // namespace lair
