// setup_kernels.cuh -- host-side entry points of the device kernels (internal).
#pragma once

#include "lair_internal.cuh"

namespace lair {

// sliced-ELL view of a subset of a matrix's rows (sell.cu)
struct SellView {
    int nrows = 0;
    int *slice_ptr = nullptr;   // nslices + 1 offsets, in entries
    int *col = nullptr;
    void *val = nullptr;        // float or double
    int *row = nullptr;         // view row -> matrix row
    void *dinv = nullptr;       // Jacobi diagonal per view row (sweep views), same type as val
    int tb = 0, grid = 0;       // launch schedule picked by the autotuner (0: 256 threads, grid capped at 16 blocks per SM)
    int rpt = 1;                // rows per thread (1 or 2: rows of two consecutive slices, same lane)
    // batched systems: the system of every slice (-1: rows of several systems) and the per-system run flags;
    // slices of a stopped system are skipped (their outputs keep older values). NULL: every slice runs.
    const int *slice_sys = nullptr;
    const uint8_t *run = nullptr;
    bool zero_stopped = false;  // products: write 0 to the rows of a stopped system's slices instead of skipping them
};

// ---- setup_graph.cu -------------------------------------------------------------------
constexpr int SMALL_SCAN_MAX = 65536;   // exclusive scans up to this length run in one CTA
// exclusive scan of m ints in one pass over many CTAs (decoupled look-back); state: scan_state_bytes(m) bytes
size_t scan_state_bytes(long long m);
cudaError_t launch_scan(long long m, const int *in, int *out, void *state, int *status, cudaStream_t s);
void small_scan(int m, const int *in, int *out, cudaStream_t s);
void launch_strength(const DCsr &A, double theta, int absmode, uint8_t *mask, int *cnt, cudaStream_t s);
void launch_graph_fill(const DCsr &A, const uint8_t *mask, const Graph &G, cudaStream_t s);
void launch_col_count(int nr, const int *rp, const int *col, int *cnt, cudaStream_t s);
void launch_transpose_scatter(int nr, const int *rp, const int *col, const double *val, const int *trp, int *cursor,
                              int *tcol, double *tval, cudaStream_t s);
void launch_sort_rows(int nr, const int *rp, int *col, double *val, int *lists, cudaStream_t s);
void launch_pmis_init(int n, const Graph &ST, uint64_t seed, double *w, int8_t *cf, cudaStream_t s);
// every grid-barrier wait of the cooperative PMIS kernel gives up after wait_polls polls (0: GRID_WAIT_POLLS)
constexpr long long GRID_WAIT_POLLS = 1ll << 22;
// lists: 2 n ints of scratch; ctl: 4 ints, zero
cudaError_t launch_pmis_all(int n, const Graph &S, const Graph &ST, double *w, int8_t *cf, int8_t *newc, int *lists,
                            int *ctl, int *status, int wait_polls, cudaStream_t s);
void launch_rs_count(const int2 *blocks, int nblocks, const Graph &S, int *maxcnt, cudaStream_t s);
// bucket-queue first pass: blocks of at most RSB_MAX_N points, lambda below nb <= 256 buckets, at most dl points
// whose lambda changes in one step
constexpr int RSB_MAX_N = 8192;
constexpr int RSB_MAX_DIRTY = 8192;
void launch_rs_degrees(const int2 *blocks, int nblocks, const Graph &S, const Graph &ST, int *out, cudaStream_t s);
// (levels of at most one block per SM stage the in-block graphs in shared memory; max_inblock: the largest
// in-block entry count of S)
cudaError_t launch_rs_bucket(const int2 *blocks, int nblocks, int Bmax, int nb, int dl, int max_inblock,
                             const Graph &S, const Graph &ST, int8_t *cf, int *status, cudaStream_t s);
size_t rsb_smem_bytes(int n, int nb, int dl);
cudaError_t launch_rs(int n, const int2 *blocks, int nblocks, int Bmax, int max_inblock, const Graph &S, const Graph &ST,
                      int8_t *cf, int *status, cudaStream_t s);
size_t rs_smem_bytes(int n, int max_inblock);
constexpr int RS_MAX_N = 32768;
void launch_cidx(int n, const int8_t *cf, int *flag, int *cidx, int *cpts, int phase, cudaStream_t s);
void launch_nb_bound(int nc, const int *cpts, const Graph &G, const int8_t *cf, int distance, int *ub, cudaStream_t s);
void launch_nb_fill(int nc, const int *cpts, const Graph &G, const int8_t *cf, int distance, const int *off, int *tmp,
                    int *cnt, cudaStream_t s);
void launch_nb_compact(int nc, const int *off, const int *tmp, const int *nb_rp, int *nb_col, cudaStream_t s);
// the sets of kept rows that hold their C point once each: row c of (rp, col) without cpts[c]
void launch_nb_from_rows(int nc, const int *rp, const int *col, const int *cpts, int *nb_rp, int *nb_col,
                         cudaStream_t s);
// one more distance: phase 0 writes the bound to cnt, phase 1 the sets at off (sizes in cnt)
void launch_nb_expand(int phase, int nc, const int *cpts, const Graph &G, const int8_t *cf, const int *nb_rp,
                      const int *nb_col, const int *off, int *tmp, int *cnt, cudaStream_t s);

// ---- setup_local.cu -------------------------------------------------------------------
struct LocalArgs {
    const int *cpts;      // C point of each coarse row
    const int *nb_rp;     // neighbourhoods, CSR over coarse rows
    const int *nb_col;
    const int *brp;       // the matrix B whose local systems are solved (A, or A^T for lAIP)
    const int *bcol;
    const double *bval;
    int *out_col;         // output rows: row c at nb_rp[c] + c, nb_rp[c+1]-nb_rp[c] + 1 entries
    double *out_val;
    float *out_val32;     // optional
    uint8_t *lsflag;      // optional, per coarse row
    int neumann_deg = -1; // >= 0: the Neumann series of that degree instead of the solve (nAIR, Sec. 3.2)
    int rows_per = 1;     // > 1: rows c = q * rows_per + t (t < rows_per) share one set; the lists hold q
};
constexpr int LOCAL_CTA_GRID = 152 * 2;
// bins of the local systems by size (s <= 6, <= 32, larger); with stride > 1 entry c of the lists is the group
// of rows c * stride .. c * stride + stride - 1 (one set), sized by its first row
// launch schedule of the local solves: systems of size s <= tmax go to one thread each, tmax < s <= wmax to
// one warp each, larger ones to one CTA each; grid caps and block size of those kernels. Every system is
// solved by the same sequence of operations whatever team takes it, so results do not depend on it.
constexpr int THREAD_SMAX = 6;    // largest system a thread team holds in registers
struct LocalSchedule {
    int tmax = THREAD_SMAX;       // 0..THREAD_SMAX
    int wmax = 32;                // tmax..32
    int warp_blocks_per_sm = 8;   // grid cap of the warp kernel (4 warps per block)
    int thread_tb = 128;          // threads per block of the thread kernel
};
void launch_local_bin(int nc, const int *nb_rp, int *lists, int *counts, int *smax, cudaStream_t s, int stride = 1,
                      int tmax = THREAD_SMAX, int wmax = 32);
cudaError_t launch_local_solves(const LocalArgs &a, int nc, const int *lists, const int *counts_dev,
                                const int counts_host[3], int smax, bool fp32, void *scratch, cudaStream_t s,
                                const LocalSchedule &sch = LocalSchedule());
size_t local_cta_scratch_bytes(int smax, bool fp32);
void launch_onepoint(int phase, const DCsr &A, const uint8_t *mask, const int8_t *cf, const int *cidx, int absmode,
                     int *choice, int *cnt, DCsr *P, cudaStream_t s);
// block sizes 2..8 (false for any other)
bool launch_block_count(int nblk, int bs, const DCsr &A, int *rowcnt, cudaStream_t s);
bool launch_block_fill(int nblk, int bs, const DCsr &A, const DCsr &out, double *dinv, int *status, cudaStream_t s);
void launch_block_apply(int nblk, int bs, const double *dinv, const double *b, double *out, cudaStream_t s);

// ---- setup_rap.cu ---------------------------------------------------------------------
struct SpgemmArgs {
    const int *xrp, *xcol;
    const double *xval;
    const int *yrp, *ycol;
    const double *yval;
    const int *off;       // upper-bound offsets (exclusive scan of ub), nr + 1
    int *tcol;            // staging, off[nr] entries
    double *tval;
    int *cnt;             // exact row lengths
    // fused third factor (one-point P: at most one entry per row); NULL for a plain product
    const int *prp = nullptr, *pcol = nullptr;
    const double *pval = nullptr;
    int pn = 0;                          // rows of P
    int *pmap_col = nullptr;             // scratch, pn entries: P's row as a direct map (thread-per-row fused kernel)
    double *pmap_val = nullptr;
};
constexpr int SPGEMM_CTA_GRID = 152;
constexpr int SPGEMM_BINS = 6;      // three warp bins by row bound, the CTA bin, two merge bins
constexpr int SPGEMM_BIN_CTA = 3;   // rows with a bound beyond the warp kernels
constexpr int SPGEMM_BIN_MERGE = 4; // rows of X with at most SPGEMM_MERGE_K entries (thread per row)
constexpr int SPGEMM_BIN_MERGE2 = 5; // rows of X with at most SPGEMM_MERGE_K2 entries (thread per row)
constexpr int SPGEMM_MERGE_K = 8;
constexpr int SPGEMM_MERGE_K2 = 32;
constexpr int SPGEMM_MERGE_MIN_ROWS = 65536;   // products with fewer rows use the warp kernels only
void launch_spgemm_ub(int nr, const int *xrp, const int *xcol, const int *yrp, int *ub, cudaStream_t s);
// merge: rows of X with at most SPGEMM_MERGE_K entries go to the thread-per-row merge bin; merge2: rows
// with at most SPGEMM_MERGE_K2 to the second merge bin (plain products only)
// (and, for the first merge bin, a bound of at most merge_ub_max products)
void launch_spgemm_classify(int nr, const int *off, const int *xrp, bool merge, bool merge2, int merge_ub_max,
                            int *lists, int *counts, int *ubmax, cudaStream_t s);
constexpr int SPGEMM_P1_CAP = 32;       // fused one-point merge: at most this many products per row
constexpr int SPGEMM_P1_THREADS = 128;  // threads per block (their result lists fill 48 KB of shared memory)
// true if every row of the product fits the fused one-point-P kernels (bins 0 and 1, the first merge bin)
bool spgemm_can_fuse(const int counts_host[SPGEMM_BINS]);
cudaError_t launch_spgemm_rows(const SpgemmArgs &g, int nr, const int *lists, const int *counts_dev,
                               const int counts_host[SPGEMM_BINS], int ubmax, int *skeys, double *svals, cudaStream_t s);
unsigned spgemm_big_cap(int ubmax);
void launch_copy_rows(int nr, const int *off, const int *tcol, const double *tval, DCsr &Z, cudaStream_t s);
// K's rows: rp[i] .. rp[i + 1], or rp[i] .. rp[i] + len[i] when len is given; rowst: 2 K.nr doubles (16-byte
// aligned) written by phase 0 and read by phase 1
void launch_lump(int phase, const DCsr &K, const int *len, double tol, int *cnt, double *rowst, const DCsr *out,
                 int *status, cudaStream_t s);
// ---- setup_nodal.cu: the nodal (block) hierarchy, nodes of k <= NODAL_MAX consecutive unknowns -------------
constexpr int NODAL_MAX = 8;
// phase 0: block columns per node into cnt; phase 1: B = the block Frobenius norms at B->rp
void launch_node_matrix(int phase, int N, int k, const DCsr &A, int *cnt, const DCsr *B, cudaStream_t s);
// per unknown: cf[i] = cfB[i / k] (cf may be NULL); per entry of A: mask = bmask of its block (mask may be NULL)
void launch_node_expand(int n, int k, const DCsr &A, const DCsr &B, const uint8_t *bmask, uint8_t *mask,
                        const int8_t *cfB, int8_t *cf, cudaStream_t s);
// node sets (NC coarse nodes) to rows of unknowns with the C unknown itself: phase 0 lengths, phase 1 rows
void launch_node_rows(int phase, int NC, int k, const int *nrp, const int *ncol, const int *cptsB, int *len,
                      const int *orp, int *ocol, cudaStream_t s);
// block one-point P from the node choice (coarse node or -1): phase 0 counts, phase 1 entries
void launch_onepoint_nodal(int phase, int n, int k, const int *choiceB, int *cnt, const DCsr *P, cudaStream_t s);
// lumping by block: phase 0 kept counts per row, phase 1 the rows of out
void launch_lump_nodal(int phase, int k, const DCsr &K, const int *len, double tol, int *cnt, const DCsr *out,
                       int *status, cudaStream_t s);
// lumping onto a kept block pattern (refresh)
void launch_lump_nodal_kept(int k, const DCsr &K, const int *len, const DCsr &out, int *status, cudaStream_t s);
// out = D^{-1} b with the k x k inverse diagonal blocks inv (row-major per node)
template <class T> void block_apply_t(int n, int k, const T *inv, const T *b, T *out, cudaStream_t s);

// the values of out (a kept pattern inside K's) from K: entries of K outside it are lumped to the diagonal
void launch_lump_kept(const DCsr &K, const int *len, const DCsr &out, int *status, cudaStream_t s);
void launch_dinv(const DCsr &A, double *dinv, float *dinv32, int *status, cudaStream_t s);
void launch_to_f32(long long n, const double *a, float *b, cudaStream_t s);
void launch_dense_setup(const DCsr &A, double *D, int *perm, double *Ainv, int *status, cudaStream_t s);

// ---- solve_kernels.cu -----------------------------------------------------------------
template <class T> void spmv(const DCsr &A, const T *x, T *y, cudaStream_t s);
template <class T>
void sweep(const DCsr &A, const int8_t *cf, int target, const T *dinv, const T *b, const T *x, T *xo, cudaStream_t s);
template <class T> void dense_apply(int n, const double *Ainv, const T *b, T *y, cudaStream_t s);
constexpr int RED_PARTS = 152 * 4;
void residual(const DCsr &A, const double *b, const double *x, double *r, float *r32, double *part, cudaStream_t s);
// the same over an FP64 sliced-ELL view of all rows (RED_PARTS block partials)
void sell_residual(const SellView &v, const double *b, const double *x, double *r, float *r32, double *part,
                   cudaStream_t s);
void multidot(int n, int m, const double *X, long long ldx, const double *y, double *part, double *out, double *acc,
              cudaStream_t s);
void finish_partials(int m, const double *part, double *out, cudaStream_t s);
void finish_partials_acc(int m, const double *part, double *out, double *acc, cudaStream_t s);
// one pass (1, 2 or 3) of CGS2 of w against the m <= 32 columns of X; block partials in part
void cgs_pass(int pass, int n, int m, const double *X, long long ldx, const double *h, double *w, double *part,
              cudaStream_t s);
void sub_combo(int n, int m, const double *X, long long ldx, const double *h, double *w, cudaStream_t s);
void add_combo(int n, int m, const double *Z, long long ldz, const double *y, double *x, cudaStream_t s);
void scale_by_norm(int n, const double *v, const double *nrm2, double *out, cudaStream_t s);
void d2f(int n, const double *a, float *b, cudaStream_t s);
void f2d(int n, const float *a, double *b, cudaStream_t s);
void axpy_f(int n, const float *e, double *x, cudaStream_t s);
void axpy_d(int n, const double *e, double *x, cudaStream_t s);
void grad_A(const DCsr &A, const double *lam, const double *x, double *g, cudaStream_t s);
void cf_stats(const DCsr &A, const int8_t *cf, unsigned long long *out4, cudaStream_t s);

// ---- sell.cu --------------------------------------------------------------------------
void launch_frows(int n, const int8_t *cf, const int *cscan, int *frows, cudaStream_t s);
// one view of a batch built together (see sell.cu)
struct SellDesc {
    const int *rows_in;      // matrix rows of the view in order (NULL: all rows)
    const int *rp, *col;     // the matrix
    const double *val, *dinv;
    int *row_out;            // view row -> matrix row (rows sorted by length inside windows)
    int nrows, win0, lin0, sl0, group;
    const int *seg;          // batched systems: first matrix row of every system (nseg + 1 entries)
    int nseg;                // (0: not batched)
    int *slice_sys;          // out: the system of every slice, -1 when its rows belong to several
    const int *slice_ptr;    // filled in before the fill pass
    int *scol;
    void *sval, *sdinv;
};
void launch_sell_prepare_multi(const SellDesc *d, int nd, int nwin, int nlin, int *cnt, unsigned long long *gsum,
                               cudaStream_t s);
void launch_sell_fill_multi(const SellDesc *d, int p0, int p1, int lin_beg, int lin_end, bool fp32, cudaStream_t s);
template <class T> void sell_spmv(const SellView &v, const T *x, T *y, cudaStream_t s);
template <class T>
void sell_sweep(const SellView &v, const int *copy, int ncopy, const T *b, const T *x, T *xo, cudaStream_t s);
// x = P x_c for a P with at most one entry per row, every entry 1 (one-point interpolation), from its dense
// column array (-1: no entry), which launch_p1_cols builds from P's CSR
// blk_sys / run (batched systems, else NULL): the system of every 32-row block (-1: several) and the run flags;
// blocks of stopped systems are skipped
template <class T>
void p1_interp(int n, const int *p1col, const int *blk_sys, const uint8_t *run, const T *xc, T *x, cudaStream_t s);
// the bottom of the V-cycle in one CTA (sell.cu): levels of at most BOTTOM_ROWS rows. A level: R restricts b to the
// next level, P interpolates (sliced ELL, or the one-point column array p1col when set), AF / AC sweep the F / C
// rows while crows / frows (nc / n - nc of them) are copied; the coarsest: x = Ainv b
template <class T> struct BottomLevel {
    int n = 0, nc = 0;
    SellView R, P, AF, AC;
    const int *p1col = nullptr;
    const int *crows = nullptr, *frows = nullptr;
    T *b = nullptr, *x[2] = {nullptr, nullptr};
};
template <class T> struct BottomCoarse {
    int n = 0;
    const double *Ainv = nullptr;
    T *b = nullptr, *x = nullptr;
};
constexpr int BOTTOM_THREADS = 1024;
constexpr int BOTTOM_ROWS = 1024;
// lv: nl level descriptors in device memory; seq3: the sweep targets (CF_F / CF_C, -1 ends)
template <class T>
void cycle_bottom(const BottomLevel<T> *lv, int nl, const BottomCoarse<T> &cz, const int *seq3, cudaStream_t s);
// the system of every 32-row block of a level (seg: first row of every system, nseg + 1 entries)
void launch_blk_sys(int n, const int *seg, int nseg, int *blk_sys, cudaStream_t s);
void launch_p1_cols(int n, const int *rp, const int *col, int *p1col, cudaStream_t s);
// batched systems: per-system residual r = b - A x (rows seg[q]..seg[q+1]), its squared norm, optional FP32 copy
// Row tiles of a batch of systems: tile t is system tile[t].x, rows [tile[t].y, tile[t].z);
// the tiles of system q are first[q] .. first[q + 1] - 1; part holds SEG_TILE_PARTS doubles per tile.
struct SegTiles {
    const int4 *tile = nullptr;
    int ntiles = 0;
    const int *first = nullptr;
    int nseg = 0;
    double *part = nullptr;
    const uint8_t *active = nullptr;   // if set, tiles of systems with active[q] == 0 are skipped
};
constexpr int SEG_TILE = 4096;
constexpr int SEG_TILE_PARTS = 32;   // partial sums per tile: the dots of a CGS2 pass (restart <= 31)
void seg_residual(const DCsr &A, const SegTiles &st, const double *b, const double *x, double *r, float *r32,
                  double *norm2, cudaStream_t s);
void seg_norm2(const SegTiles &st, const double *v, double *norm2, cudaStream_t s);
template <class T>
void seg_axpy(const SegTiles &st, const uint8_t *active, const T *e, double *x, cudaStream_t s);
// one pass of the batched CGS2 step (see k_tile_cgs) over the m <= 31 columns of X, then the per-system sums:
// passes 1 and 2 write the m dots of every running system to out[q * hs + k] and add them to acc[q * hs + k],
// pass 3 writes the squared norm of the new w to out[q]
void seg_cgs_pass(const SegTiles &st, int pass, int m, const double *X, long long ldx, int hs, const double *h, double *w,
                  double *out, double *acc, cudaStream_t s);
void seg_add_combo(const SegTiles &st, const int *cnt, const double *Z, long long ldz, int hs, const double *y, double *x,
                   cudaStream_t s);
void seg_scale(const SegTiles &st, const double *v, const double *nrm2, double *out, cudaStream_t s);
void gather_int(int m, const int *idx, const int *src, int *out, cudaStream_t s);
// device-side state of the batched outer loops (one entry per system; see solve_kernels.cu)
constexpr int BATCH_HS = 32;      // Hessenberg column stride: restart lengths up to 31
struct BatchCtl {
    int nseg = 0, m = 0, hs = BATCH_HS, max_iter = 0;
    double tol = 0.0;
    const double *bn = nullptr;   // ||b_q|| (1 where b_q = 0)
    double *rl = nullptr;         // relative residual at the last check
    int *its = nullptr;           // cycles applied
    uint8_t *run = nullptr;       // still iterating (the tile kernels' active flags)
    uint8_t *done = nullptr;      // FGMRES: stopped for good
    int *jd = nullptr;            // FGMRES: steps of the current restart
    double *g = nullptr, *cs = nullptr, *sn = nullptr, *Hm = nullptr;   // FGMRES: (m + 1), m, m, (m + 1) m each
    int *nan = nullptr;           // set when a norm is not finite
};
void bat_bnorm(int nseg, const double *nrm2, double *bn, cudaStream_t s);
void bat_stat_check(const BatchCtl &c, const double *nrm2, int it, int *count, cudaStream_t s);
void bat_fg_restart(const BatchCtl &c, const double *nrm2, int *count, cudaStream_t s);
void bat_fg_givens(const BatchCtl &c, int j, const double *hsum, const double *nrm2w, int *count, cudaStream_t s);
void bat_fg_solve_y(const BatchCtl &c, double *y, cudaStream_t s);

}  // namespace lair
