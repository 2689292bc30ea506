// lair_solve.cu -- the outer FP64 iterations around the V-cycle: preconditioner application,
// stationary refinement and right-preconditioned FGMRES(m) with CGS2 for one system, and the
// batched systems' per-system refinement and FGMRES steered on the device (Sec. 4: V-cycles as
// the preconditioner of GMRES; the cycle in FP32 inside the FP64 outer iteration in mixed precision).
#include "lair_host.cuh"

namespace lair {

// z = M^{-1} v (one cycle, zero initial guess); v, z: FP64 device vectors of length n0
lair_status precond(lair_handle *h, Hier &H, const double *v, double *z) {
    Level &L = H.lev[0];
    const int n = L.A.nr;
    if (h->o.precision == LAIR_MIXED) {
        d2f(n, v, L.b32, h->s);
        CU(cudaGraphLaunch(H.graph, h->s));
        count_launch(H.graph_nodes);
        h->graph_pending = h->o.timing;
        f2d(n, L.x32[L.xfinal], z, h->s);
    } else {
        CU(cudaMemcpyAsync(L.b64, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->s));
        CU(cudaGraphLaunch(H.graph, h->s));
        count_launch(H.graph_nodes);
        h->graph_pending = h->o.timing;
        CU(cudaMemcpyAsync(z, L.x64[L.xfinal], sizeof(double) * n, cudaMemcpyDeviceToDevice, h->s));
    }
    return LAIR_OK;
}

lair_status ensure_work(lair_handle *h, int n, int m) {
    if (!h->wb) {
        TRY(dalloc(h, &h->wb, (size_t)n));
        TRY(dalloc(h, &h->wx, (size_t)n));
        TRY(dalloc(h, &h->wr, (size_t)n));
        TRY(dalloc(h, &h->part, (size_t)RED_PARTS * 33));
        TRY(dalloc(h, &h->dsc, (size_t)256));
    }
    if (m > 0 && h->fg_m < m) {
        TRY(dalloc(h, &h->V, (size_t)n * (m + 1)));
        TRY(dalloc(h, &h->Z, (size_t)n * m));
        h->fg_m = m;
    }
    return LAIR_OK;
}

static lair_status norm2_dev(lair_handle *h, int n, const double *v, double *out_dev, double *out_host) {
    multidot(n, 1, v, n, v, h->part, out_dev, nullptr, h->s);
    if (out_host) {
        CU(cudaMemcpyAsync(h->h_dbl, out_dev, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));
        flush_timers(h);
        *out_host = h->h_dbl[0];
    }
    return LAIR_OK;
}

// solve A0 x = b on hierarchy H (device vectors b, x of length n; b already scaled)
static lair_status solve_dev(lair_handle *h, Hier &H, const double *b, double *x, double tol, int cycle, int max_iter,
                             lair_report *rep) {
    Level &L0 = H.lev[0];
    const DCsr &A = L0.A;
    const int n = A.nr;
    const int m = cycle == LAIR_CYCLE_FGMRES ? (h->o.fgmres_restart > 0 ? h->o.fgmres_restart : 30) : 0;
    if (m > 31) return fail(h, LAIR_ERR_INVALID_ARG, "fgmres_restart must be <= 31");
    TRY(ensure_work(h, n, m));
    double bn2 = 0.0;
    TRY(norm2_dev(h, n, b, h->dsc, &bn2));
    double bn = std::sqrt(bn2);
    if (bn == 0.0) bn = 1.0;
    int it = 0, nh = 0;
    auto hist = [&](double v) {
        if (rep && rep->hist && nh < rep->hist_cap) rep->hist[nh] = v;
        ++nh;
    };
    const bool mixed = h->o.precision == LAIR_MIXED;
    double rel = 0.0;
    lair_status st = LAIR_ERR_NOT_CONVERGED;
    if (cycle == LAIR_CYCLE_STATIONARY) {
        for (;;) {
            // r = b - A x written straight into the cycle's input buffer (mixed: its FP32 copy only)
            int tr = tbegin(h, "outer_residual", (double)A.nnz * 12.0 + (double)n * (4.0 + 16.0 + (mixed ? 4.0 : 8.0)));
            sell_residual(L0.A64, b, x, mixed ? nullptr : L0.b64, mixed ? L0.b32 : nullptr, h->part, h->s);
            tend(h, tr);
            finish_partials(1, h->part, h->dsc, h->s);
            CU(cudaMemcpyAsync(h->h_dbl, h->dsc, sizeof(double), cudaMemcpyDeviceToHost, h->s));
            CU(cudaStreamSynchronize(h->s));

            flush_timers(h);
            rel = std::sqrt(h->h_dbl[0]) / bn;
            hist(rel);
            if (!std::isfinite(rel)) { st = LAIR_ERR_NAN; break; }
            if (rel <= tol) { st = LAIR_OK; break; }
            if (it >= max_iter) break;
            CU(cudaGraphLaunch(H.graph, h->s));
            count_launch(H.graph_nodes);
            h->graph_pending = h->o.timing;
            if (mixed) axpy_f(n, L0.x32[L0.xfinal], x, h->s);
            else axpy_d(n, L0.x64[L0.xfinal], x, h->s);
            ++it;
        }
    } else {
        double *V = h->V, *Z = h->Z;
        std::vector<double> Hm((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), hc(m + 2), y(m + 1);
        // device scalars: |r|^2 at 1, Hessenberg column at 8 (32), the two CGS2 projections at 48 (64), y at 112 (32)
        double *hsum = h->dsc + 8, *hbuf = h->dsc + 48, *nrm = h->dsc + 1, *ydev = h->dsc + 112;
        sell_residual(L0.A64, b, x, V, nullptr, h->part, h->s);
        finish_partials(1, h->part, nrm, h->s);
        CU(cudaMemcpyAsync(h->h_dbl, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CU(cudaStreamSynchronize(h->s));

        flush_timers(h);
        double beta = std::sqrt(h->h_dbl[0]);
        rel = beta / bn;
        hist(rel);
        while (std::isfinite(rel) && rel > tol && it < max_iter) {
            scale_by_norm(n, V, nrm, V, h->s);
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int jdone = 0;
            for (int j = 0; j < m && it < max_iter; ++j) {
                double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
                TRY(precond(h, H, vj, zj));
                ++it;
                int ts = tbegin(h, "outer_spmv", bytes_spmv(A, 8.0));
                sell_spmv<double>(L0.A64, zj, w, h->s);
                tend(h, ts);
                CU(cudaMemsetAsync(hsum, 0, sizeof(double) * (j + 1), h->s));
                int to = tbegin(h, "outer_cgs2", 8.0 * n * (3.0 * (j + 2) + 4.0));
                cgs_pass(1, n, j + 1, V, n, nullptr, w, h->part, h->s);
                finish_partials_acc(j + 1, h->part, hbuf, hsum, h->s);
                cgs_pass(2, n, j + 1, V, n, hbuf, w, h->part, h->s);
                finish_partials_acc(j + 1, h->part, hbuf + 32, hsum, h->s);
                cgs_pass(3, n, j + 1, V, n, hbuf + 32, w, h->part, h->s);
                finish_partials(1, h->part, nrm, h->s);
                scale_by_norm(n, w, nrm, w, h->s);
                tend(h, to);
                CU(cudaMemcpyAsync(h->h_dbl, hsum, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, h->s));
                CU(cudaMemcpyAsync(h->h_dbl + 40, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->s));
                CU(cudaStreamSynchronize(h->s));

                flush_timers(h);
                for (int k = 0; k <= j; ++k) hc[k] = h->h_dbl[k];
                double hn = std::sqrt(h->h_dbl[40]);
                hc[j + 1] = hn;
                for (int k = 0; k < j; ++k) {
                    double t = cs[k] * hc[k] + sn[k] * hc[k + 1];
                    hc[k + 1] = -sn[k] * hc[k] + cs[k] * hc[k + 1];
                    hc[k] = t;
                }
                double den = std::sqrt(hc[j] * hc[j] + hc[j + 1] * hc[j + 1]);
                cs[j] = den > 0.0 ? hc[j] / den : 1.0;
                sn[j] = den > 0.0 ? hc[j + 1] / den : 0.0;
                hc[j] = den;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                for (int k = 0; k <= j; ++k) Hm[(size_t)k * m + j] = hc[k];
                double est = std::fabs(g[j + 1]) / bn;
                hist(est);
                jdone = j + 1;
                if (est <= tol || hn == 0.0 || !std::isfinite(est)) break;
            }
            for (int k = jdone - 1; k >= 0; --k) {
                double acc = g[k];
                for (int c = k + 1; c < jdone; ++c) acc -= Hm[(size_t)k * m + c] * y[c];
                y[k] = acc / Hm[(size_t)k * m + k];
            }
            CU(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * jdone, cudaMemcpyHostToDevice, h->s));
            add_combo(n, jdone, Z, n, ydev, x, h->s);
            sell_residual(L0.A64, b, x, V, nullptr, h->part, h->s);
            finish_partials(1, h->part, nrm, h->s);
            CU(cudaMemcpyAsync(h->h_dbl, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->s));
            CU(cudaStreamSynchronize(h->s));

            flush_timers(h);
            beta = std::sqrt(h->h_dbl[0]);
            rel = beta / bn;
        }
        if (!std::isfinite(rel)) st = LAIR_ERR_NAN;
        else if (rel <= tol) st = LAIR_OK;
    }
    CU(cudaStreamSynchronize(h->s));
    if (rep) {
        rep->iters = it;
        rep->final_rel = rel;
        rep->hist_len = nh < rep->hist_cap ? nh : rep->hist_cap;
    }
    if (st == LAIR_ERR_NOT_CONVERGED) fail(h, st, "not converged: relative residual %.3e after %d cycles", rel, it);
    if (st == LAIR_ERR_NAN) fail(h, st, "residual became NaN/Inf after %d cycles", it);
    return st;
}

// row tiles of the batch's systems at level 0 (SEG_TILE rows at most, never across systems)
static lair_status ensure_tiles(lair_handle *h, const Level &L0) {
    if (h->segt.tile) return LAIR_OK;
    const std::vector<int> &seg = L0.seg_h;
    const int nseg = (int)seg.size() - 1;
    std::vector<int4> tiles;
    std::vector<int> first(nseg + 1);
    for (int q = 0; q < nseg; ++q) {
        first[q] = (int)tiles.size();
        for (int b0 = seg[q]; b0 < seg[q + 1]; b0 += SEG_TILE)
            tiles.push_back(make_int4(q, b0, b0 + SEG_TILE < seg[q + 1] ? b0 + SEG_TILE : seg[q + 1], 0));
    }
    first[nseg] = (int)tiles.size();
    int4 *dt;
    int *df;
    double *dp;
    TRY(dalloc(h, &dt, tiles.size() + 1));
    TRY(dalloc(h, &df, (size_t)nseg + 1));
    TRY(dalloc(h, &dp, (tiles.size() + 1) * (size_t)SEG_TILE_PARTS));
    if (!tiles.empty()) CU(cudaMemcpyAsync(dt, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, h->s));
    CU(cudaMemcpyAsync(df, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, h->s));
    CU(cudaStreamSynchronize(h->s));   // the host vectors are copied from pageable memory
    h->segt.tile = dt;
    h->segt.ntiles = (int)tiles.size();
    h->segt.first = df;
    h->segt.nseg = nseg;
    h->segt.part = dp;
    return LAIR_OK;
}

// batched systems: stationary refinement where every system is tested on its own relative
// residual and stops being updated once it is <= tol (the cycle itself acts on all systems)
// the device-side state of the batched outer loops, for FGMRES(m) (m = 0: stationary refinement only)
static lair_status ensure_batch_ctl(lair_handle *h, int m) {
    const int nseg = h->nseg;
    BatchCtl &c = h->bctl;
    if (!c.bn) {
        double *bn;
        TRY(dalloc(h, &bn, (size_t)nseg));
        c.bn = bn;
        TRY(dalloc(h, &c.rl, (size_t)nseg));
        TRY(dalloc(h, &c.its, (size_t)nseg));
        TRY(dalloc(h, &c.jd, (size_t)nseg));
        // the run flags are the ones the cycle's kernels read (set-up allocates them with the views)
        if (h->sys_run) c.run = h->sys_run;
        else TRY(dalloc(h, &c.run, (size_t)nseg));
        TRY(dalloc(h, &c.done, (size_t)nseg));
        TRY(dalloc(h, &c.nan, 1));
        TRY(dalloc(h, &h->d_ring, (size_t)lair_handle::RING));
        CU(cudaMallocHost(&h->h_ring, sizeof(int) * lair_handle::RING));
        for (cudaEvent_t &e : h->ring_ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c.nseg = nseg;
    }
    if (m > h->bctl_m) {
        TRY(dalloc(h, &c.g, (size_t)nseg * (m + 1)));
        TRY(dalloc(h, &c.cs, (size_t)nseg * m));
        TRY(dalloc(h, &c.sn, (size_t)nseg * m));
        TRY(dalloc(h, &c.Hm, (size_t)nseg * (m + 1) * m));
        h->bctl_m = m;
    }
    c.m = m;
    return LAIR_OK;
}

// The cycle's kernels skip the rows of stopped systems, whose cycle buffers then keep older values; the
// coarsest level's dense inverse multiplies those by exact zeros. Every buffer is cleared when a batched solve
// starts, so those values are always finite ones from this solve.
static lair_status clear_cycle_buffers(lair_handle *h, Hier &H) {
    for (Level &L : H.lev) {
        const size_t n = (size_t)L.A.nr;
        if (h->o.precision == LAIR_MIXED) {
            CU(cudaMemsetAsync(L.b32, 0, sizeof(float) * n, h->s));
            for (float *x : L.x32) CU(cudaMemsetAsync(x, 0, sizeof(float) * n, h->s));
        } else {
            CU(cudaMemsetAsync(L.b64, 0, sizeof(double) * n, h->s));
            for (double *x : L.x64) CU(cudaMemsetAsync(x, 0, sizeof(double) * n, h->s));
        }
    }
    return LAIR_OK;
}

// the running-system count of step k: zeroed, filled by the step's control kernel, copied back without waiting
static int *ring_slot(lair_handle *h, long long k) { return h->d_ring + (int)(k % lair_handle::RING); }

static lair_status ring_post(lair_handle *h, long long k) {
    const int r = (int)(k % lair_handle::RING);
    CU(cudaMemcpyAsync(h->h_ring + r, h->d_ring + r, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CU(cudaEventRecord(h->ring_ev[r], h->s));
    return LAIR_OK;
}

// the count of step k, which was queued LAG steps ago and is normally complete already
static lair_status ring_read(lair_handle *h, long long k, int *out) {
    const int r = (int)(k % lair_handle::RING);
    CU(cudaEventSynchronize(h->ring_ev[r]));
    *out = h->h_ring[r];
    return LAIR_OK;
}

static lair_status batch_finish(lair_handle *h, double tol, int *iters, double *rel) {
    const int nseg = h->nseg;
    // every system runs again in cycles outside the batched loops
    CU(cudaMemsetAsync(h->bctl.run, 1, (size_t)nseg, h->s));
    std::vector<int> its(nseg);
    std::vector<double> rl(nseg);
    int nan = 0;
    CU(cudaMemcpyAsync(its.data(), h->bctl.its, sizeof(int) * nseg, cudaMemcpyDeviceToHost, h->s));
    CU(cudaMemcpyAsync(rl.data(), h->bctl.rl, sizeof(double) * nseg, cudaMemcpyDeviceToHost, h->s));
    CU(cudaMemcpyAsync(&nan, h->bctl.nan, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    flush_timers(h);
    lair_status st = nan ? LAIR_ERR_NAN : LAIR_OK;
    int worst = -1;
    for (int q = 0; q < nseg; ++q) {
        if (iters) iters[q] = its[q];
        if (rel) rel[q] = rl[q];
        if (st == LAIR_OK && !(rl[q] <= tol)) {
            st = LAIR_ERR_NOT_CONVERGED;
            worst = q;
        }
    }
    if (worst >= 0) fail(h, st, "system %d not converged: relative residual %.3e", worst, rl[worst]);
    return st;
}

// batched systems, stationary refinement per system: every iteration the residual of the running systems,
// a per-system stopping test on the device, one V-cycle of the whole batch and the update of the running
// systems. The host reads the running-system count of an iteration LAG iterations later (without draining
// the stream) and stops once it is zero; the iterations queued meanwhile change nothing.
lair_status solve_batched_dev(lair_handle *h, Hier &H, const double *b, double *x, double tol, int max_iter,
                                     int *iters, double *rel) {
    Level &L0 = H.lev[0];
    const DCsr &A = L0.A;
    const int n = A.nr, nseg = h->nseg;
    const bool mixed = h->o.precision == LAIR_MIXED;
    TRY(ensure_work(h, n, 0));
    TRY(ensure_tiles(h, L0));
    TRY(ensure_batch_ctl(h, 0));
    TRY(clear_cycle_buffers(h, H));
    if ((size_t)nseg > (size_t)RED_PARTS * 16) return fail(h, LAIR_ERR_UNSUPPORTED, "at most %d systems", RED_PARTS * 16);
    double *nrm = h->part;                                  // RED_PARTS * 33 doubles >= nseg
    BatchCtl c = h->bctl;
    c.tol = tol;
    c.max_iter = max_iter;
    SegTiles sta = h->segt;
    sta.active = c.run;
    seg_norm2(h->segt, b, nrm, h->s);
    bat_bnorm(nseg, nrm, const_cast<double *>(c.bn), h->s);
    CU(cudaMemsetAsync(c.its, 0, sizeof(int) * nseg, h->s));
    CU(cudaMemsetAsync(c.run, 1, (size_t)nseg, h->s));
    CU(cudaMemsetAsync(c.nan, 0, sizeof(int), h->s));
    for (long long it = 0; it <= (long long)max_iter + lair_handle::LAG + 1; ++it) {
        if (it >= lair_handle::LAG) {
            int running = 0;
            TRY(ring_read(h, it - lair_handle::LAG, &running));
            if (running == 0) break;
        }
        double *r = mixed ? h->wr : L0.b64;
        seg_residual(A, sta, b, x, r, mixed ? L0.b32 : nullptr, nrm, h->s);
        CU(cudaMemsetAsync(ring_slot(h, it), 0, sizeof(int), h->s));
        bat_stat_check(c, nrm, (int)std::min<long long>(it, max_iter), ring_slot(h, it), h->s);
        TRY(ring_post(h, it));
        CU(cudaGraphLaunch(H.graph, h->s));
        count_launch(H.graph_nodes);
        h->graph_pending = h->o.timing;
        if (mixed) seg_axpy<float>(h->segt, c.run, L0.x32[L0.xfinal], x, h->s);
        else seg_axpy<double>(h->segt, c.run, L0.x64[L0.xfinal], x, h->s);
    }
    return batch_finish(h, tol, iters, rel);
}

// batched systems, right-preconditioned FGMRES(m) per system in lockstep: one Arnoldi step for
// every running system per iteration (classical Gram-Schmidt twice on each system's rows), each
// system with its own Givens rotations, stopping test and restarts
lair_status solve_batched_fgmres(lair_handle *h, Hier &H, const double *b, double *x, double tol, int max_iter,
                                        int *iters, double *rel) {
    constexpr int HS = BATCH_HS;
    Level &L0 = H.lev[0];
    const DCsr &A = L0.A;
    const int n = A.nr, nseg = h->nseg;
    const int m = h->o.fgmres_restart > 0 ? h->o.fgmres_restart : 30;
    TRY(ensure_work(h, n, m));
    TRY(ensure_tiles(h, L0));
    TRY(ensure_batch_ctl(h, m));
    TRY(clear_cycle_buffers(h, H));
    if (!h->d_bat) TRY(dalloc(h, &h->d_bat, (size_t)nseg * (3 * HS + 1)));
    double *hsum = h->d_bat, *hbuf = hsum + (size_t)nseg * HS, *ydev = hbuf + (size_t)nseg * HS,
           *nrm = ydev + (size_t)nseg * HS;
    double *V = h->V, *Z = h->Z;
    BatchCtl c = h->bctl;
    c.tol = tol;
    c.max_iter = max_iter;
    SegTiles sta = h->segt;   // the Arnoldi kernels skip the tiles of systems that are not running
    sta.active = c.run;
    seg_norm2(h->segt, b, nrm, h->s);
    bat_bnorm(nseg, nrm, const_cast<double *>(c.bn), h->s);
    CU(cudaMemsetAsync(c.its, 0, sizeof(int) * nseg, h->s));
    CU(cudaMemsetAsync(c.done, 0, (size_t)nseg, h->s));
    CU(cudaMemsetAsync(c.nan, 0, sizeof(int), h->s));
    long long step = 0;   // ring position
    for (int restart = 0; restart <= max_iter; ++restart) {
        seg_residual(A, h->segt, b, x, V, nullptr, nrm, h->s);
        CU(cudaMemsetAsync(ring_slot(h, step), 0, sizeof(int), h->s));
        bat_fg_restart(c, nrm, ring_slot(h, step), h->s);
        TRY(ring_post(h, step));
        int running = 0;
        TRY(ring_read(h, step, &running));   // one wait per restart
        ++step;
        flush_timers(h);
        if (running == 0) break;
        seg_scale(sta, V, nrm, V, h->s);
        const long long first = step;
        for (int j = 0; j < m; ++j) {
            if (step - first >= lair_handle::LAG) {
                TRY(ring_read(h, step - lair_handle::LAG, &running));
                if (running == 0) break;
            }
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
            TRY(precond(h, H, vj, zj));
            int ts = tbegin(h, "outer_spmv", bytes_spmv(A, 8.0));
            sell_spmv<double>(L0.A64, zj, w, h->s);
            tend(h, ts);
            CU(cudaMemsetAsync(hsum, 0, sizeof(double) * (size_t)nseg * HS, h->s));
            // CGS2 in three streaming passes over V: dots; update and dots; update and norm
            seg_cgs_pass(sta, 1, j + 1, V, n, HS, nullptr, w, hbuf, hsum, h->s);
            seg_cgs_pass(sta, 2, j + 1, V, n, HS, hbuf, w, hbuf, hsum, h->s);
            seg_cgs_pass(sta, 3, j + 1, V, n, HS, hbuf, w, nrm, nullptr, h->s);
            seg_scale(sta, w, nrm, w, h->s);
            CU(cudaMemsetAsync(ring_slot(h, step), 0, sizeof(int), h->s));
            bat_fg_givens(c, j, hsum, nrm, ring_slot(h, step), h->s);
            TRY(ring_post(h, step));
            ++step;
        }
        // per-system least-squares solutions y and the update x += Z y of the systems that ran
        bat_fg_solve_y(c, ydev, h->s);
        seg_add_combo(h->segt, c.jd, Z, n, HS, ydev, x, h->s);
    }
    return batch_finish(h, tol, iters, rel);
}

static void fill_report(lair_handle *h, Hier &H, lair_report *rep) {
    if (!rep) return;
    rep->setup_ms = H.setup_ms;
    rep->nlevels = (int)H.lev.size();
    rep->singular_R = H.singular_R;
    rep->singular_P = H.singular_P;
    double nnz0 = (double)H.lev[0].A.nnz, tot = 0.0, cyc = 0.0;
    for (auto &L : H.lev) {
        tot += L.A.nnz;
        if (!L.coarsest) cyc += 3.0 * L.A.nnz + L.R.nnz + L.P.nnz;
        else cyc += (double)L.A.nr * L.A.nr;
    }
    rep->op_complexity = tot / nnz0;
    rep->cycle_complexity = cyc / nnz0;
}

lair_status run_solve(lair_handle *h, Hier &H, const double *b, double *x, double tol, int cycle, int max_iter,
                             lair_report *rep, bool scale) {
    auto t0 = std::chrono::steady_clock::now();
    const int n = H.lev[0].A.nr;
    TRY(ensure_work(h, n, 0));
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    double *db = h->wb, *dx = h->wx;
    if (bdev) CU(cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->s));
    else CU(cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyHostToDevice, h->s));
    if (xdev) CU(cudaMemcpyAsync(dx, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->s));
    else CU(cudaMemcpyAsync(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice, h->s));
    if (scale && H.bs > 1) {
        launch_block_apply(n / H.bs, H.bs, H.blk_inv, db, h->wr, h->s);
        CU(cudaMemcpyAsync(db, h->wr, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->s));
    }
    lair_status st = solve_dev(h, H, db, dx, tol, cycle, max_iter, rep);
    if (st != LAIR_OK && st != LAIR_ERR_NOT_CONVERGED) return st;
    if (xdev) CU(cudaMemcpyAsync(x, dx, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->s));
    else CU(cudaMemcpyAsync(x, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
    CU(cudaStreamSynchronize(h->s));
    fill_report(h, H, rep);
    if (rep) rep->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

}  // namespace lair
