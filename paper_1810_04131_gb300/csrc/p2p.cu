// Host side of the far-field evaluators (kernels in p2p_kernels.cuh): the FP64
// tile and neighbour lists, the matvec and normal-derivative drivers for the
// dense, cut-off and FMM far fields, the FMM leaf-size autotuner, and the
// off-surface potential.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

// this translation unit holds the far-field kernels themselves
#define YK_DEFINE_P2P_KERNELS
#include "p2p_kernels.cuh"
#include "yk_internal.cuh"

namespace yk {

// The FP64 tile list for a split distance (kind 0: residual, 1: gradient,
// 2: all pairs), built on first use and after the particles move.
static int tile_list(yk_geom* g, int kind, const int2** list, int* count) {
    PairList& L = g->lists[kind];
    if (!L.valid) {
        cudaStream_t st = g->ctx->stream;
        const double thr = kind == 0 ? g->tile_gap
                           : kind == 1 ? g->tile_gap_grad
                           : kind == 2 ? INFINITY : g->cutoff_gap;
        int* d_count = g->d_counter;
        YK_TRY_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), st));
        YK_LAUNCH(k_pair_list, ceil_div(g->np, 4), 128, 0, st, g->np, g->d_part, thr,
                  !g->use_self, d_count, (int2*)nullptr, 0);
        int n = 0;
        YK_TRY_CUDA(cudaMemcpyAsync(&n, d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        if (n > L.cap) {
            dev_free(L.d, st);
            L.d = nullptr;
            L.cap = 0;
            YK_TRY(dev_alloc((void**)&L.d, sizeof(int2) * (size_t)n, st));
            L.cap = n;
        }
        YK_TRY_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), st));
        YK_LAUNCH(k_pair_list, ceil_div(g->np, 4), 128, 0, st, g->np, g->d_part, thr,
                  !g->use_self, d_count, L.d, L.cap);
        YK_TRY_CUDA(cudaGetLastError());
        L.n = n;
        L.valid = true;
    }
    *list = L.d;
    *count = L.n;
    return YK_OK;
}

// The particle pairs of the symmetric FP32 far field (k_p2p_f32_sym), sorted
// by P: kind 0 for the inner operator, kind 1 for the precision-split
// residual (pairs of the FP64 tiles left out). Built on first use and after
// the particles move.
static int sym_list(yk_geom* g, int kind, const int2** list, int* count) {
    PairList& L = g->sym[kind];
    if (!L.valid && kind >= 3) {
        // from neighbour lists: 3 the FMM near field; the cut-off neighbours
        // 4 beyond the value split, 5 beyond the normal-derivative split, 6 all
        cudaStream_t st = g->ctx->stream;
        GeomView G = g->view();
        const int* noff = kind == 3 ? g->fmm.near_off : g->nbr_off;
        const int* nlst = kind == 3 ? g->fmm.near : g->nbr;
        const bool mask = kind == 4 || kind == 5;
        const double gap = kind == 4 ? g->split_gap : (kind == 5 ? g->split_gap_grad : 0.0);
        int* counts = (int*)g->ws.partial;
        int* off = counts + g->np;
        YK_LAUNCH(k_sym_near<false>, ceil_div(g->np, 4), 128, 0, st, G, noff, nlst, mask, gap,
                  counts, (const int*)nullptr, (int2*)nullptr);
        YK_LAUNCH(k_scan_offsets, 1, 1024, 0, st, g->np, counts, off);
        int n = 0;
        YK_TRY_CUDA(cudaMemcpyAsync(&n, off + g->np, sizeof(int), cudaMemcpyDeviceToHost, st));
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        if (n > L.cap) {
            dev_free(L.d, st);
            L.d = nullptr;
            L.cap = 0;
            YK_TRY(dev_alloc((void**)&L.d, sizeof(int2) * (size_t)n, st));
            L.cap = n;
        }
        if (n > 0)
            YK_LAUNCH(k_sym_near<true>, ceil_div(g->np, 4), 128, 0, st, G, noff, nlst, mask, gap,
                      (int*)nullptr, off, L.d);
        YK_TRY_CUDA(cudaGetLastError());
        L.n = n;
        L.valid = true;
    }
    if (!L.valid) {
        cudaStream_t st = g->ctx->stream;
        GeomView G = g->view();
        const bool mask = kind >= 1;   // 1: value split, 2: normal-derivative split
        const double gap = kind == 1 ? g->split_gap : (kind == 2 ? g->split_gap_grad : 0.0);
        int* counts = (int*)g->ws.partial;   // 2 np + 1 ints of scratch (partial holds >= n doubles)
        int* off = counts + g->np;
        YK_LAUNCH(k_sym_count, ceil_div(g->np, 4), 128, 0, st, G, mask, gap, counts);
        YK_LAUNCH(k_scan_offsets, 1, 1024, 0, st, g->np, counts, off);
        int n = 0;
        YK_TRY_CUDA(cudaMemcpyAsync(&n, off + g->np, sizeof(int), cudaMemcpyDeviceToHost, st));
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        if (n > L.cap) {
            dev_free(L.d, st);
            L.d = nullptr;
            L.cap = 0;
            YK_TRY(dev_alloc((void**)&L.d, sizeof(int2) * (size_t)n, st));
            L.cap = n;
        }
        if (n > 0) YK_LAUNCH(k_sym_fill, ceil_div(g->np, 4), 128, 0, st, G, mask, gap, off, L.d);
        YK_TRY_CUDA(cudaGetLastError());
        L.n = n;
        L.valid = true;
    }
    *list = L.d;
    *count = L.n;
    return YK_OK;
}

// Launch shape of the symmetric kernel for a geometry's pair list kind:
// Q-node ranges as short as 64 until there are work items for about eight
// blocks per SM (small systems), up to SYM_TASKS items per block beyond.
int sym_params(yk_geom* g, int kind, SymParams* p) {
    YK_TRY(sym_list(g, kind, &p->tasks, &p->ntasks));
    // 64 of P's nodes per warp, as few warps as cover a particle (up to 4):
    // particles of few nodes leave no warp idle
    p->nw = std::min(F32_TPB / 32, ceil_div(g->npp, 64));
    const int64_t npc = ceil_div(g->npp, 64 * p->nw);
    int qch = STILE;
    while (qch > 64 && (int64_t)p->ntasks * npc * ceil_div(g->npp, qch) < 152 * 8) qch /= 2;
    const int64_t items = (int64_t)p->ntasks * npc * ceil_div(g->npp, qch);
    p->qch = qch;
    p->ipb = (int)std::max<int64_t>(1, std::min<int64_t>(SYM_TASKS, items / (152 * 12)));
    p->blocks = items == 0 ? 0 : ceil_div(items, p->ipb);
    p->kscale = sqrt(LOG2E) / (2.0 * PI * g->prm.rho);   // units of PairF32
    return YK_OK;
}

// FP32 far field of the dense operator by the symmetric kernel, added to out.
static int far_sym(yk_geom* g, int kind, double* out) {
    SymParams p;
    YK_TRY(sym_params(g, kind, &p));
    if (p.blocks == 0) return YK_OK;
    if (p.nw == F32_TPB / 32)
        YK_LAUNCH(k_p2p_f32_sym<true>, (unsigned)p.blocks, F32_TPB, 0, g->ctx->stream, g->view(),
                  g->ws.src4, p.tasks, p.ntasks, p.qch, p.ipb, p.nw, p.kscale, out);
    else
        YK_LAUNCH(k_p2p_f32_sym<false>, (unsigned)p.blocks, 32 * p.nw, 0, g->ctx->stream,
                  g->view(), g->ws.src4, p.tasks, p.ntasks, p.qch, p.ipb, p.nw, p.kscale, out);
    return YK_OK;
}

// FP32 far field of the split normal derivative by the symmetric kernel
// (pairs beyond the normal derivative's split distance), added to out.
static int far_symg(yk_geom* g, int kind, const double* sigma, double* out) {
    SymParams p;
    YK_TRY(sym_params(g, kind, &p));
    if (p.blocks == 0) return YK_OK;
    const int64_t npairs = (int64_t)g->np * ((g->npp + 1) / 2);
    cudaStream_t st = g->ctx->stream;
    YK_LAUNCH(k_src_grad_pairs, (unsigned)((npairs + 255) / 256), 256, 0, st, g->view(), sigma,
              (float)(LOG2E / g->prm.rho), g->ws.src4g);
    const double kscale = sqrt(LOG2E) * (1.0 / g->prm.rho) * (LOG2E / g->prm.rho) / (2.0 * PI);
    if (p.nw == F32_TPB / 32)
        YK_LAUNCH(k_p2p_f32_symg<true>, (unsigned)p.blocks, F32_TPB, 0, st, g->view(), g->ws.src4g,
                  p.tasks, p.ntasks, p.qch, p.ipb, p.nw, kscale, out);
    else
        YK_LAUNCH(k_p2p_f32_symg<false>, (unsigned)p.blocks, 32 * p.nw, 0, st, g->view(),
                  g->ws.src4g, p.tasks, p.ntasks, p.qch, p.ipb, p.nw, kscale, out);
    return YK_OK;
}

// Q-node ranges per FP64 tile (k_tiles_f64): enough work items for about
// four blocks per SM, each range at least 32 nodes.
static int tiles_qsplit(const yk_geom* g, int ntiles) {
    const int npc = ceil_div(g->npp, TILE_TPB);
    const int64_t base = (int64_t)std::max(1, ntiles) * npc;
    const int want = (int)std::min<int64_t>(ceil_div(152 * 4, base), ceil_div(g->npp, 32));
    return std::max(1, want);
}

static int tiles_grid(const yk_geom* g, int ntiles) {
    const int64_t items = (int64_t)ntiles * ceil_div(g->npp, TILE_TPB) * tiles_qsplit(g, ntiles);
    return (int)std::max<int64_t>(1, std::min<int64_t>(items, 152 * 16));
}

// Own-particle far pairs of the FP64 operators: the precomputed self blocks
// (the pair lists then hold no P == Q tiles).
static int self_blocks_f32(yk_geom* g, const double* sigma, double* extra, bool accumulate) {
    if (!g->use_self) return YK_OK;
    const dim3 grid(g->np, ceil_div(g->npp, BAPPLY_ROWS));
    const size_t smem = blocks_apply_smem<float>(g->npp);
    if (accumulate)
        YK_LAUNCH((k_blocks_apply<float, true>), grid, BAPPLY_ROWS * BAPPLY_SLICES, smem,
                  g->ctx->stream, g->npp, g->d_shape_of, g->d_self32, sigma, extra);
    else
        YK_LAUNCH((k_blocks_apply<float, false>), grid, BAPPLY_ROWS * BAPPLY_SLICES, smem,
                  g->ctx->stream, g->npp, g->d_shape_of, g->d_self32, sigma, extra);
    return YK_OK;
}

static int self_blocks(yk_geom* g, const double* sigma, double* extra, bool grad) {
    if (!g->use_self) return YK_OK;
    const dim3 grid(g->np, ceil_div(g->npp, BAPPLY_ROWS));
    YK_LAUNCH((k_blocks_apply<double, true>), grid, BAPPLY_ROWS * BAPPLY_SLICES,
              blocks_apply_smem<double>(g->npp), g->ctx->stream, g->npp, g->d_shape_of,
              grad ? g->d_self_grad : g->d_self, sigma, extra);
    return YK_OK;
}

// The own-particle part of the FP32 inner operator, y_P = A_PP x_P for
// every particle P: the FP32 self block and the QBX near rows.
int own_apply_f32(yk_geom* g, const double* x, double* y) {
    if (!g->use_self) return YK_ERR_ARG;
    double* extra = g->ws.vec[5];
    YK_TRY(self_blocks_f32(g, x, extra, false));
    GeomView G = g->view();
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, g->ctx->stream, G, 0, g->ws.partial, extra,
              G.cval, x, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// The FP32 source records of sigma (k_src_pairs), before any FP32 far-field kernel.
static int stage_sources(yk_geom* g, const double* sigma) {
    const int64_t npairs = (int64_t)g->np * ((g->npp + 1) / 2);
    YK_LAUNCH(k_src_pairs, (unsigned)((npairs + 255) / 256), 256, 0, g->ctx->stream, g->view(),
              sigma, (float)(LOG2E / g->prm.rho), g->ws.src4);
    return YK_OK;
}

// Cut-off neighbour lists (CSR), built on first use and after the particles move.
static int neighbours(yk_geom* g) {
    if (g->nbr_valid) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    if (!g->nbr_off) YK_TRY(dev_alloc((void**)&g->nbr_off, sizeof(int) * (g->np + 1), st));
    int* counts = (int*)g->ws.partial;   // np ints of scratch (partial holds >= n doubles)
    YK_LAUNCH(k_nbr_count, ceil_div(g->np, 128), 128, 0, st, g->np, g->d_part, g->cutoff_gap,
              counts);
    YK_LAUNCH(k_scan_offsets, 1, 1024, 0, st, g->np, counts, g->nbr_off);
    int total = 0;
    YK_TRY_CUDA(cudaMemcpyAsync(&total, g->nbr_off + g->np, sizeof(int), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    if (total > g->nbr_cap) {
        dev_free(g->nbr, st);
        g->nbr = nullptr;
        g->nbr_cap = 0;
        YK_TRY(dev_alloc((void**)&g->nbr, sizeof(int) * (size_t)total, st));
        g->nbr_cap = total;
    }
    YK_LAUNCH(k_nbr_fill, ceil_div(g->np, 128), 128, 0, st, g->np, g->d_part, g->cutoff_gap,
              g->nbr_off, g->nbr);
    YK_TRY_CUDA(cudaGetLastError());
    g->nbr_valid = true;
    return YK_OK;
}

// Cut-off far field: FP32 per target particle over its neighbours (masked
// against the FP64 tiles for the split operators), FP64 tiles over the
// in-cut-off pairs for the FP64 path.
static int matvec_cutoff(yk_geom* g, const double* sigma, double* y, Prec prec, bool grad) {
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    YK_TRY(neighbours(g));
    const double ks = sqrt(LOG2E) / (2.0 * PI * g->prm.rho);
    double* extra = nullptr;
    int used = 1;
    if (prec == Prec::F32) {
        YK_TRY(stage_sources(g, sigma));
        if (!grad && g->use_self) {
            // own particle by the FP32 self block, neighbour pairs P < Q by the
            // symmetric kernel
            extra = g->ws.vec[5];
            YK_TRY(self_blocks_f32(g, sigma, extra, false));
            YK_TRY(far_sym(g, 6, extra));
            used = 0;
        } else if (grad) {
            YK_LAUNCH(k_p2p_f32_grad_cut<false>, g->np, F32_TPB, 0, st, G, g->ws.src4, 0.0,
                      g->nbr_off, g->nbr, g->ws.partial);
        } else {
            YK_LAUNCH(k_p2p_f32_cut<false>, g->np, F32_TPB, 0, st, G, g->ws.src4, (float)ks, 0.0,
                      g->use_self, g->nbr_off, g->nbr, g->ws.partial);
        }
    } else {
        const int kind = (prec == Prec::F64) ? 3 : (grad ? 1 : 0);
        const int2* list;
        int ntiles;
        YK_TRY(tile_list(g, kind, &list, &ntiles));
        extra = g->ws.vec[5];
        YK_TRY_CUDA(cudaMemsetAsync(extra, 0, sizeof(double) * g->n, st));
        YK_TRY(self_blocks(g, sigma, extra, grad));
        used = 0;
        if (prec == Prec::SPLIT) {   // neighbour pairs beyond the split distance, symmetric FP32
            if (grad) {
                YK_TRY(far_symg(g, 5, sigma, extra));
            } else {
                YK_TRY(stage_sources(g, sigma));
                YK_TRY(far_sym(g, 4, extra));
            }
        }
        if (grad)
            YK_LAUNCH(k_tiles_f64<true>, tiles_grid(g, ntiles), TILE_TPB, 0, st, G, sigma, list,
                      ntiles, tiles_qsplit(g, ntiles), extra);
        else
            YK_LAUNCH(k_tiles_f64<false>, tiles_grid(g, ntiles), TILE_TPB, 0, st, G, sigma, list,
                      ntiles, tiles_qsplit(g, ntiles), extra);
        if (prec == Prec::SPLIT) YK_TRY(band_expansions(g, sigma, extra, grad));
    }
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, st, G, used, g->ws.partial, extra,
              grad ? G.cgrad : G.cval, sigma, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// FP32 inner operator with the FMM far field: near lists by FP32 P2P, the
// rest by expansions (fmm.cu), plus the QBX rows.
static int fmm_apply(yk_geom* g, const double* sigma, double* y) {
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    double* extra = g->ws.vec[5];
    YK_TRY(fmm_far(g, sigma, extra));
    YK_TRY(self_blocks_f32(g, sigma, extra, true));
    YK_TRY(stage_sources(g, sigma));
    int chunks = 0;
    if (g->use_self) {
        // near field by the symmetric kernel over the near lists' pairs P < Q
        // (the own particle's pairs come from the self block)
        YK_TRY(far_sym(g, 3, extra));
    } else {
        const double ks = sqrt(LOG2E) / (2.0 * PI * g->prm.rho);
        YK_LAUNCH(k_p2p_f32_cut<false>, g->np, F32_TPB, 0, st, G, g->ws.src4, (float)ks, 0.0,
                  g->use_self, g->fmm.near_off, g->fmm.near, g->ws.partial);
        chunks = 1;
    }
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, st, G, chunks, g->ws.partial, extra,
              G.cval, sigma, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// Autotuned leaf sides (in units of the bounding radius R), shared by every
// geometry of the process: systems with the same order, nodes per particle,
// rho/R and particle density (both on a quarter-octave grid) reuse the
// choice instead of timing the candidates again.
using FmmTuneKey = std::tuple<int, int, int, int>;
static std::mutex g_fmm_tune_mutex;
static std::map<FmmTuneKey, double> g_fmm_tune;

static FmmTuneKey fmm_tune_key(yk_geom* g) {
    double x0, y0, side;
    fmm_root_box(g, &x0, &y0, &side);
    const double R = g->max_radius;
    const double dens = (double)g->np * R * R / std::max(side * side, R * R);
    return FmmTuneKey(g->prm.fmm_order, g->npp, (int)lround(4.0 * log2(g->prm.rho / R)),
                      (int)lround(4.0 * log2(dens)));
}

// Leaf level of the FMM: the one given (fmm_leaf), the cached choice for
// similar systems, or the fastest of the admissible ones, timed with CUDA
// events on the first application (each candidate applied once to warm up,
// then twice timed). Without an admissible level the far field falls back
// to the cut-off P2P.
static int fmm_tune(yk_geom* g, const double* sigma, double* y) {
    FmmTree& F = g->fmm;
    const double leaf = g->prm.fmm_leaf;
    int lo = 0, hi = -1;
    if (leaf > 0.0) {
        double x0, y0, side;
        fmm_root_box(g, &x0, &y0, &side);
        int L = 0;
        while (L < FMM_LMAX && side / (double)(1 << L) > leaf) ++L;
        const double b = side / (double)(1 << L), R = g->max_radius;
        // the discs of an interacting pair must be disjoint: 2 (b/sqrt2 + R) < 3 b
        F.far_off = !(2.0 * (b * M_SQRT1_2 + R) < 3.0 * b);
        F.Lsel = L;
        F.tuned = true;
        return YK_OK;
    }
    YK_TRY(fmm_candidates(g, &lo, &hi));
    if (lo > hi) {
        F.far_off = true;
        F.tuned = true;
        return YK_OK;
    }
    F.far_off = false;
    F.Lsel = hi;
    const FmmTuneKey key = fmm_tune_key(g);
    double cached = 0.0;
    {
        std::lock_guard<std::mutex> lk(g_fmm_tune_mutex);
        auto it = g_fmm_tune.find(key);
        if (it != g_fmm_tune.end()) cached = it->second;
    }
    if (lo < hi && cached > 0.0) {
        // the admissible level whose leaf side is closest to the cached one
        double x0, y0, side;
        fmm_root_box(g, &x0, &y0, &side);
        double best = INFINITY;
        for (int L = lo; L <= hi; ++L) {
            const double d = fabs(log(side / (double)(1 << L) / (cached * g->max_radius)));
            if (d < best) best = d, F.Lsel = L;
        }
    } else if (lo < hi) {
        cudaStream_t st = g->ctx->stream;
        cudaEvent_t e0, e1;
        YK_TRY_CUDA(cudaEventCreate(&e0));
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return YK_ERR_CUDA;
        }
        float best = INFINITY;
        int rc = YK_OK;
        for (int L = lo; L <= hi && rc == YK_OK; ++L) {
            rc = fmm_build(g, L);
            if (rc == YK_OK) rc = fmm_apply(g, sigma, y);
            if (rc == YK_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = YK_ERR_CUDA;
            for (int r = 0; r < 2 && rc == YK_OK; ++r) rc = fmm_apply(g, sigma, y);
            float ms = 0.0f;
            if (rc == YK_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                                cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = YK_ERR_CUDA;
            if (rc == YK_OK && ms < best) best = ms, F.Lsel = L;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        YK_TRY(rc);
        F.valid = false;
        double x0, y0, side;
        fmm_root_box(g, &x0, &y0, &side);
        std::lock_guard<std::mutex> lk(g_fmm_tune_mutex);
        g_fmm_tune[key] = side / (double)(1 << F.Lsel) / g->max_radius;
    }
    F.tuned = true;
    return YK_OK;
}

static int matvec_fmm(yk_geom* g, const double* sigma, double* y) {
    FmmTree& F = g->fmm;
    if (!F.tuned) YK_TRY(fmm_tune(g, sigma, y));
    if (F.far_off) return matvec_cutoff(g, sigma, y, Prec::F32, false);
    if (!F.valid || F.L != F.Lsel) YK_TRY(fmm_build(g, F.Lsel));
    return fmm_apply(g, sigma, y);
}

static int matvec_body(yk_geom* g, const double* sigma, double* y, Prec prec) {
    if (g->prm.farfield == YK_FARFIELD_FMM && prec == Prec::F32) return matvec_fmm(g, sigma, y);
    if (g->prm.farfield != YK_FARFIELD_DENSE) return matvec_cutoff(g, sigma, y, prec, false);
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int nchunk = g->ws.nchunk;
    const int ppc = ceil_div(g->np, nchunk);
    dim3 grid(ceil_div(g->n, TPB), nchunk);
    const double ks = sqrt(LOG2E) / (2.0 * PI * g->prm.rho);   // units of PairF32
    double* extra = nullptr;
    int used_chunks = nchunk;
    if (prec == Prec::F32 && g->use_self) {
        // own-particle far pairs by the FP32 self block, all other pairs by
        // the symmetric kernel
        YK_TRY(stage_sources(g, sigma));
        extra = g->ws.vec[5];
        YK_TRY(self_blocks_f32(g, sigma, extra, false));
        YK_TRY(far_sym(g, 0, extra));
        used_chunks = 0;
    } else if (prec == Prec::F32) {
        YK_TRY(stage_sources(g, sigma));
        YK_LAUNCH(k_p2p_f32<false>, grid, F32_TPB, 0, st, G, g->ws.src4, ppc, (float)ks, 0.0,
                  g->use_self, g->ws.partial);
    } else {
        const int kind = (prec == Prec::F64) ? 2 : 0;
        const int2* list;
        int ntiles;
        YK_TRY(tile_list(g, kind, &list, &ntiles));
        extra = g->ws.vec[5];
        YK_TRY_CUDA(cudaMemsetAsync(extra, 0, sizeof(double) * g->n, st));
        YK_TRY(self_blocks(g, sigma, extra, false));
        if (prec == Prec::SPLIT) {   // pairs beyond the split distance in FP32
            YK_TRY(stage_sources(g, sigma));
            YK_TRY(far_sym(g, 1, extra));
        }
        used_chunks = 0;
        YK_LAUNCH(k_tiles_f64<false>, tiles_grid(g, ntiles), TILE_TPB, 0, st, G, sigma, list,
                  ntiles, tiles_qsplit(g, ntiles), extra);
        if (prec == Prec::SPLIT) YK_TRY(band_expansions(g, sigma, extra, false));
    }
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, st, G, used_chunks, g->ws.partial, extra,
              G.cval, sigma, y);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

static int normal_derivative_body(yk_geom* g, const double* sigma, double* un, Prec prec) {
    if (g->prm.farfield != YK_FARFIELD_DENSE) return matvec_cutoff(g, sigma, un, prec, true);
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int kind = (prec == Prec::F64) ? 2 : 1;
    const int2* list;
    int ntiles;
    YK_TRY(tile_list(g, kind, &list, &ntiles));
    double* extra = g->ws.vec[5];
    YK_TRY_CUDA(cudaMemsetAsync(extra, 0, sizeof(double) * g->n, st));
    YK_TRY(self_blocks(g, sigma, extra, true));
    const int used_chunks = 0;
    if (prec != Prec::F64) YK_TRY(far_symg(g, 2, sigma, extra));   // pairs beyond the split distance
    YK_LAUNCH(k_tiles_f64<true>, tiles_grid(g, ntiles), TILE_TPB, 0, st, G, sigma, list, ntiles,
              tiles_qsplit(g, ntiles), extra);
    if (prec != Prec::F64) YK_TRY(band_expansions(g, sigma, extra, true));
    YK_LAUNCH(k_assemble, ceil_div(g->n, 256), 256, 0, st, G, used_chunks, g->ws.partial, extra,
              G.cgrad, sigma, un);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

// The operators, with the near-contact correction (contact.cu) on top of
// every far-field mode and precision.
int matvec(yk_geom* g, const double* sigma, double* y, Prec prec) {
    YK_TRY(matvec_body(g, sigma, y, prec));
    return contact_apply(g, sigma, y, false);
}

int normal_derivative(yk_geom* g, const double* sigma, double* un, Prec prec) {
    YK_TRY(normal_derivative_body(g, sigma, un, prec));
    return contact_apply(g, sigma, un, true);
}

int potential(yk_geom* g, const double* sigma, const double* targets, int64_t nt, double* u) {
    if (nt <= 0) return YK_OK;
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int nct = ceil_div(nt, TPB);
    int nchunk = std::max(1, std::min(g->np, ceil_div(4 * 152, nct)));
    const int ppc = ceil_div(g->np, nchunk);
    nchunk = ceil_div(g->np, ppc);
    double* part = nullptr;
    YK_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * nchunk * nt, st));
    dim3 grid(nct, nchunk);
    YK_LAUNCH(k_potential, grid, TPB, 0, st, G, sigma, targets, nt, ppc, part);
    YK_LAUNCH(k_sum_chunks, ceil_div(nt, 256), 256, 0, st, nt, nchunk, part, u);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    YK_TRY_CUDA(e);
    return YK_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free off-surface potential (yk_eval_potential_noalloc).
//
// yk_eval_potential stages its per-chunk partial sums in a buffer it
// allocates for each call. Some callers must not allocate device memory
// where they evaluate the potential: real-time loops that cannot block in
// the allocator, or applications that reserved the GPU's memory up front
// and give libraries a fixed budget. For them this variant keeps the
// scratch in a file-scope device array of STATIC_SCRATCH_DOUBLES doubles
// (8 MiB), which every GPU that loads the library holds until the process
// exits.
//
// In host code the array's name only stands for the symbol; the kernels
// receive its device address, looked up once per device with
// cudaGetSymbolAddress while that device is current. The lookup happens on
// the first call on each device, so that first call should come before any
// stream capture begins. The address is kept for the life of the process; a
// device reset invalidates it.
//
// All calls share the one array and it keeps the last call's contents.
// Nothing in it has to start at zero: every partial sum the reduction reads
// is written by the same call first. Calls whose kernels overlap on the GPU
// (for example two streams, or two contexts on one device) race on the
// array; callers must order them.
// ---------------------------------------------------------------------------
constexpr int64_t STATIC_SCRATCH_DOUBLES = (int64_t)1 << 20;
static __device__ __align__(256) double g_static_scratch[STATIC_SCRATCH_DOUBLES];

static std::mutex g_static_scratch_mutex;
static double* g_static_scratch_ptr[256] = {};   // device address, per device ordinal

static int static_scratch_address(int device, double** out) {
    if (device < 0 || device >= 256) return YK_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_static_scratch_mutex);
    if (!g_static_scratch_ptr[device]) {
        void* ptr = nullptr;
        // the current device is the context's device (set by the caller)
        YK_TRY_CUDA(cudaGetSymbolAddress(&ptr, g_static_scratch));
        g_static_scratch_ptr[device] = (double*)ptr;
    }
    *out = g_static_scratch_ptr[device];
    return YK_OK;
}

int potential_noalloc(yk_geom* g, const double* sigma, const double* targets, int64_t nt,
                      double* u) {
    if (nt <= 0) return YK_OK;
    if (nt > STATIC_SCRATCH_DOUBLES) return YK_ERR_TOO_LARGE;
    double* scratch = nullptr;
    YK_TRY(static_scratch_address(g->ctx->device, &scratch));
    cudaStream_t st = g->ctx->stream;
    GeomView G = g->view();
    const int nct = ceil_div(nt, TPB);
    // as many source chunks as the scratch holds (at least one)
    const int64_t fit = STATIC_SCRATCH_DOUBLES / nt;
    int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(g->np, fit),
                                                             ceil_div(4 * 152, nct)));
    const int ppc = ceil_div(g->np, nchunk);
    nchunk = ceil_div(g->np, ppc);
    dim3 grid(nct, nchunk);
    YK_LAUNCH(k_potential, grid, TPB, 0, st, G, sigma, targets, nt, ppc, scratch);
    YK_LAUNCH(k_sum_chunks, ceil_div(nt, 256), 256, 0, st, nt, nchunk, scratch, u);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}
}  // namespace yk
