// Batched mixed-precision solves of several independent configurations
// (yk_solve_batch; the serving loop uses it for the small requests it
// admits together).
//
// Every system keeps its own geometry, Krylov workspace and tolerances; the
// refinement residual of each system (the FP64-accurate precision-split
// operator, Eq. bie) is formed per system as in yk_solve. What is batched is
// the inner FP32 GMRES, which holds nearly all of the steps: the systems'
// inner solves advance in lock step, and each step of the Arnoldi process
// is ONE launch per kernel for all of them:
//   z_j = M^-1 v_j (block preconditioner, kept: the solution is Z y), the
//   FP32 source records of z_j, the FP32 self block, the symmetric FP32 far field, the near
//   QBX rows (the operator of Eq. bie), the CGS2 dot products and
//   projections, the Givens update and the normalisation.
// A launch's grid covers the largest system; the blocks of smaller systems
// beyond their own size, and of systems that have converged, return at
// once. A per-system descriptor in device memory (SysDesc) tells each block
// where its system's data lives. The host reads all systems' residual
// estimates with one copy every few steps (as many as the slowest-closing
// system's recent rate of decrease says are still needed) and retires the
// systems that met their tolerance; a retired system's basis is only used up
// to the step that met it, so its solution is the one a separate solve
// stopping there would form.
//
// Systems that do not fit this path (FP64 precision, cut-off or FMM far
// field, no self blocks, no block preconditioner, near-contact corrections)
// are solved one by one with yk_solve's code path.
#include <math.h>

#include <algorithm>
#include <vector>

#include "block_apply.cuh"
#include "p2p_kernels.cuh"
#include "yk_internal.cuh"

namespace yk {

constexpr int BT = 256;          // threads of the node-wise batched kernels
constexpr int BATCH_STEPS = 4;   // Arnoldi steps per host look at most

// Where one system's data lives (device memory, read by every batched kernel).
struct SysDesc {
    GeomView G;
    double *V, *H, *gv, *cs, *sn, *h1, *h2, *ybuf, *dotpart, *status, *hist;
    double *Zp, *extra;   // Zp: kept z_j = M^-1 v_j [m][n]
    float4* rec;
    const float* minv32;
    const float* self32;
    const int2* tasks;
    const double* b;   // right-hand side of the inner solve
    double* x;         // its solution
    double kscale;
    float kpf;
    int ntasks, qch, ipb, nw, sym_blocks, dot_blocks, m, k1, active;
};

// part[k][blk] of the dot products: src 0: V_k . V_{j+1}; 1: V_{j+1} . V_{j+1}; 2: b . b
__global__ void kb_dots(const SysDesc* __restrict__ D, int src, int j) {
    const SysDesc& S = D[blockIdx.z];
    if (!S.active || (int)blockIdx.x >= S.dot_blocks) return;
    const int k = blockIdx.y;
    const int64_t n = S.G.n;
    const double* a = src == 0 ? S.V + (int64_t)k * n : (src == 1 ? S.V + (int64_t)(j + 1) * n : S.b);
    const double* c = src == 2 ? S.b : S.V + (int64_t)(j + 1) * n;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < n; i += (int64_t)S.dot_blocks * BT)
        acc = fma(a[i], c[i], acc);
    __shared__ double red[BT];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = BT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) S.dotpart[k * S.dot_blocks + blockIdx.x] = red[0];
}

// dst 0: h1[k], 1: h2[k], 2: status[2] = sum over blocks of part[k][.]
__global__ void kb_reduce(const SysDesc* __restrict__ D, int nvec, int dst) {
    const SysDesc& S = D[blockIdx.x];
    if (!S.active) return;
    double* out = dst == 0 ? S.h1 : (dst == 1 ? S.h2 : S.status + 2);
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < S.dot_blocks; ++b) s += S.dotpart[k * S.dot_blocks + b];
        out[k] = s;
    }
}

// V_{j+1} -= sum_{k <= j} V_k h[k] (h = h1 or h2)
__global__ void kb_sub_proj(const SysDesc* __restrict__ D, int j, int which) {
    const SysDesc& S = D[blockIdx.y];
    if (!S.active) return;
    const int64_t n = S.G.n;
    if ((int64_t)blockIdx.x * BT >= n) return;
    __shared__ double hs[1024];
    const double* h = which ? S.h2 : S.h1;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) hs[k] = h[k];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i >= n) return;
    double* w = S.V + (int64_t)(j + 1) * n;
    double acc = w[i];
    for (int k = 0; k <= j; ++k) acc = fma(-S.V[(int64_t)k * n + i], hs[k], acc);
    w[i] = acc;
}

// Start: g = (beta, 0, ...), status[0] = status[1] = beta = sqrt(status[2]).
__global__ void kb_init(const SysDesc* __restrict__ D) {
    const SysDesc& S = D[blockIdx.x];
    if (!S.active || threadIdx.x != 0) return;
    const double beta = sqrt(fmax(S.status[2], 0.0));
    for (int k = 0; k <= S.m; ++k) S.gv[k] = 0.0;
    S.gv[0] = beta;
    S.status[0] = S.status[1] = beta;
}

// One Arnoldi column with the Givens update (as in the single-system solver).
__global__ void kb_arnoldi(const SysDesc* __restrict__ D, int j) {
    const SysDesc& S = D[blockIdx.x];
    if (!S.active || threadIdx.x != 0) return;
    const int ldh = S.m + 1;
    double* col = S.H + (int64_t)j * ldh;
    for (int k = 0; k <= j; ++k) col[k] = S.h1[k] + S.h2[k];
    const double hn = sqrt(fmax(S.status[2], 0.0));
    col[j + 1] = hn;
    S.status[1] = hn;
    for (int k = 0; k < j; ++k) {
        const double a = col[k], b = col[k + 1];
        col[k] = S.cs[k] * a + S.sn[k] * b;
        col[k + 1] = -S.sn[k] * a + S.cs[k] * b;
    }
    const double a = col[j], b = col[j + 1];
    const double den = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (den > 0.0) {
        c = a / den;
        s = b / den;
    }
    col[j] = den;
    col[j + 1] = 0.0;
    S.cs[j] = c;
    S.sn[j] = s;
    S.gv[j + 1] = -s * S.gv[j];
    S.gv[j] = c * S.gv[j];
    S.status[0] = fabs(S.gv[j + 1]);
    S.hist[2 * j] = S.status[0];
    S.hist[2 * j + 1] = hn;
}

// mode 0: V_0 = b / status[1]; mode 1: V_{j+1} /= status[1] (kept at an exact breakdown)
__global__ void kb_scale(const SysDesc* __restrict__ D, int j, int mode) {
    const SysDesc& S = D[blockIdx.y];
    if (!S.active) return;
    const int64_t n = S.G.n;
    const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i >= n) return;
    const double s = S.status[1];
    const double f = s > 0.0 ? 1.0 / s : 1.0;
    if (mode == 0) S.V[i] = S.b[i] * f;
    else S.V[(int64_t)(j + 1) * n + i] *= f;
}

// z_j = M^-1 V_j (FP32 block preconditioner), kept for the solution
__global__ void __launch_bounds__(BAPPLY_ROWS * BAPPLY_SLICES)
kb_precond(const SysDesc* __restrict__ D, int j) {
    extern __shared__ unsigned char kb_smem[];
    const SysDesc& S = D[blockIdx.z];
    if (!S.active || (int)blockIdx.x >= S.G.np || (int)blockIdx.y * BAPPLY_ROWS >= S.G.npp) return;
    blocks_apply_tile<float, false>(S.G.npp, S.G.shape_of, S.minv32, S.V + (int64_t)j * S.G.n,
                                    S.Zp + (int64_t)j * S.G.n, blockIdx.x,
                                    blockIdx.y * BAPPLY_ROWS, kb_smem);
}

// extra = FP32 self block x z_j (own-particle far pairs)
__global__ void __launch_bounds__(BAPPLY_ROWS * BAPPLY_SLICES)
kb_self(const SysDesc* __restrict__ D, int j) {
    extern __shared__ unsigned char kb_smem[];
    const SysDesc& S = D[blockIdx.z];
    if (!S.active || (int)blockIdx.x >= S.G.np || (int)blockIdx.y * BAPPLY_ROWS >= S.G.npp) return;
    blocks_apply_tile<float, false>(S.G.npp, S.G.shape_of, S.self32, S.Zp + (int64_t)j * S.G.n,
                                    S.extra, blockIdx.x, blockIdx.y * BAPPLY_ROWS, kb_smem);
}

// FP32 source records of z_j
__global__ void kb_src(const SysDesc* __restrict__ D, int j) {
    const SysDesc& S = D[blockIdx.y];
    if (!S.active) return;
    src_pairs_at(S.G, S.Zp + (int64_t)j * S.G.n, S.kpf, S.rec,
                 blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// extra += symmetric FP32 far field of the records
__global__ void __launch_bounds__(F32_TPB, 6) kb_sym(const SysDesc* __restrict__ D) {
    const SysDesc& S = D[blockIdx.y];
    if (!S.active || (int)blockIdx.x >= S.sym_blocks) return;
    sym_items<false>(S.G, S.rec, S.tasks, S.ntasks, S.qch, S.ipb, S.nw, S.kscale, S.extra,
                     blockIdx.x);
}

// V_{j+1} = extra + near QBX rows x z_j
__global__ void kb_assemble(const SysDesc* __restrict__ D, int j) {
    const SysDesc& S = D[blockIdx.y];
    if (!S.active) return;
    assemble_at(S.G, 0, nullptr, S.extra, S.G.cval, S.Zp + (int64_t)j * S.G.n,
                S.V + (int64_t)(j + 1) * S.G.n, blockIdx.x * (int64_t)BT + threadIdx.x);
}

// y = H(0:k1,0:k1)^-1 g(0:k1)
__global__ void kb_tri_solve(const SysDesc* __restrict__ D) {
    const SysDesc& S = D[blockIdx.x];
    if (!S.active || threadIdx.x != 0) return;
    const int ldh = S.m + 1;
    for (int r = S.k1 - 1; r >= 0; --r) {
        double s = S.gv[r];
        for (int c = r + 1; c < S.k1; ++c) s -= S.H[(int64_t)c * ldh + r] * S.ybuf[c];
        S.ybuf[r] = s / S.H[(int64_t)r * ldh + r];
    }
}

// x = sum_{k < k1} z_k y[k] (the solution M^-1 V y from a zero start, from the
// kept z_k, so that the FP32 preconditioner adds no rounding of its own)
__global__ void kb_add_basis(const SysDesc* __restrict__ D) {
    const SysDesc& S = D[blockIdx.y];
    if (!S.active) return;
    const int64_t n = S.G.n;
    if ((int64_t)blockIdx.x * BT >= n) return;
    __shared__ double ys[1024];
    for (int k = threadIdx.x; k < S.k1; k += blockDim.x) ys[k] = S.ybuf[k];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int k = 0; k < S.k1; ++k) acc = fma(S.Zp[(int64_t)k * n + i], ys[k], acc);
    S.x[i] = acc;
}

// out[s][0] = status[1] (mode 0), or out[s][2 b + {0,1}] = hist[2 (j0 + b) + {0,1}], b < k
__global__ void kb_gather(const SysDesc* __restrict__ D, int nsys, int mode, int j0, int k,
                          double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const SysDesc& S = D[s];
    double* o = out + (int64_t)s * 2 * BATCH_STEPS;
    if (mode == 0) o[0] = S.status[1];
    else
        for (int b = 0; b < 2 * k && j0 + b / 2 < S.m; ++b) o[b] = S.hist[2 * j0 + b];
}

__global__ void kb_set(SysDesc* __restrict__ D, int s, int active, int k1) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        D[s].active = active;
        D[s].k1 = k1;
    }
}

// z = a - b and x += d, per system (node-wise helpers of the refinement)
__global__ void kb_axpy_sub(double* __restrict__ sigma, const double* __restrict__ d,
                            int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) sigma[i] += d[i];
}
__global__ void kb_residual(double* __restrict__ r, const double* __restrict__ f,
                            const double* __restrict__ ax, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) r[i] = f[i] - ax[i];
}

// ---------------------------------------------------------------------------

static int batch_steps(double res, double prev, double tol_abs) {
    if (!(prev > 0.0) || !(res > 0.0) || !(res < prev)) return 1;
    const double need = log(tol_abs / res) / log(res / prev);
    if (!(need > 2.0)) return 1;
    return (int)std::min<double>(BATCH_STEPS, floor(need - 1.0));
}

static double* pinned(yk_ctx* ctx, size_t count) {
    if (ctx->h_batch_cap < count) {
        if (ctx->h_batch) cudaFreeHost(ctx->h_batch);
        ctx->h_batch = nullptr;
        ctx->h_batch_cap = 0;
        if (cudaMallocHost((void**)&ctx->h_batch, count * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->h_batch_cap = count;
    }
    return ctx->h_batch;
}

struct Inner {
    yk_geom* g;
    double tol_abs;
    int steps = 0;      // Arnoldi steps kept (k1)
    bool done = false;
    double prev = 0.0, res = 0.0;
};

// Lock-step GMRES on the FP32 inner operators: for every system s, solve
// A32_s x_s = b_s (x_s from 0) to ||b_s - A32_s x_s|| <= tol_abs_s, within one
// cycle of at most m steps.
static int batched_gmres(std::vector<Inner>& sys, const std::vector<const double*>& b,
                         const std::vector<double*>& x) {
    const int ns = (int)sys.size();
    yk_ctx* ctx = sys[0].g->ctx;
    cudaStream_t st = ctx->stream;
    std::vector<SysDesc> h(ns);
    int64_t max_n = 0;
    int max_np = 0, max_npp = 0, max_sym = 0, max_dot = 0, max_m = 0;
    for (int s = 0; s < ns; ++s) {
        yk_geom* g = sys[s].g;
        SymParams p;
        YK_TRY(sym_params(g, 0, &p));
        Workspace& w = g->ws;
        SysDesc& d = h[s];
        d.G = g->view();
        d.V = w.V;
        d.H = w.H;
        d.gv = w.gvec;
        d.cs = w.cs;
        d.sn = w.sn;
        d.h1 = w.hbuf;
        d.h2 = w.hbuf + (w.m + 2);
        d.ybuf = w.ybuf;
        d.dotpart = w.dotpart;
        d.status = w.status;
        d.hist = w.hist;
        if (!w.Zp) YK_TRY(dev_alloc((void**)&w.Zp, sizeof(double) * (size_t)w.m * g->n, st));
        d.Zp = w.Zp;
        d.extra = w.vec[5];
        d.rec = w.src4;
        d.minv32 = g->d_minv32;
        d.self32 = g->d_self32;
        d.tasks = p.tasks;
        d.b = b[s];
        d.x = x[s];
        d.kscale = p.kscale;
        d.kpf = (float)(LOG2E / g->prm.rho);
        d.ntasks = p.ntasks;
        d.qch = p.qch;
        d.ipb = p.ipb;
        d.nw = p.nw;
        d.sym_blocks = p.blocks;
        d.dot_blocks = w.dot_blocks;
        d.m = w.m;
        d.k1 = 0;
        d.active = 1;
        max_n = std::max<int64_t>(max_n, g->n);
        max_np = std::max(max_np, g->np);
        max_npp = std::max(max_npp, g->npp);
        max_sym = std::max(max_sym, p.blocks);
        max_dot = std::max(max_dot, w.dot_blocks);
        max_m = std::max(max_m, w.m);
    }
    SysDesc* D = nullptr;
    double* dgat = nullptr;
    YK_TRY(dev_alloc((void**)&D, sizeof(SysDesc) * ns, st));
    int rc = dev_alloc((void**)&dgat, sizeof(double) * 2 * BATCH_STEPS * ns, st);
    double* hg = pinned(ctx, (size_t)2 * BATCH_STEPS * ns);
    if (rc == YK_OK && !hg) rc = YK_ERR_NO_MEMORY;
    if (rc == YK_OK && cudaMemcpyAsync(D, h.data(), sizeof(SysDesc) * ns, cudaMemcpyHostToDevice,
                                       st) != cudaSuccess)
        rc = YK_ERR_CUDA;
    const int nb = ceil_div(max_n, BT);
    const int npairs = ceil_div((int64_t)max_np * ((max_npp + 1) / 2), BT);
    const dim3 gblk(max_np, ceil_div(max_npp, BAPPLY_ROWS), ns);
    const size_t smem = blocks_apply_smem<float>(max_npp);
    auto gather = [&](int mode, int j0, int k) -> int {
        YK_LAUNCH(kb_gather, ceil_div(ns, 64), 64, 0, st, D, ns, mode, j0, k, dgat);
        YK_TRY_CUDA(cudaMemcpyAsync(hg, dgat, sizeof(double) * 2 * BATCH_STEPS * ns,
                                    cudaMemcpyDeviceToHost, st));
        YK_TRY_CUDA(cudaStreamSynchronize(st));
        return YK_OK;
    };
    auto retire = [&](int s, int k1) {
        sys[s].done = true;
        sys[s].steps = k1;
        YK_LAUNCH(kb_set, 1, 32, 0, st, D, s, 0, k1);
    };
    if (rc == YK_OK) {
        // r = b, beta = ||b||, V_0 = b / beta
        YK_LAUNCH(kb_dots, dim3(max_dot, 1, ns), BT, 0, st, D, 2, 0);
        YK_LAUNCH(kb_reduce, ns, 128, 0, st, D, 1, 2);
        YK_LAUNCH(kb_init, ns, 32, 0, st, D);
        YK_LAUNCH(kb_scale, dim3(nb, ns), BT, 0, st, D, 0, 0);
        rc = gather(0, 0, 0);
    }
    int live = 0;
    if (rc == YK_OK) {
        for (int s = 0; s < ns; ++s) {
            const double beta = hg[(size_t)s * 2 * BATCH_STEPS];
            sys[s].prev = beta;
            sys[s].res = beta;
            if (!(beta > sys[s].tol_abs)) retire(s, 0);   // nothing to do (or b = 0)
            else ++live;
        }
    }
    int j = 0, batch = 1;
    while (rc == YK_OK && live > 0 && j < max_m) {
        // no live system may step past its own basis size m
        int room = max_m - j;
        for (int s = 0; s < ns; ++s)
            if (!sys[s].done) room = std::min(room, h[s].m - j);
        const int k = std::min(batch, room);
        for (int q = 0; q < k && rc == YK_OK; ++q) {
            const int jj = j + q;
            YK_LAUNCH(kb_precond, gblk, BAPPLY_ROWS * BAPPLY_SLICES, smem, st, D, jj);
            YK_LAUNCH(kb_src, dim3(npairs, ns), BT, 0, st, D, jj);
            YK_LAUNCH(kb_self, gblk, BAPPLY_ROWS * BAPPLY_SLICES, smem, st, D, jj);
            if (max_sym > 0) YK_LAUNCH(kb_sym, dim3(max_sym, ns), F32_TPB, 0, st, D);
            YK_LAUNCH(kb_assemble, dim3(nb, ns), BT, 0, st, D, jj);
            for (int pass = 0; pass < 2; ++pass) {   // CGS2
                YK_LAUNCH(kb_dots, dim3(max_dot, jj + 1, ns), BT, 0, st, D, 0, jj);
                YK_LAUNCH(kb_reduce, ns, 128, 0, st, D, jj + 1, pass);
                YK_LAUNCH(kb_sub_proj, dim3(nb, ns), BT, 0, st, D, jj, pass);
            }
            YK_LAUNCH(kb_dots, dim3(max_dot, 1, ns), BT, 0, st, D, 1, jj);
            YK_LAUNCH(kb_reduce, ns, 128, 0, st, D, 1, 2);
            YK_LAUNCH(kb_arnoldi, ns, 32, 0, st, D, jj);
            YK_LAUNCH(kb_scale, dim3(nb, ns), BT, 0, st, D, jj, 1);
            if (cudaGetLastError() != cudaSuccess) rc = YK_ERR_CUDA;
        }
        if (rc == YK_OK) rc = gather(1, j, k);
        if (rc != YK_OK) break;
        batch = BATCH_STEPS;
        for (int s = 0; s < ns; ++s) {
            Inner& I = sys[s];
            if (I.done) continue;
            const double* o = hg + (size_t)s * 2 * BATCH_STEPS;
            int used = -1;
            for (int q = 0; q < k && j + q < h[s].m; ++q) {
                const double r = o[2 * q], hn = o[2 * q + 1];
                I.prev = I.res;
                I.res = r;
                if (r <= I.tol_abs || hn == 0.0 || !isfinite(r)) {
                    used = q + 1;
                    break;
                }
            }
            if (used > 0) {
                retire(s, j + used);
                --live;
            } else if (j + k >= h[s].m) {   // the cycle is full: keep what it has
                retire(s, h[s].m);
                --live;
            } else {
                batch = std::min(batch, batch_steps(I.res, I.prev, I.tol_abs));
            }
        }
        j += k;
    }
    // x = M^-1 V y = Z y for every system with steps (x = 0 for the others)
    if (rc == YK_OK) {
        for (int s = 0; s < ns; ++s) {
            if (sys[s].steps > 0) YK_LAUNCH(kb_set, 1, 32, 0, st, D, s, 1, sys[s].steps);
            else if (cudaMemsetAsync(x[s], 0, sizeof(double) * sys[s].g->n, st) != cudaSuccess)
                rc = YK_ERR_CUDA;
        }
        YK_LAUNCH(kb_tri_solve, ns, 32, 0, st, D);
        YK_LAUNCH(kb_add_basis, dim3(nb, ns), BT, 0, st, D);
        if (cudaGetLastError() != cudaSuccess) rc = YK_ERR_CUDA;
    }
    dev_free(D, st);
    dev_free(dgat, st);
    return rc;
}

static bool batchable(yk_geom* g) {
    const yk_params& P = g->prm;
    if (P.precision != YK_MIXED || P.farfield != YK_FARFIELD_DENSE) return false;
    if (!g->use_self || P.precond != YK_PRECOND_BLOCK || !g->d_minv32) return false;
    if (g->npp > 1024 || P.gmres_restart > 1000) return false;
    int ntgt = 0;
    if (contact_targets(g, &ntgt) != YK_OK || ntgt > 0) return false;
    return true;
}

int solve_batch(yk_geom* const* gs, int count, const double* const* f, double* const* sigma,
                yk_solve_info* info) {
    int first_rc = YK_OK;
    auto note = [&](int rc) {
        if (first_rc == YK_OK || (first_rc == YK_ERR_NOT_CONVERGED && rc != YK_OK)) first_rc = rc;
    };
    std::vector<int> idx;
    for (int s = 0; s < count; ++s) {
        if (batchable(gs[s])) {
            idx.push_back(s);
        } else {
            yk_solve_info inf{};
            const int rc = solve(gs[s], f[s], sigma[s], nullptr, &inf);
            if (info) info[s] = inf;
            if (rc != YK_OK) note(rc);
        }
    }
    if (idx.empty()) return first_rc;
    cudaStream_t st = gs[idx[0]]->ctx->stream;
    const int nsys = (int)idx.size();
    std::vector<double> fn(nsys), rel(nsys);
    std::vector<yk_solve_info> inf(nsys);
    // sigma = 0, r = f
    for (int q = 0; q < nsys; ++q) {
        yk_geom* g = gs[idx[q]];
        const size_t bytes = sizeof(double) * g->n;
        YK_TRY_CUDA(cudaMemsetAsync(sigma[idx[q]], 0, bytes, st));
        YK_TRY_CUDA(cudaMemcpyAsync(g->ws.vec[1], f[idx[q]], bytes, cudaMemcpyDeviceToDevice, st));
        fn[q] = device_norm2(g, f[idx[q]]);
        rel[q] = fn[q] > 0.0 ? 1.0 : 0.0;
    }
    for (int ref = 0;; ++ref) {
        std::vector<Inner> sys;
        std::vector<int> who;
        std::vector<const double*> b;
        std::vector<double*> x;
        for (int q = 0; q < nsys; ++q) {
            yk_geom* g = gs[idx[q]];
            const yk_params& P = g->prm;
            if (!(rel[q] > P.gmres_tol) || inf[q].refinements >= P.max_refine ||
                inf[q].iterations >= P.max_iter)
                continue;
            Inner I;
            I.g = g;
            I.tol_abs = inner_tolerance(P, rel[q]) * rel[q] * fn[q];
            sys.push_back(I);
            who.push_back(q);
            b.push_back(g->ws.vec[1]);
            x.push_back(g->ws.vec[2]);
        }
        if (sys.empty()) break;
        YK_TRY(batched_gmres(sys, b, x));
        for (size_t k = 0; k < sys.size(); ++k) {
            const int q = who[k];
            yk_geom* g = gs[idx[q]];
            const int64_t n = g->n;
            double* sg = sigma[idx[q]];
            inf[q].iterations += sys[k].steps;
            inf[q].matvecs_fp32 += sys[k].steps;
            YK_LAUNCH(kb_axpy_sub, ceil_div(n, 256), 256, 0, st, sg, g->ws.vec[2], n);
            YK_TRY(matvec(g, sg, g->ws.vec[3], Prec::SPLIT));
            YK_LAUNCH(kb_residual, ceil_div(n, 256), 256, 0, st, g->ws.vec[1], f[idx[q]],
                      g->ws.vec[3], n);
            inf[q].matvecs_fp64++;
            inf[q].refinements++;
            rel[q] = device_norm2(g, g->ws.vec[1]) / fn[q];
        }
    }
    for (int q = 0; q < nsys; ++q) {
        inf[q].rel_residual = rel[q];
        if (info) info[idx[q]] = inf[q];
        if (!(rel[q] <= gs[idx[q]]->prm.gmres_tol)) note(YK_ERR_NOT_CONVERGED);
    }
    YK_TRY_CUDA(cudaGetLastError());
    return first_rc;
}

}  // namespace yk
