// Device GMRES for 1/2 sigma + D sigma = f (Eq. bie; Algorithm 1, GMRES
// step) and the mixed-precision iterative refinement around it.
//
// GMRES: Arnoldi with classical Gram-Schmidt applied twice (CGS2) on an
// FP64 Krylov basis, Givens rotations on the Hessenberg matrix, restart
// after m steps. Every vector operation, the rotations and the small
// triangular solve run on the device. The host enqueues up to
// GMRES_BATCH Arnoldi steps at a time, as many as the residual's recent
// rate of decrease says are still needed, and then reads the residual
// estimates those steps left in a device history. Steps after the first
// one that met the tolerance only write later Hessenberg columns and
// right-hand-side entries, so the solution is formed from the steps up to
// that one, exactly as if the host had stopped there.
//
// Mixed: sigma <- sigma + GMRES_32(r), r = f - A_64 sigma, where A_32 is
// the FP32-far-field operator (accurate to about 1e-6) and A_64 the
// FP64-accurate precision-split operator; stops when ||r|| <= tol ||f||.
// With a right preconditioner the z_j = M^{-1} v_j are kept and a cycle's
// correction is Z y (the form of flexible GMRES), so an FP32 M adds no
// rounding of its own to the correction. The FP32 GMRES may be deflated by
// a coarse space (coarse.cu): each Arnoldi column A z_j is then corrected to
// the deflated operator's, and the correction by the coarse term.
#include <math.h>

#include <algorithm>
#include <functional>

#include "yk_internal.cuh"

namespace yk {

constexpr int DOT_TPB = 256;

// part[k * nblk + b] = sum over block b's slice of V[k][i] * w[i]
__global__ void k_dots(const double* __restrict__ V, int64_t n, const double* __restrict__ w,
                       double* __restrict__ part) {
    const int k = blockIdx.y;
    const double* v = V + (int64_t)k * n;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)DOT_TPB + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * DOT_TPB)
        acc = fma(v[i], w[i], acc);
    __shared__ double red[DOT_TPB];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = DOT_TPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_reduce_parts(int nvec, int nblk, const double* __restrict__ part,
                               double* __restrict__ out) {
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[k * nblk + b];
        out[k] = s;
    }
}

// w -= sum_k V[k] h[k]
__global__ void k_sub_proj(double* __restrict__ w, const double* __restrict__ V, int64_t n,
                           int nvec, const double* __restrict__ h) {
    __shared__ double hs[1024];
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) hs[k] = h[k];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int k = 0; k < nvec; ++k) acc = fma(-V[(int64_t)k * n + i], hs[k], acc);
    w[i] = acc;
}

// One Arnoldi column: H[:, j] = h1 + h2, H[j+1, j] = ||w||, previous
// rotations, a new rotation, and the residual estimate |g[j+1]|.
// status[0] = residual estimate, status[1] = ||w|| (before normalisation);
// hist[2 j], hist[2 j + 1] keep the same two numbers for step j.
__global__ void k_arnoldi_col(int j, int ldh, double* H, const double* h1, const double* h2,
                              const double* wn2, double* cs, double* sn, double* g,
                              double* status, double* hist) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* col = H + (int64_t)j * ldh;
    for (int k = 0; k <= j; ++k) col[k] = h1[k] + h2[k];
    const double hn = sqrt(fmax(wn2[0], 0.0));
    col[j + 1] = hn;
    status[1] = hn;
    for (int k = 0; k < j; ++k) {
        const double a = col[k], b = col[k + 1];
        col[k] = cs[k] * a + sn[k] * b;
        col[k + 1] = -sn[k] * a + cs[k] * b;
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
    cs[j] = c;
    sn[j] = s;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    status[0] = fabs(g[j + 1]);
    hist[2 * j] = status[0];
    hist[2 * j + 1] = hn;
}

// dst = src / s[0] (unchanged when s[0] = 0, an exact breakdown), or
// dst = src * scale when s == nullptr
__global__ void k_scale(double* dst, const double* src, int64_t n, const double* s,
                        double scale) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = s ? (s[0] > 0.0 ? 1.0 / s[0] : 1.0) : scale;
    dst[i] = src[i] * f;
}

// Start a cycle: g = (beta, 0, ...), status[1] = beta.
__global__ void k_init_cycle(int m, const double* bn2, double* g, double* status) {
    if (threadIdx.x != 0) return;
    const double beta = sqrt(fmax(bn2[0], 0.0));
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta;
    status[1] = beta;
    status[0] = beta;
}

// y = H(0:k,0:k)^{-1} g(0:k), back substitution (k+1 unknowns)
__global__ void k_tri_solve(int k1, int ldh, const double* H, const double* g, double* y) {
    if (threadIdx.x != 0) return;
    for (int r = k1 - 1; r >= 0; --r) {
        double s = g[r];
        for (int c = r + 1; c < k1; ++c) s -= H[(int64_t)c * ldh + r] * y[c];
        y[r] = s / H[(int64_t)r * ldh + r];
    }
}

// x += sum_k V[k] y[k]
__global__ void k_add_basis(double* __restrict__ x, const double* __restrict__ V, int64_t n,
                            int k1, const double* __restrict__ y) {
    __shared__ double ys[1024];
    for (int k = threadIdx.x; k < k1; k += blockDim.x) ys[k] = y[k];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = x[i];
    for (int k = 0; k < k1; ++k) acc = fma(V[(int64_t)k * n + i], ys[k], acc);
    x[i] = acc;
}

// z = a - b
__global__ void k_sub(double* z, const double* a, const double* b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = a[i] - b[i];
}

// x += d
__global__ void k_axpy1(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] += d[i];
}

// ---------------------------------------------------------------------------

int alloc_krylov(Workspace& w, int64_t n, int m, cudaStream_t st) {
    w.m = m;
    w.dot_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(296, (n + 2047) / 2048));
    YK_TRY(dev_alloc((void**)&w.V, sizeof(double) * (m + 1) * n, st));
    YK_TRY(dev_alloc((void**)&w.H, sizeof(double) * (m + 1) * m, st));
    YK_TRY(dev_alloc((void**)&w.gvec, sizeof(double) * (m + 1), st));
    YK_TRY(dev_alloc((void**)&w.cs, sizeof(double) * m, st));
    YK_TRY(dev_alloc((void**)&w.sn, sizeof(double) * m, st));
    YK_TRY(dev_alloc((void**)&w.hbuf, sizeof(double) * 2 * (m + 2), st));
    YK_TRY(dev_alloc((void**)&w.ybuf, sizeof(double) * (m + 1), st));
    YK_TRY(dev_alloc((void**)&w.dotpart, sizeof(double) * (m + 2) * w.dot_blocks, st));
    YK_TRY(dev_alloc((void**)&w.status, sizeof(double) * 8, st));
    YK_TRY(dev_alloc((void**)&w.hist, sizeof(double) * 2 * (m + 1), st));
    for (int k = 0; k < 8; ++k) YK_TRY(dev_alloc((void**)&w.vec[k], sizeof(double) * n, st));
    return YK_OK;
}

int alloc_workspace(yk_geom* g) {
    Workspace& w = g->ws;
    cudaStream_t st = g->ctx->stream;
    const int64_t n = g->n;
    const int nct = ceil_div(n, 256);
    int nchunk = std::max(1, std::min(g->np, ceil_div(152 * 32, nct)));
    const int ppc = ceil_div(g->np, nchunk);
    w.nchunk = ceil_div(g->np, ppc);
    YK_TRY(dev_alloc((void**)&w.partial, sizeof(double) * w.nchunk * n, st));
    YK_TRY(dev_alloc((void**)&w.src4, sizeof(float4) * 2 * (size_t)g->np * ((g->npp + 1) / 2), st));
    YK_TRY(dev_alloc((void**)&w.src4g, sizeof(float4) * 3 * (size_t)g->np * ((g->npp + 1) / 2),
                     st));
    YK_TRY(alloc_krylov(w, n, g->prm.gmres_restart, st));
    if (!host_status(g->ctx)) return YK_ERR_NO_MEMORY;
    return YK_OK;
}

void free_workspace(Workspace& w, cudaStream_t st) {
    dev_free(w.partial, st);
    dev_free(w.src4, st);
    dev_free(w.src4g, st);
    dev_free(w.V, st);
    dev_free(w.Zp, st);
    dev_free(w.H, st);
    dev_free(w.gvec, st);
    dev_free(w.cs, st);
    dev_free(w.sn, st);
    dev_free(w.hbuf, st);
    dev_free(w.ybuf, st);
    dev_free(w.dotpart, st);
    dev_free(w.status, st);
    dev_free(w.hist, st);
    for (int k = 0; k < 8; ++k) dev_free(w.vec[k], st);
    w = Workspace{};
}

void free_workspace(yk_geom* g) { free_workspace(g->ws, g->ctx->stream); }

// out[0..nvec) = V[0..nvec)^T w
static void dots(const KrylovOp& op, const double* V, int nvec, const double* w, double* out) {
    cudaStream_t st = op.ctx->stream;
    dim3 grid(op.ws->dot_blocks, nvec);
    YK_LAUNCH(k_dots, grid, DOT_TPB, 0, st, V, op.n, w, op.ws->dotpart);
    YK_LAUNCH(k_reduce_parts, 1, 128, 0, st, nvec, op.ws->dot_blocks, op.ws->dotpart, out);
}

static int read_status(const KrylovOp& op, double* s0, double* s1) {
    cudaStream_t st = op.ctx->stream;
    double* hs = op.ctx->h_status;
    YK_TRY_CUDA(cudaMemcpyAsync(hs, op.ws->status, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    *s0 = hs[0];
    *s1 = hs[1];
    return YK_OK;
}

// Arnoldi steps enqueued before the host looks at the residuals (at most
// four (residual, norm) pairs fit the pinned status mirror).
constexpr int GMRES_BATCH = 4;

// Reads the history of steps [j0, j0 + k) into res[], hn[].
static int read_hist(const KrylovOp& op, int j0, int k, double* res, double* hn) {
    cudaStream_t st = op.ctx->stream;
    double* hs = op.ctx->h_status;
    YK_TRY_CUDA(cudaMemcpyAsync(hs, op.ws->hist + 2 * j0, 2 * k * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < k; ++i) {
        res[i] = hs[2 * i];
        hn[i] = hs[2 * i + 1];
    }
    return YK_OK;
}

// Steps to enqueue next: as many as a geometric decrease at the last
// observed rate needs to reach tol_abs, less one, within [1, GMRES_BATCH].
static int next_batch(double res, double prev, double tol_abs) {
    if (!(prev > 0.0) || !(res > 0.0) || !(res < prev)) return 1;
    const double need = log(tol_abs / res) / log(res / prev);
    if (!(need > 2.0)) return 1;
    return (int)std::min<double>(GMRES_BATCH, floor(need - 1.0));
}

// GMRES on A(prec) x = b with initial guess x (x_zero: x is taken as 0).
// Stops when the residual estimate <= tol_abs. Returns iterations used.
static int gmres(const KrylovOp& op, Prec prec, const double* b, double* x, bool x_zero,
                 double tol_abs, int max_iter, int* iters_out, double* res_out, int* matvecs) {
    Workspace& w = *op.ws;
    cudaStream_t st = op.ctx->stream;
    const int64_t n = op.n;
    const int m = w.m;
    const int ldh = m + 1;
    const int nb = ceil_div(n, 256);
    const bool pc = (bool)op.precond;
    const bool defl = pc && prec == Prec::F32 && (bool)op.deflate;
    double* r = w.vec[0];
    double* h1 = w.hbuf;
    double* h2 = w.hbuf + (m + 2);
    if (pc && !w.Zp) YK_TRY(dev_alloc((void**)&w.Zp, sizeof(double) * (size_t)m * n, st));
    int total = 0;
    double res = INFINITY;
    bool have_x = !x_zero;
    if (x_zero) YK_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    while (true) {
        // r = b - A x
        if (have_x) {
            YK_TRY(op.apply(x, r, prec));
            ++*matvecs;
            YK_LAUNCH(k_sub, nb, 256, 0, st, r, b, r, n);
        } else {
            YK_TRY_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        }
        dots(op, r, 1, r, w.status + 2);
        YK_LAUNCH(k_init_cycle, 1, 32, 0, st, m, w.status + 2, w.gvec, w.status);
        double beta, dummy;
        YK_TRY(read_status(op, &beta, &dummy));
        res = beta;
        if (beta <= tol_abs || beta == 0.0 || total >= max_iter) break;
        YK_LAUNCH(k_scale, nb, 256, 0, st, w.V, r, n, w.status + 1, 0.0);
        int j = 0;
        bool done = false;
        double prev = beta;
        int batch = 1;
        while (j < m && total < max_iter && !done) {
            const int k = std::min(batch, std::min(m - j, max_iter - total));
            for (int b = 0; b < k; ++b) {
                const int jj = j + b;
                const double* vj = w.V + (int64_t)jj * n;
                double* wv = w.V + (int64_t)(jj + 1) * n;
                if (pc) {   // right preconditioning: w = A z_j, z_j = M^{-1} v_j kept
                    double* zj = w.Zp + (int64_t)jj * n;
                    YK_TRY(op.precond(vj, zj, prec == Prec::F32));
                    YK_TRY(op.apply(zj, wv, prec));
                } else {
                    YK_TRY(op.apply(vj, wv, prec));
                }
                ++*matvecs;
                if (defl) YK_TRY(op.deflate(vj, wv, jj));
                // CGS2
                dots(op, w.V, jj + 1, wv, h1);
                YK_LAUNCH(k_sub_proj, nb, 256, 0, st, wv, w.V, n, jj + 1, h1);
                dots(op, w.V, jj + 1, wv, h2);
                YK_LAUNCH(k_sub_proj, nb, 256, 0, st, wv, w.V, n, jj + 1, h2);
                dots(op, wv, 1, wv, w.status + 2);
                YK_LAUNCH(k_arnoldi_col, 1, 32, 0, st, jj, ldh, w.H, h1, h2, w.status + 2, w.cs,
                          w.sn, w.gvec, w.status, w.hist);
                YK_LAUNCH(k_scale, nb, 256, 0, st, wv, wv, n, w.status + 1, 0.0);
            }
            double rs[GMRES_BATCH], hs[GMRES_BATCH];
            YK_TRY(read_hist(op, j, k, rs, hs));
            int used = k;   // steps kept: up to the first that stops the cycle
            for (int b = 0; b < k; ++b) {
                if (rs[b] <= tol_abs || hs[b] == 0.0 || !isfinite(rs[b])) {
                    used = b + 1;
                    done = true;
                    break;
                }
            }
            res = rs[used - 1];
            const double before = used >= 2 ? rs[used - 2] : prev;
            prev = rs[used - 1];
            j += used;
            total += used;
            batch = done ? 1 : next_batch(res, before, tol_abs);
        }
        // x += V y
        YK_LAUNCH(k_tri_solve, 1, 32, 0, st, j, ldh, w.H, w.gvec, w.ybuf);
        if (pc) {
            // x += M^{-1} V y = Z y from the kept z_j (a fresh application of an
            // FP32 M would add its own rounding to the correction); deflated:
            // x += M^{-1} P V y = Z y - (M^{-1} Z_c) C sum_k y_k u_k
            YK_LAUNCH(k_add_basis, nb, 256, 0, st, x, w.Zp, n, j, w.ybuf);
            if (defl) YK_TRY(op.deflate_end(j, w.ybuf, x));
        } else {
            YK_LAUNCH(k_add_basis, nb, 256, 0, st, x, w.V, n, j, w.ybuf);
        }
        have_x = true;
        YK_TRY_CUDA(cudaGetLastError());
        if (done || total >= max_iter || !isfinite(res)) break;
    }
    *iters_out = total;
    *res_out = res;
    return YK_OK;
}

// The inner (FP32) solve's relative tolerance in a refinement step taken at
// relative residual rel: no tighter than what brings rel to gmres_tol with a
// 10x margin, no looser than 0.1, and not below inner_tol.
double inner_tolerance(const yk_params& P, double rel) {
    return std::max(P.inner_tol, std::min(0.1, 0.1 * P.gmres_tol / rel));
}

static double norm2(const KrylovOp& op, const double* v) {
    dots(op, v, 1, v, op.ws->status + 2);
    cudaStream_t st = op.ctx->stream;
    double* hs = op.ctx->h_status;
    cudaMemcpyAsync(hs + 2, op.ws->status + 2, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return sqrt(hs[2]);
}

KrylovOp yukawa_op(yk_geom* g) {
    KrylovOp op;
    op.ctx = g->ctx;
    op.ws = &g->ws;
    op.n = g->n;
    op.apply = [g](const double* x, double* y, Prec p) { return matvec(g, x, y, p); };
    if (g->prm.precond == YK_PRECOND_BLOCK)
        op.precond = [g](const double* x, double* y, bool f32) {
            return apply_preconditioner(g, x, y, f32);
        };
    if (g->coarse.on) {
        op.deflate = [g](const double* v, double* w, int j) { return coarse_deflate(g, v, w, j); };
        op.deflate_end = [g](int k, const double* y, double* t) {
            return coarse_correct(g, k, y, t);
        };
    }
    return op;
}

double device_norm2(yk_geom* g, const double* v) { return norm2(yukawa_op(g), v); }

int solve_op(const KrylovOp& op, const yk_params& P, Prec residual, const double* f,
             double* sigma, const double* sigma0, yk_solve_info* info) {
    cudaStream_t st = op.ctx->stream;
    const int64_t n = op.n;
    const int nb = ceil_div(n, 256);
    yk_solve_info inf{};
    const double fn = norm2(op, f);
    if (fn == 0.0) {
        YK_TRY_CUDA(cudaMemsetAsync(sigma, 0, sizeof(double) * n, st));
        if (info) *info = inf;
        return YK_OK;
    }
    if (sigma0 && sigma0 != sigma)
        YK_TRY_CUDA(cudaMemcpyAsync(sigma, sigma0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    int rc = YK_OK;
    if (P.precision == YK_FP64) {
        int it = 0, nmv = 0;
        double res = 0.0;
        YK_TRY(gmres(op, Prec::F64, f, sigma, sigma0 == nullptr, P.gmres_tol * fn, P.max_iter, &it,
                     &res, &nmv));
        inf.iterations = it;
        inf.rel_residual = res / fn;
        inf.matvecs_fp64 = nmv;
        if (!(inf.rel_residual <= P.gmres_tol)) rc = YK_ERR_NOT_CONVERGED;
    } else {
        double* r = op.ws->vec[1];
        double* d = op.ws->vec[2];
        double* ax = op.ws->vec[3];
        if (sigma0) {
            YK_TRY(op.apply(sigma, ax, residual));
            YK_LAUNCH(k_sub, nb, 256, 0, st, r, f, ax, n);
            inf.matvecs_fp64++;
        } else {
            YK_TRY_CUDA(cudaMemsetAsync(sigma, 0, sizeof(double) * n, st));
            YK_TRY_CUDA(cudaMemcpyAsync(r, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        }
        double rel = norm2(op, r) / fn;
        int total = 0;
        int ref = 0;
        while (rel > P.gmres_tol && ref < P.max_refine && total < P.max_iter) {
            const double rn = rel * fn;
            const double itol = inner_tolerance(P, rel);
            int it = 0, nmv = 0;
            double res = 0.0;
            YK_TRY(gmres(op, Prec::F32, r, d, true, itol * rn, P.max_iter - total, &it, &res,
                         &nmv));
            total += it;
            inf.matvecs_fp32 += nmv;
            YK_LAUNCH(k_axpy1, nb, 256, 0, st, sigma, d, n);
            YK_TRY(op.apply(sigma, ax, residual));
            YK_LAUNCH(k_sub, nb, 256, 0, st, r, f, ax, n);
            inf.matvecs_fp64++;
            rel = norm2(op, r) / fn;
            ++ref;
        }
        inf.iterations = total;
        inf.refinements = ref;
        inf.rel_residual = rel;
        if (!(rel <= P.gmres_tol)) rc = YK_ERR_NOT_CONVERGED;
    }
    YK_TRY_CUDA(cudaGetLastError());
    if (info) *info = inf;
    return rc;
}

int solve(yk_geom* g, const double* f, double* sigma, const double* sigma0,
          yk_solve_info* info) {
    YK_TRY(coarse_prepare(g));
    const int rc = solve_op(yukawa_op(g), g->prm, Prec::SPLIT, f, sigma, sigma0, info);
    if (info) info->coarse_dim = g->coarse.on ? g->coarse.nc : 0;
    return rc;
}

}  // namespace yk
