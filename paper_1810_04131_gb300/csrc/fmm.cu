// Fast multipole far field for the FP32 inner operator of the mixed solver
// (YK_FARFIELD_FMM). The paper evaluates its far field with an FMM inside
// GIGAQBX (Section 5); this is a uniform quadtree over the particle centres
// with expansions from Graf's addition theorem in its Yukawa form (Eq.
// graf-addition with K0(z) = (i pi/2) H0(iz)). All of it runs in FP64; the
// direct part runs in the FP32 P2P kernels.
//
// With w_j sigma_j nu_j the double-layer weights of the nodes y_j and z = r/rho:
//   P2M  (about centre c)   M_n = sum_j w_j sigma_j nu_j . grad_y[I_n(|y-c|/rho) e^{-i n phi}]
//        u(x) = (1/2pi) sum_n M_n K_n(|x-c|/rho) e^{i n theta}, M_{-n} = conj M_n
//   M2M  (child c to parent c', t = c - c')
//        M'_k = sum_n M_n I_{k-n}(|t|/rho) e^{-i (k-n) arg t}
//   M2L  (source c_s to target c_t, D = c_t - c_s)
//        L_m = (-1)^m sum_n M_n K_{n+m}(|D|/rho) e^{i (n+m) arg D}
//   L2L  (parent c to child c'' = c + s)
//        L''_j = sum_m L_m I_{m-j}(|s|/rho) e^{-i (m-j) arg s}
//   L2P  u(x) = (1/2pi) sum_m L_m I_m(|x-c|/rho) e^{-i m arg(x-c)}, L_{-m} = conj L_m
// M2M and L2L follow from the addition theorem of I_n (exact for all
// offsets); M2L from that of K_n, which needs the source and target discs to
// be disjoint. Orders are truncated at |n| <= p.
//
// Tree: the root is the bounding square of the particle centres; a particle
// belongs to the leaf holding its centre, so its nodes lie within
// a_l = b_l / sqrt(2) + R of its box centre at level l (R the largest bounding
// radius). Leaves at most FMM_SEP boxes apart (Chebyshev distance) interact
// directly; the interaction list of a box is the children of its parent's
// near boxes that are not near it. With FMM_SEP = 2 the centres of an
// interacting pair are at least 3 b_l apart, so the two discs are disjoint
// once b_l > 2R / (3 - sqrt 2); the leaf sizes offered to the autotuner keep
// the convergence ratio 2 a_l / (3 b_l) at most 0.7 and a_l / rho below
// 3p/4. The screened kernel decays like e^{-gap/rho}: interactions across
// gaps larger than the cut-off gap (at most 60 rho) are left out, and so are
// the coarse levels whose closest interacting pair is beyond it.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bessel.cuh"
#include "yk_internal.cuh"

namespace yk {

// defined in p2p.cu: exclusive scan of n counts into off[0..n]
__global__ void k_scan_offsets(int np, const int* __restrict__ counts, int* __restrict__ off);

static_assert(FMM_LMAX + 1 <= (int)(sizeof(FmmTree::use32) / sizeof(bool)), "use32 holds every level");

static inline int64_t level_offset(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }

// ---------------------------------------------------------------------------
// Tree build: leaf of each particle, particles by leaf (sorted by index within
// a leaf, so every sum runs in a fixed order), box counts, near lists.
// ---------------------------------------------------------------------------
__global__ void k_fmm_leaf_count(int np, const d4* __restrict__ part, double x0, double y0,
                                 double inv_b, int nb, int* __restrict__ leaf_of,
                                 int* __restrict__ counts) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= np) return;
    const d4 c = part[P];
    const int ix = min(max((int)floor((c.x - x0) * inv_b), 0), nb - 1);
    const int iy = min(max((int)floor((c.y - y0) * inv_b), 0), nb - 1);
    const int leaf = iy * nb + ix;
    leaf_of[P] = leaf;
    atomicAdd(&counts[leaf], 1);
}

__global__ void k_fmm_leaf_fill(int np, const int* __restrict__ leaf_of,
                                const int* __restrict__ leaf_off, int* __restrict__ cursor,
                                int* __restrict__ leaf_part) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= np) return;
    const int leaf = leaf_of[P];
    leaf_part[leaf_off[leaf] + atomicAdd(&cursor[leaf], 1)] = P;
}

// Insertion sort of each leaf's (short) particle list.
__global__ void k_fmm_leaf_sort(int nleaf, const int* __restrict__ leaf_off,
                                int* __restrict__ leaf_part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nleaf) return;
    const int a = leaf_off[k], b = leaf_off[k + 1];
    for (int i = a + 1; i < b; ++i) {
        const int v = leaf_part[i];
        int j = i - 1;
        while (j >= a && leaf_part[j] > v) {
            leaf_part[j + 1] = leaf_part[j];
            --j;
        }
        leaf_part[j + 1] = v;
    }
}

__global__ void k_fmm_count_leaves(int nleaf, const int* __restrict__ leaf_off,
                                   int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nleaf) cnt[k] = leaf_off[k + 1] - leaf_off[k];
}

// counts of level l from level l + 1 (cnt_l and cnt_c are the levels' slices)
__global__ void k_fmm_count_up(int l, const int* __restrict__ cnt_c, int* __restrict__ cnt_l) {
    const int nl = 1 << l;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nl * nl) return;
    const int i = k % nl, j = k / nl, nc = 2 * nl;
    cnt_l[k] = cnt_c[(2 * j) * nc + 2 * i] + cnt_c[(2 * j) * nc + 2 * i + 1] +
               cnt_c[(2 * j + 1) * nc + 2 * i] + cnt_c[(2 * j + 1) * nc + 2 * i + 1];
}

// Near list of target particle Q: the particles of the leaves at most
// FMM_SEP boxes from Q's leaf (Q included), leaf by leaf in row order.
template <bool FILL>
__global__ void k_fmm_near(int np, int nb, const int* __restrict__ leaf_of,
                           const int* __restrict__ leaf_off, const int* __restrict__ leaf_part,
                           int* __restrict__ counts, const int* __restrict__ near_off,
                           int* __restrict__ near) {
    const int Q = blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= np) return;
    const int leaf = leaf_of[Q];
    const int i = leaf % nb, j = leaf / nb;
    int c = 0;
    int k = FILL ? near_off[Q] : 0;
    for (int jj = max(j - FMM_SEP, 0); jj <= min(j + FMM_SEP, nb - 1); ++jj)
        for (int ii = max(i - FMM_SEP, 0); ii <= min(i + FMM_SEP, nb - 1); ++ii) {
            const int n = jj * nb + ii;
            const int a = leaf_off[n], b = leaf_off[n + 1];
            if (FILL)
                for (int t = a; t < b; ++t) near[k++] = leaf_part[t];
            else
                c += b - a;
        }
    if (!FILL) counts[Q] = c;
}

// ---------------------------------------------------------------------------
// Expansions (FP64). One warp per box; lane m holds order m (m <= p).
// ---------------------------------------------------------------------------

// e^{i k pi/4}: the offsets of a box's children (and of a child from its
// parent) lie at odd multiples of pi/4.
__constant__ double2 c_w8[8] = {{1.0, 0.0},        {M_SQRT1_2, M_SQRT1_2},
                                {0.0, 1.0},        {-M_SQRT1_2, M_SQRT1_2},
                                {-1.0, 0.0},       {-M_SQRT1_2, -M_SQRT1_2},
                                {0.0, -1.0},       {M_SQRT1_2, -M_SQRT1_2}};
__device__ __forceinline__ double2 w8(int k) { return c_w8[k & 7]; }
// quadrant (qx, qy) of a child relative to its parent's centre, in units of pi/4
__device__ __forceinline__ int quadrant_angle(int qx, int qy) {
    return qy ? (qx ? 1 : 3) : (qx ? 7 : 5);
}

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// P2M about each leaf centre (leaf level slice M). The moments feed only
// the FP32 inner operator, so the sums run in FP32; I_n comes from the FP64
// series and recurrence (FP32 would underflow at high orders). With a fixed
// order PF (the default 12) the moments stay in registers and I_n is taken
// in FP32 (bessel_i_down_f) wherever s/rho >= BESSEL_I_F32_XMIN.
template <int PF>
__global__ void __launch_bounds__(128) k_fmm_p2m(GeomView G, const double* __restrict__ sigma,
                                                 int p_rt, int nb, double x0, double y0, double b,
                                                 const int* __restrict__ leaf_off,
                                                 const int* __restrict__ leaf_part,
                                                 double2* __restrict__ M) {
    constexpr int NP = PF > 0 ? PF : FMM_PMAX;            // array bound, loop bound if fixed
    const int p = PF > 0 ? PF : p_rt;
    const int leaf = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (leaf >= nb * nb) return;
    const int t0 = leaf_off[leaf], t1 = leaf_off[leaf + 1];
    if (t0 == t1) return;                                  // warp-uniform
    const double cx = x0 + (leaf % nb + 0.5) * b, cy = y0 + (leaf / nb + 0.5) * b;
    const double rho = G.rho, rinv = 1.0 / rho;
    const float rinvf = (float)rinv;
    float mre[NP + 1], mim[NP + 1];
    double I[FMM_PMAX + 2];
#pragma unroll
    for (int n = 0; n <= NP; ++n) mre[n] = mim[n] = 0.0f;
    for (int t = t0; t < t1; ++t) {
        const int P = leaf_part[t];
        for (int l = lane; l < G.npp; l += 32) {
            const int64_t j = (int64_t)P * G.npp + l;
            const double ex = G.x[j] - cx, ey = G.y[j] - cy;
            const double s = sqrt(ex * ex + ey * ey);
            const float ws = (float)(G.w[j] * sigma[j]);
            const float nx = (float)G.nx[j], ny = (float)G.ny[j];
            if (s < 1e-8 * rho) {
                // at the centre only n = 1 survives: grad[I_1(s/rho) e^{-i phi}] = (1, -i)/(2 rho)
                mre[1] += ws * nx * 0.5f * rinvf;
                mim[1] -= ws * ny * 0.5f * rinvf;
                continue;
            }
            const double sinv = 1.0 / s;
            const float esx = (float)(ex * sinv), esy = (float)(ey * sinv);
            const float a_s = nx * esx + ny * esy;             // nu . e_s
            const float a_p = -nx * esy + ny * esx;            // nu . e_phi
            const float sinvf = (float)sinv;
            float If[NP + 2];
            if (PF > 0 && s * rinv >= (double)BESSEL_I_F32_XMIN) {
                if constexpr (PF > 0) bessel_i_down_f<PF + 1>((float)(s * rinv), If);
            } else {
                bessel_i_down(p + 1, s * rinv, I);
#pragma unroll
                for (int n = 0; n <= NP + 1; ++n) If[n] = (n <= p + 1) ? (float)I[n] : 0.0f;
            }
            float cn = 1.0f, sn = 0.0f;                        // e^{i n phi}
            float Iprev = If[1], Icur = If[0];                 // I_{n-1} (I_1 at n = 0), I_n
#pragma unroll
            for (int n = 0; n <= NP; ++n) {
                if (PF == 0 && n > p) break;
                const float Inext = If[n + 1];
                const float ip = (n == 0) ? Inext : 0.5f * (Iprev + Inext);
                const float ar = a_s * ip * rinvf;
                const float ai = -(float)n * a_p * Icur * sinvf;
                mre[n] = fmaf(ws, cn * ar + sn * ai, mre[n]);   // e^{-i n phi} (ar + i ai)
                mim[n] = fmaf(ws, cn * ai - sn * ar, mim[n]);
                const float c2 = cn * esx - sn * esy;
                sn = sn * esx + cn * esy;
                cn = c2;
                Iprev = Icur;
                Icur = Inext;
            }
        }
    }
#pragma unroll
    for (int n = 0; n <= NP; ++n) {
        if (PF == 0 && n > p) break;
        float a = mre[n], c = mim[n];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) M[(int64_t)leaf * (p + 1) + n] = make_double2((double)a, (double)c);
    }
}

// I_d(x) for d = 0..2p into a warp's shared slice (series per order).
__device__ __forceinline__ void warp_bessel_table(int p, double x, double* Iv, int lane) {
    for (int d = 2 * lane + 1; d <= 2 * p + 1; d += 64) {
        double a, b;
        bessel_i_pair(d, x, a, b);
        if (d <= 2 * p) Iv[d] = a;
        Iv[d - 1] = b;
    }
    __syncwarp();
}

// M2M: parents at level l (slice Mp, counts cnt_p) from children (Mc, cnt_c).
__global__ void __launch_bounds__(128) k_fmm_m2m(int l, int p, double rho, double bc,
                                                 const int* __restrict__ cnt_c,
                                                 const double2* __restrict__ Mc,
                                                 const int* __restrict__ cnt_p,
                                                 double2* __restrict__ Mp) {
    __shared__ double Ish[4][2 * FMM_PMAX + 1];
    const int nl = 1 << l;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (k >= nl * nl || cnt_p[k] == 0) return;            // warp-uniform
    double* Iv = Ish[wib];
    warp_bessel_table(p, bc * M_SQRT1_2 / rho, Iv, lane); // |t| = bc / sqrt 2
    const int i = k % nl, j = k / nl, nc = 2 * nl;
    double ar = 0.0, ai = 0.0;
    for (int q = 0; q < 4; ++q) {
        const int qx = q & 1, qy = q >> 1;
        const int c = (2 * j + qy) * nc + 2 * i + qx;
        if (cnt_c[c] == 0) continue;
        const int kq = quadrant_angle(qx, qy);                 // arg t = kq pi/4
        const double2 mine = (lane <= p) ? Mc[(int64_t)c * (p + 1) + lane] : make_double2(0.0, 0.0);
        for (int n = 0; n <= p; ++n) {
            const double2 Mn = shfl2(mine, n);
            if (lane > p) continue;
            // +n: M_n I_{|k-n|} e^{-i (k-n) th}
            {
                const int d = lane - n;
                const double2 w = w8(d * kq);
                const double cd = w.x, sd = w.y;
                const double Iq = Iv[d < 0 ? -d : d];
                ar += Iq * (Mn.x * cd + Mn.y * sd);
                ai += Iq * (Mn.y * cd - Mn.x * sd);
            }
            // -n: conj(M_n) I_{k+n} e^{-i (k+n) th}
            if (n > 0) {
                const int d = lane + n;
                const double2 w = w8(d * kq);
                const double cd = w.x, sd = w.y;
                const double Iq = Iv[d];
                ar += Iq * (Mn.x * cd - Mn.y * sd);
                ai += Iq * (-Mn.y * cd - Mn.x * sd);
            }
        }
    }
    if (lane <= p) Mp[(int64_t)k * (p + 1) + lane] = make_double2(ar, ai);
}

// M2L translation table of one level: for a source box at offset (ox, oy)
// boxes from the target (D = -(ox, oy) b_l), K_|k|(|D|/rho) e^{i k arg D} for
// k = -p..2p. Offsets span [-W, W]^2 with W = 2 FMM_SEP + 1.
constexpr int FMM_W = 2 * FMM_SEP + 1;
constexpr int FMM_NOFF = (2 * FMM_W + 1) * (2 * FMM_W + 1);

__global__ void k_fmm_m2l_table(int p, double rho, double bl, double2* __restrict__ T,
                                float2* __restrict__ T32) {
    __shared__ double Kv[2 * FMM_PMAX + 1];
    const int o = blockIdx.x;
    const int ox = o % (2 * FMM_W + 1) - FMM_W, oy = o / (2 * FMM_W + 1) - FMM_W;
    double2* To = T + (int64_t)o * (3 * p + 1);
    float2* To32 = T32 + (int64_t)o * (3 * p + 1);
    if (max(abs(ox), abs(oy)) <= FMM_SEP) {
        for (int k = threadIdx.x; k <= 3 * p; k += blockDim.x) {
            To[k] = make_double2(0.0, 0.0);
            To32[k] = make_float2(0.0f, 0.0f);
        }
        return;
    }
    const double Dx = -ox * bl, Dy = -oy * bl;
    const double z = sqrt(Dx * Dx + Dy * Dy) / rho;
    const double psi = atan2(Dy, Dx);
    if (threadIdx.x == 0) {
        double a, c;
        k01(z, a, c);
        Kv[0] = a;
        Kv[1] = c;
        for (int n = 1; n < 2 * p; ++n) Kv[n + 1] = Kv[n - 1] + (2.0 * n / z) * Kv[n];
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= 3 * p; t += blockDim.x) {
        const int kk = t - p;
        double s_, c_;
        sincos(kk * psi, &s_, &c_);
        const double K = Kv[kk < 0 ? -kk : kk];
        To[t] = make_double2(K * c_, K * s_);
        To32[t] = make_float2((float)(K * c_), (float)(K * s_));
    }
}

// M2L in FP32 (a level whose translation table fits the FP32 range): the
// same sums as k_fmm_m2l with the moments and the table rounded to FP32, the
// sum over each source box in FP32 and over the interaction list in FP64.
__global__ void __launch_bounds__(128) k_fmm_m2l_f32(int l, int p, double bl, double a2,
                                                     double gcut, const int* __restrict__ cnt,
                                                     const double2* __restrict__ M,
                                                     const float2* __restrict__ T,
                                                     double2* __restrict__ Lc) {
    const int nl = 1 << l;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nl * nl || cnt[k] == 0) return;               // warp-uniform
    const int i = k % nl, j = k / nl, pi = i >> 1, pj = j >> 1;
    const int m = lane;
    const bool act = m <= p;
    double lr = 0.0, li = 0.0;
    for (int sj = max(2 * (pj - FMM_SEP), 0); sj <= min(2 * (pj + FMM_SEP) + 1, nl - 1); ++sj)
        for (int si = max(2 * (pi - FMM_SEP), 0); si <= min(2 * (pi + FMM_SEP) + 1, nl - 1);
             ++si) {
            const int ox = si - i, oy = sj - j;
            if (max(abs(ox), abs(oy)) <= FMM_SEP) continue;
            const int s = sj * nl + si;
            if (cnt[s] == 0) continue;
            if (bl * sqrt((double)(ox * ox + oy * oy)) - a2 > gcut) continue;
            const float2* Tt =
                T + (int64_t)((oy + FMM_W) * (2 * FMM_W + 1) + (ox + FMM_W)) * (3 * p + 1) + p;
            const double2 md = act ? M[(int64_t)s * (p + 1) + lane] : make_double2(0.0, 0.0);
            const float mx0 = (float)md.x, my0 = (float)md.y;
            float ar = 0.0f, ai = 0.0f;
            for (int n = 0; n <= p; ++n) {
                const float mx = __shfl_sync(0xffffffffu, mx0, n);
                const float my = __shfl_sync(0xffffffffu, my0, n);
                if (!act) continue;
                const float2 t1 = Tt[n + m];                       // M_n T[n+m]
                ar = fmaf(mx, t1.x, fmaf(-my, t1.y, ar));
                ai = fmaf(mx, t1.y, fmaf(my, t1.x, ai));
                if (n > 0) {
                    const float2 t2 = Tt[m - n];                   // conj(M_n) T[m-n]
                    ar = fmaf(mx, t2.x, fmaf(my, t2.y, ar));
                    ai = fmaf(mx, t2.y, fmaf(-my, t2.x, ai));
                }
            }
            lr += (double)ar;
            li += (double)ai;
        }
    if (act) {
        const double sg = (m & 1) ? -1.0 : 1.0;
        double2& L = Lc[(int64_t)k * (p + 1) + m];
        L.x += sg * lr;
        L.y += sg * li;
    }
}

// M2L into the target boxes of level l (slices cnt, M, Lc of that level):
// L_m += (-1)^m sum over the interaction list sum_n M_n T[n + m].
// a2 = 2 a_l; pairs whose discs are more than gcut apart are left out.
__global__ void __launch_bounds__(128) k_fmm_m2l(int l, int p, double bl, double a2, double gcut,
                                                 const int* __restrict__ cnt,
                                                 const double2* __restrict__ M,
                                                 const double2* __restrict__ T,
                                                 double2* __restrict__ Lc) {
    const int nl = 1 << l;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nl * nl || cnt[k] == 0) return;               // warp-uniform
    const int i = k % nl, j = k / nl, pi = i >> 1, pj = j >> 1;
    const int m = lane;
    double lr = 0.0, li = 0.0;
    for (int sj = max(2 * (pj - FMM_SEP), 0); sj <= min(2 * (pj + FMM_SEP) + 1, nl - 1); ++sj)
        for (int si = max(2 * (pi - FMM_SEP), 0); si <= min(2 * (pi + FMM_SEP) + 1, nl - 1);
             ++si) {
            const int ox = si - i, oy = sj - j;
            if (max(abs(ox), abs(oy)) <= FMM_SEP) continue;
            const int s = sj * nl + si;
            if (cnt[s] == 0) continue;
            if (bl * sqrt((double)(ox * ox + oy * oy)) - a2 > gcut) continue;
            const double2* Tt =
                T + (int64_t)((oy + FMM_W) * (2 * FMM_W + 1) + (ox + FMM_W)) * (3 * p + 1);
            const double2 mine =
                (lane <= p) ? M[(int64_t)s * (p + 1) + lane] : make_double2(0.0, 0.0);
            for (int n = 0; n <= p; ++n) {
                const double2 Mn = shfl2(mine, n);
                if (m > p) continue;
                const double2 t1 = Tt[n + m + p];                  // M_n T[n+m]
                lr += Mn.x * t1.x - Mn.y * t1.y;
                li += Mn.x * t1.y + Mn.y * t1.x;
                if (n > 0) {
                    const double2 t2 = Tt[m - n + p];              // conj(M_n) T[m-n]
                    lr += Mn.x * t2.x + Mn.y * t2.y;
                    li += Mn.x * t2.y - Mn.y * t2.x;
                }
            }
        }
    if (m <= p) {
        const double sg = (m & 1) ? -1.0 : 1.0;
        double2& L = Lc[(int64_t)k * (p + 1) + m];
        L.x += sg * lr;
        L.y += sg * li;
    }
}

// L2L from level lc - 1 (slice Lp) into the boxes of level lc (slices cnt_c, Lc).
__global__ void __launch_bounds__(128) k_fmm_l2l(int lc, int p, double rho, double bc,
                                                 const int* __restrict__ cnt_c,
                                                 const double2* __restrict__ Lp,
                                                 double2* __restrict__ Lc) {
    __shared__ double Ish[4][2 * FMM_PMAX + 1];
    const int nc = 1 << lc;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (k >= nc * nc || cnt_c[k] == 0) return;             // warp-uniform
    double* Iv = Ish[wib];
    warp_bessel_table(p, bc * M_SQRT1_2 / rho, Iv, lane);  // |s| = bc / sqrt 2
    const int i = k % nc, j = k / nc;
    const int pk = (j >> 1) * (nc >> 1) + (i >> 1);
    const int kq = quadrant_angle(i & 1, j & 1);               // arg s = kq pi/4
    const double2 mine = (lane <= p) ? Lp[(int64_t)pk * (p + 1) + lane] : make_double2(0.0, 0.0);
    const int jj = lane;
    double ar = 0.0, ai = 0.0;
    for (int m = 0; m <= p; ++m) {
        const double2 Lm = shfl2(mine, m);
        if (jj > p) continue;
        {   // +m: L_m I_{|m-j|} e^{-i (m-j) th}
            const int d = m - jj;
            const double2 w = w8(d * kq);
            const double cd = w.x, sd = w.y;
            const double Iq = Iv[d < 0 ? -d : d];
            ar += Iq * (Lm.x * cd + Lm.y * sd);
            ai += Iq * (Lm.y * cd - Lm.x * sd);
        }
        if (m > 0) {   // -m: conj(L_m) I_{m+j} e^{i (m+j) th}
            const int d = m + jj;
            const double2 w = w8(d * kq);
            const double cd = w.x, sd = w.y;
            const double Iq = Iv[d];
            ar += Iq * (Lm.x * cd + Lm.y * sd);
            ai += Iq * (Lm.x * sd - Lm.y * cd);
        }
    }
    if (jj <= p) {
        double2& L = Lc[(int64_t)k * (p + 1) + jj];
        L.x += ar;
        L.y += ai;
    }
}

// L2P: value of the leaf's local expansion at every node (written to out),
// summed in R (FP32 when every level's coefficients fit its range); I_m
// from the FP64 series and recurrence, or, with a fixed order PF and R =
// float, from the FP32 series wherever r/rho >= BESSEL_I_F32_XMIN.
template <typename R, int PF>
__global__ void __launch_bounds__(128) k_fmm_l2p(GeomView G, int p_rt, int nb, double x0, double y0,
                                                 double b, const int* __restrict__ leaf_of,
                                                 const double2* __restrict__ Lleaf,
                                                 double* __restrict__ out) {
    constexpr int NP = PF > 0 ? PF : FMM_PMAX;
    const int p = PF > 0 ? PF : p_rt;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= G.n) return;
    const int leaf = leaf_of[i / G.npp];
    const double2* L = Lleaf + (int64_t)leaf * (p + 1);
    const double vx = G.x[i] - (x0 + (leaf % nb + 0.5) * b);
    const double vy = G.y[i] - (y0 + (leaf / nb + 0.5) * b);
    const double r = sqrt(vx * vx + vy * vy);
    if (r < 1e-8 * G.rho) {                                 // I_m(0) = delta_m0
        out[i] = L[0].x / (2.0 * PI);
        return;
    }
    R Ir[NP + 2];
    const double x = r / G.rho;
    if (PF > 0 && sizeof(R) == sizeof(float) && x >= (double)BESSEL_I_F32_XMIN) {
        if constexpr (PF > 0) {
            float If[PF + 2];
            bessel_i_down_f<PF + 1>((float)x, If);
#pragma unroll
            for (int n = 0; n <= PF + 1; ++n) Ir[n] = (R)If[n];
        }
    } else {
        double I[FMM_PMAX + 2];
        bessel_i_down(p + 1, x, I);
#pragma unroll
        for (int n = 0; n <= NP + 1; ++n) Ir[n] = (n <= p + 1) ? (R)I[n] : (R)0;
    }
    const double rinv = 1.0 / r;
    const R erx = (R)(vx * rinv), ery = (R)(vy * rinv);
    R acc = (R)L[0].x * Ir[0];
    R cm = erx, sm = ery;                                   // (cos, sin)(m theta), m = 1
#pragma unroll
    for (int m = 1; m <= NP; ++m) {
        if (PF == 0 && m > p) break;
        const double2 Lm = L[m];
        // 2 Re[L_m e^{-i m theta}] I_m
        acc = fma((R)2 * Ir[m], (R)Lm.x * cm + (R)Lm.y * sm, acc);
        const R c2 = cm * erx - sm * ery;
        sm = sm * erx + cm * ery;
        cm = c2;
    }
    out[i] = (double)acc / (2.0 * PI);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void fmm_root_box(yk_geom* g, double* x0, double* y0, double* side) {
    double xmin = INFINITY, ymin = INFINITY, xmax = -INFINITY, ymax = -INFINITY;
    for (const yk_particle& P : g->parts) {
        xmin = std::min(xmin, P.cx);
        xmax = std::max(xmax, P.cx);
        ymin = std::min(ymin, P.cy);
        ymax = std::max(ymax, P.cy);
    }
    const double ext = std::max(std::max(xmax - xmin, ymax - ymin), 1e-6 * (1.0 + g->max_radius));
    *side = ext * (1.0 + 1e-9);
    *x0 = xmin - 0.5 * (*side - (xmax - xmin));
    *y0 = ymin - 0.5 * (*side - (ymax - ymin));
}

// Leaf levels the autotuner may try: 2 a_L / (3 b_L) <= 0.7 (b_L >= 2R / (2.1 - sqrt 2)),
// a_L / rho <= 3p/4, at most 64 leaves per particle, at most three levels (the
// finest admissible ones). Returns YK_OK with *lo > *hi when none is admissible.
int fmm_candidates(yk_geom* g, int* lo, int* hi) {
    double x0, y0, side;
    fmm_root_box(g, &x0, &y0, &side);
    const double R = g->max_radius, rho = g->prm.rho;
    const int p = g->prm.fmm_order;
    const double b_lo = 2.0 * R / (2.1 - M_SQRT2);
    const double b_hi = M_SQRT2 * (0.75 * p * rho - R);
    *lo = 1;
    *hi = 0;
    for (int L = 0; L <= FMM_LMAX; ++L) {
        const double b = side / (double)(1 << L);
        if ((int64_t(1) << (2 * L)) > 64 * (int64_t)g->np + 64) break;
        if (b >= b_lo && b <= b_hi) {
            if (*lo > *hi) *lo = L;
            *hi = L;
        }
    }
    if (*lo <= *hi) *lo = std::max(*lo, *hi - 2);
    return YK_OK;
}

static int grow(void** ptr, int64_t* cap, int64_t need, size_t elem, cudaStream_t st) {
    if (need <= *cap && *ptr) return YK_OK;
    dev_free(*ptr, st);
    *ptr = nullptr;
    *cap = 0;
    YK_TRY(dev_alloc(ptr, elem * (size_t)std::max<int64_t>(need, 1), st));
    *cap = need;
    return YK_OK;
}

int fmm_build(yk_geom* g, int L) {
    FmmTree& F = g->fmm;
    cudaStream_t st = g->ctx->stream;
    if (L < 0 || L > FMM_LMAX) return YK_ERR_ARG;
    g->sym[3].valid = false;   // the near lists change with the tree
    fmm_root_box(g, &F.x0, &F.y0, &F.side);
    F.L = L;
    F.p = g->prm.fmm_order;
    F.leaf = F.side / (double)(1 << L);
    const int p = F.p, np = g->np, nb = 1 << L, nleaf = nb * nb;
    F.nbox = level_offset(L + 1);
    if (!F.leaf_of) {
        YK_TRY(dev_alloc((void**)&F.leaf_of, sizeof(int) * np, st));
        YK_TRY(dev_alloc((void**)&F.leaf_part, sizeof(int) * np, st));
        YK_TRY(dev_alloc((void**)&F.near_off, sizeof(int) * (np + 1), st));
    }
    if (nleaf + 1 > F.leaf_cap || !F.leaf_off) {
        dev_free(F.leaf_off, st);
        dev_free(F.cursor, st);
        F.leaf_off = F.cursor = nullptr;
        F.leaf_cap = 0;
        YK_TRY(dev_alloc((void**)&F.leaf_off, sizeof(int) * (nleaf + 1), st));
        YK_TRY(dev_alloc((void**)&F.cursor, sizeof(int) * (nleaf + 1), st));
        F.leaf_cap = nleaf + 1;
    }
    YK_TRY(grow((void**)&F.box_count, &F.box_cap, F.nbox, sizeof(int), st));
    if (F.nbox * (p + 1) > F.coef_cap || !F.M) {
        dev_free(F.M, st);
        dev_free(F.Lc, st);
        F.M = F.Lc = nullptr;
        F.coef_cap = 0;
        YK_TRY(dev_alloc((void**)&F.M, sizeof(double2) * F.nbox * (p + 1), st));
        YK_TRY(dev_alloc((void**)&F.Lc, sizeof(double2) * F.nbox * (p + 1), st));
        F.coef_cap = F.nbox * (p + 1);
    }
    YK_TRY(grow((void**)&F.T, &F.t_cap, (int64_t)(L + 1) * FMM_NOFF * (3 * p + 1), sizeof(double2),
                st));
    YK_TRY(grow((void**)&F.T32, &F.t32_cap, (int64_t)(L + 1) * FMM_NOFF * (3 * p + 1),
                sizeof(float2), st));
    // particles by leaf
    YK_TRY_CUDA(cudaMemsetAsync(F.cursor, 0, sizeof(int) * (nleaf + 1), st));
    YK_LAUNCH(k_fmm_leaf_count, ceil_div(np, 128), 128, 0, st, np, g->d_part, F.x0, F.y0,
              1.0 / F.leaf, nb, F.leaf_of, F.cursor);
    YK_LAUNCH(k_scan_offsets, 1, 1024, 0, st, nleaf, F.cursor, F.leaf_off);
    YK_TRY_CUDA(cudaMemsetAsync(F.cursor, 0, sizeof(int) * (nleaf + 1), st));
    YK_LAUNCH(k_fmm_leaf_fill, ceil_div(np, 128), 128, 0, st, np, F.leaf_of, F.leaf_off, F.cursor,
              F.leaf_part);
    YK_LAUNCH(k_fmm_leaf_sort, ceil_div(nleaf, 128), 128, 0, st, nleaf, F.leaf_off, F.leaf_part);
    // box counts, leaves up to the root
    YK_LAUNCH(k_fmm_count_leaves, ceil_div(nleaf, 128), 128, 0, st, nleaf, F.leaf_off,
              F.box_count + level_offset(L));
    for (int l = L - 1; l >= 0; --l)
        YK_LAUNCH(k_fmm_count_up, ceil_div(1 << (2 * l), 128), 128, 0, st, l,
                  F.box_count + level_offset(l + 1), F.box_count + level_offset(l));
    // near lists
    YK_LAUNCH(k_fmm_near<false>, ceil_div(np, 128), 128, 0, st, np, nb, F.leaf_of, F.leaf_off,
              F.leaf_part, g->d_counts, (const int*)nullptr, (int*)nullptr);
    YK_LAUNCH(k_scan_offsets, 1, 1024, 0, st, np, g->d_counts, F.near_off);
    int total = 0;
    YK_TRY_CUDA(cudaMemcpyAsync(&total, F.near_off + np, sizeof(int), cudaMemcpyDeviceToHost, st));
    YK_TRY_CUDA(cudaStreamSynchronize(st));
    YK_TRY(grow((void**)&F.near, &F.near_cap, total, sizeof(int), st));
    YK_LAUNCH(k_fmm_near<true>, ceil_div(np, 128), 128, 0, st, np, nb, F.leaf_of, F.leaf_off,
              F.leaf_part, (int*)nullptr, F.near_off, F.near);
    // levels that can hold an interaction within the reach gcut: the closest
    // interacting pair of level l is (3 - sqrt 2) b_l - 2R apart
    const double rho = g->prm.rho, R = g->max_radius;
    F.gcut = std::min(g->fmm_gap, 60.0 * rho);
    F.lmin = L + 1;
    for (int l = 2; l <= L; ++l) {
        const double bl = F.side / (double)(1 << l);
        if ((3.0 - M_SQRT2) * bl - 2.0 * R <= F.gcut) {
            F.lmin = l;
            break;
        }
    }
    // FP32 translation at level l when its table fits the FP32 range: the
    // closest pair is 3 b_l apart, and K_nu(z) <= Gamma(nu) 2^{nu-1} z^{-nu}
    // bounds the largest entry K_{2p}(3 b_l / rho) below 1e30; the source and
    // target discs must also stay within a_l / rho <= 40 (I_0(40) ~ 1e16).
    F.all32 = true;
    for (int l = 0; l <= FMM_LMAX; ++l) F.use32[l] = false;
    for (int l = F.lmin; l <= L; ++l) {
        const double bl = F.side / (double)(1 << l);
        const double z = 3.0 * bl / rho, nu = 2.0 * p;
        const double logk = lgamma(nu) + nu * log(2.0 / z) - log(2.0);
        F.use32[l] = logk < log(1e30) && (bl * M_SQRT1_2 + R) / rho <= 40.0;
        F.all32 = F.all32 && F.use32[l];
        YK_LAUNCH(k_fmm_m2l_table, FMM_NOFF, 64, 0, st, p, rho, bl,
                  F.T + (int64_t)l * FMM_NOFF * (3 * p + 1),
                  F.T32 + (int64_t)l * FMM_NOFF * (3 * p + 1));
    }
    YK_TRY_CUDA(cudaGetLastError());
    F.valid = true;
    return YK_OK;
}

// Far field of the FP32 inner operator at every node (written to out): the
// particles outside each target's near list, by expansions.
int fmm_far(yk_geom* g, const double* sigma, double* out) {
    FmmTree& F = g->fmm;
    if (!F.valid) return YK_ERR_ARG;
    cudaStream_t st = g->ctx->stream;
    const int L = F.L, p = F.p, nb = 1 << L;
    const double rho = g->prm.rho, R = g->max_radius;
    if (F.lmin > L) {                       // every interaction is direct
        YK_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * g->n, st));
        return YK_OK;
    }
    GeomView G = g->view();
    const int64_t o0 = level_offset(F.lmin);
    YK_TRY_CUDA(cudaMemsetAsync(F.Lc + o0 * (p + 1), 0,
                                sizeof(double2) * (F.nbox - o0) * (p + 1), st));
    auto lvl = [&](int l) { return (int64_t)level_offset(l); };
    auto side = [&](int l) { return F.side / (double)(1 << l); };
    if (p == FMM_FIXED_ORDER)
        YK_LAUNCH(k_fmm_p2m<FMM_FIXED_ORDER>, ceil_div((int64_t)nb * nb * 32, 128), 128, 0, st, G,
                  sigma, p, nb, F.x0, F.y0, F.leaf, F.leaf_off, F.leaf_part, F.M + lvl(L) * (p + 1));
    else
        YK_LAUNCH(k_fmm_p2m<0>, ceil_div((int64_t)nb * nb * 32, 128), 128, 0, st, G, sigma, p, nb,
                  F.x0, F.y0, F.leaf, F.leaf_off, F.leaf_part, F.M + lvl(L) * (p + 1));
    for (int l = L - 1; l >= F.lmin; --l)
        YK_LAUNCH(k_fmm_m2m, ceil_div((int64_t(1) << (2 * l)) * 32, 128), 128, 0, st, l, p, rho,
                  side(l + 1), F.box_count + lvl(l + 1), F.M + lvl(l + 1) * (p + 1),
                  F.box_count + lvl(l), F.M + lvl(l) * (p + 1));
    for (int l = F.lmin; l <= L; ++l) {
        const double bl = side(l);
        const double a2 = 2.0 * (bl * M_SQRT1_2 + R);
        if (F.use32[l])
            YK_LAUNCH(k_fmm_m2l_f32, ceil_div((int64_t(1) << (2 * l)) * 32, 128), 128, 0, st, l, p,
                      bl, a2, F.gcut, F.box_count + lvl(l), F.M + lvl(l) * (p + 1),
                      F.T32 + (int64_t)l * FMM_NOFF * (3 * p + 1), F.Lc + lvl(l) * (p + 1));
        else
            YK_LAUNCH(k_fmm_m2l, ceil_div((int64_t(1) << (2 * l)) * 32, 128), 128, 0, st, l, p,
                      bl, a2, F.gcut, F.box_count + lvl(l), F.M + lvl(l) * (p + 1),
                      F.T + (int64_t)l * FMM_NOFF * (3 * p + 1), F.Lc + lvl(l) * (p + 1));
        if (l < L)
            YK_LAUNCH(k_fmm_l2l, ceil_div((int64_t(1) << (2 * (l + 1))) * 32, 128), 128, 0, st,
                      l + 1, p, rho, side(l + 1), F.box_count + lvl(l + 1),
                      F.Lc + lvl(l) * (p + 1), F.Lc + lvl(l + 1) * (p + 1));
    }
    auto l2p = F.all32 ? (p == FMM_FIXED_ORDER ? &k_fmm_l2p<float, FMM_FIXED_ORDER>
                                               : &k_fmm_l2p<float, 0>)
                       : &k_fmm_l2p<double, 0>;
    YK_LAUNCH(l2p, ceil_div(g->n, 128), 128, 0, st, G, p, nb, F.x0, F.y0, F.leaf, F.leaf_of,
              F.Lc + lvl(L) * (p + 1), out);
    YK_TRY_CUDA(cudaGetLastError());
    return YK_OK;
}

void fmm_free(yk_geom* g) {
    FmmTree& F = g->fmm;
    cudaStream_t st = g->ctx->stream;
    void* bufs[] = {F.leaf_of, F.leaf_part, F.near_off, F.near, F.leaf_off, F.cursor,
                    F.box_count, F.M, F.Lc, F.T, F.T32};
    for (void* b : bufs) dev_free(b, st);
    F = FmmTree{};
}

}  // namespace yk
