// Internal state of the yk library: contexts, geometries and workspaces.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <functional>
#include <set>
#include <vector>

#include "../../include/yk.h"
#include "geom_view.cuh"

#define YK_TRY_CUDA(expr)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) {                            \
            yk::set_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return YK_ERR_CUDA;                             \
        }                                                   \
    } while (0)

// Every kernel launch of the library goes through YK_LAUNCH so that the
// number of launches can be reported (yk_kernel_launches).
#define YK_LAUNCH(kernel, grid, block, smem, stream, ...)         \
    do {                                                         \
        ::yk::note_launch();                                     \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__); \
    } while (0)

#define YK_TRY(expr)                 \
    do {                             \
        int rc_ = (expr);            \
        if (rc_ != YK_OK) return rc_; \
    } while (0)

namespace yk {

void set_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void note_launch();

struct Workspace {
    double* partial = nullptr;   // [nchunk][n]
    int nchunk = 0;
    float4* src4 = nullptr;      // pair-packed FP32 source records [np][ceil(npp/2)][2]
    float4* src4g = nullptr;     // the same for the normal derivative [np][ceil(npp/2)][3]
    double* V = nullptr;         // Krylov basis [(m+1)][n]
    double* Zp = nullptr;        // preconditioned basis z_j = M^{-1} v_j [m][n] (on first use)
    double* H = nullptr;         // Hessenberg (m+1) x m, column-major
    double* gvec = nullptr;      // rotated rhs, m+1
    double* cs = nullptr;        // Givens cosines, m
    double* sn = nullptr;        // Givens sines, m
    double* hbuf = nullptr;      // 2 (m+2) dot products
    double* ybuf = nullptr;      // m+1 least-squares coefficients
    double* dotpart = nullptr;   // partial dots [(m+2)][nblk]
    double* status = nullptr;    // [0] residual estimate, [1] norm, [2..] scratch
    double* hist = nullptr;      // (residual estimate, norm) of every Arnoldi step, 2 (m+1)
    double* vec[8] = {};         // N-length scratch vectors
    int m = 0;
    int dot_blocks = 0;
};

// Per-target-particle source lists (CSR) for the expansion band.
struct BandList {
    int* off = nullptr;
    int* idx = nullptr;
    int n = 0;
    int cap = 0;
    bool valid = false;
};

// Particle pairs (P <= Q) evaluated by the FP64 tiles.
struct PairList {
    int2* d = nullptr;
    int n = 0;
    int cap = 0;
    bool valid = false;
};

}  // namespace yk

struct yk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    void* server = nullptr;  // serving state (serve.cu)
    std::set<yk_geom*> geoms;  // live geometries made from this context
    double* h_status = nullptr;  // pinned host mirror of solver status (8 doubles)
    double* h_batch = nullptr;   // pinned host buffer of batched solves' residuals
    size_t h_batch_cap = 0;      // its length in doubles
};

namespace yk {
// Uniform quadtree of the FMM far field (fmm.cu). Boxes of level l are
// numbered j * 2^l + i after those of the coarser levels
// (offset (4^l - 1) / 3); particles belong to the leaf holding their centre.
struct FmmTree {
    bool valid = false;        // built for the current particle positions
    bool tuned = false;        // leaf size chosen (autotuned or given)
    bool far_off = false;      // no admissible leaf size: far field by cut-off P2P
    int L = -1;                // leaf level
    int Lsel = -1;             // leaf level chosen for these particles
    int lmin = 2;              // coarsest level with interactions
    int p = 12;                // expansion order (terms |n| <= p)
    double x0 = 0.0, y0 = 0.0, side = 0.0;   // root box
    double leaf = 0.0;         // chosen leaf side
    double gcut = 0.0;         // interactions across larger gaps are left out
    int64_t nbox = 0;
    int* leaf_of = nullptr;    // [np] leaf of each particle
    int* leaf_part = nullptr;  // [np] particles by leaf (CSR with leaf_off)
    int* near_off = nullptr;   // [np + 1] near lists (CSR)
    int* near = nullptr;       // particles in leaves within FMM_SEP boxes
    int64_t near_cap = 0;
    int* leaf_off = nullptr;   // [nleaf + 1]
    int* cursor = nullptr;     // [nleaf] scratch
    int64_t leaf_cap = 0;
    int* box_count = nullptr;  // [nbox] particles per box
    double2* M = nullptr;      // [nbox][p + 1] multipole moments
    double2* Lc = nullptr;     // [nbox][p + 1] local coefficients
    int64_t box_cap = 0;       // capacity of box_count (boxes)
    int64_t coef_cap = 0;      // capacity of M and Lc (coefficients)
    double2* T = nullptr;      // M2L tables [level][offset][3p + 1]
    int64_t t_cap = 0;
    float2* T32 = nullptr;     // the same rounded to FP32
    int64_t t32_cap = 0;
    bool use32[11] = {};       // level translates in FP32 (table within FP32 range)
    bool all32 = false;        // every active level does (L2P in FP32)
};
}  // namespace yk

namespace yk {
// Near-contact lists (contact.cu): for every boundary node, the panels of
// other particles close enough to need oversampled quadrature (CSR).
struct Contact {
    bool valid = false;
    int ntgt = 0;                  // nodes with at least one entry
    int* partners = nullptr;       // [np][CONTACT_MAX_PARTNERS] particles within reach
    int* npartners = nullptr;      // [np]
    int* off = nullptr;            // [n + 1] entries of node i: ent[off[i] .. off[i+1])
    int* tgt = nullptr;            // [n] nodes with entries
    int* flag = nullptr;           // [2] overflow flag, node counter
    int2* ent = nullptr;           // (particle, panel)
    int64_t cap = 0;
};

// Device state of the particle dynamics (dynamics.cu).
struct Dynamics {
    yk_particle* parts = nullptr;  // [np] device copy of the particles
    double* sigma = nullptr;       // [n] density of the last step (warm start)
    double* f = nullptr;           // [n] Dirichlet data
    double* un = nullptr;          // [n] normal derivative
    double* work = nullptr;        // forces, torques, repulsion, energies
    int* bad = nullptr;            // overlap flag of the repulsion
    bool have_sigma = false;
};
}  // namespace yk

namespace yk {
// A far particle pair of the Stokes far field (stokes.cu).
struct StokesFar {
    double2 z0;      // c_P - c_Q
    double2 zi;      // 1 / z0
    double logd;     // log |z0|
    int q;           // source particle
    short p64, p32;  // expansion orders for 1e-17 (FP64) and 1e-8 (FP32)
};

// Stokes mobility state (stokes.cu), built on the first Stokes call.
struct Stokes {
    bool ready = false;
    double* B0 = nullptr;       // per shape, body frame: 1/2 I + K* of the own particle
    double* Bw = nullptr;       //   the same plus the rigid-motion projector W
    float* Bw32 = nullptr;      //   Bw rounded to FP32 (inner operator)
    double* S = nullptr;        //   on-surface single layer; all [shape][col][row], 2 npp square
    double* moments = nullptr;  // log moments [3][ngl][ngl]
    double* shapeLJ = nullptr;  // per shape: perimeter, int |y - a|^2 ds
    double* LJ = nullptr;       // the same per particle
    double4* s64 = nullptr;     // FP64 source records (x, y, w sigma)
    float4* s32 = nullptr;      // FP32 source records (offset from the centre, w sigma)
    double *sinc = nullptr, *mu = nullptr, *rhs = nullptr, *tmp = nullptr, *u = nullptr;  // 2n
    double* vo = nullptr;       // 3 np scratch
    double2* coef64 = nullptr;  // particle multipoles [np][3][41], FP64
    double2* loc64 = nullptr;   // local expansions [np][4][41], FP64
    float2* coef32 = nullptr;   // the same in FP32 (inner operator)
    float2* loc32 = nullptr;
    int* lmax64 = nullptr;      // [np] highest local order used (0: no far pair)
    int* lmax32 = nullptr;
    bool lists_valid = false;   // pair lists for the current positions
    int* near_off = nullptr;    // [np + 1] near partners (CSR)
    int* near_idx = nullptr;
    int near_cap = 0;
    int* far_off = nullptr;     // [np + 1] far pairs (CSR)
    StokesFar* far = nullptr;
    int far_cap = 0;
    Workspace ws;               // Krylov workspace on vectors of 2n
};
}  // namespace yk

namespace yk {
// Coarse space of the inner GMRES (coarse.cu): three density modes per
// particle, B Z per coupled particle pair and (Z^T B Z)^{-1}.
struct Coarse {
    bool valid = false;         // built (or found unusable) for the current positions
    bool on = false;            // deflation in use for these positions
    int nc = 0;                 // 3 np
    int* off = nullptr;         // [np + 1] coupled source particles of each target (CSR)
    int2* ent = nullptr;        // (target, source) of every entry, in CSR order
    int cap = 0;
    double* Z = nullptr;        // [3][n] modes, orthonormal over each particle's nodes
    double* Y = nullptr;        // [3][n] M Z (M: the FP32 block preconditioner)
    double* O = nullptr;        // [3][n] own-particle part of A M Z
    float* W = nullptr;         // [entry][3][npp] B Z on the target's nodes
    size_t wcap = 0;            // floats
    float* C = nullptr;         // [nc][nc] Z^T B Z, then its inverse
    float* piv = nullptr;       // Gauss-Jordan panel: D^{-1}, M_:K copy, D^{-1} M_K:
    double* U = nullptr;        // [m][nc] Z^T (B v_j - v_j) of the Arnoldi steps
    double* cv = nullptr;       // [2][nc] scratch
    int* flag = nullptr;        // [1] failed pivot
};
}  // namespace yk

struct yk_geom {
    yk_ctx* ctx = nullptr;
    yk_params prm{};
    int np = 0, npan = 0, ngl = 0, npp = 0, n_near = 0, nshape = 0;
    int64_t n = 0;
    std::vector<yk_particle> parts;
    std::vector<int> shape_of_h;           // host copy of shape indices
    std::vector<double2> shape_ab;         // (A, B) of each shape
    double max_perimeter = 0.0, max_radius = 0.0;
    double split_gap = 0.0;                // gap above which FP32 is used (mixed residual)
    double split_gap_grad = 0.0;           // the same for the normal derivative
    double cutoff_gap = INFINITY;          // far field: source particles beyond are left out
    double fmm_gap = INFINITY;             // reach of the FMM far field (inner operator)
    double tile_gap = 0.0;                 // split operators: FP64 tiles below this gap,
    double tile_gap_grad = 0.0;            //   FP64 expansions up to the split gap
    yk::BandList bands[2];                 // expansion bands (value, normal derivative)
    int* d_counts = nullptr;               // np ints of scratch for list building
    double2* d_mpole = nullptr;            // multipole moments [np][order + 1]
    double2* d_local = nullptr;            // local coefficients [np][order + 1]
    int* nbr_off = nullptr;                // cut-off neighbour lists (CSR offsets, np + 1)
    int* nbr = nullptr;                    // neighbour particle indices
    int nbr_cap = 0;
    bool nbr_valid = false;
    yk::FmmTree fmm;                       // FMM far field (YK_FARFIELD_FMM)
    yk::Dynamics dyn;                      // particle dynamics (yk_step)
    yk::Stokes stokes;                     // Stokes mobility (yk_mobility)
    yk::Contact contact;                   // near-contact lists
    yk::Coarse coarse;                     // coarse space of the inner GMRES
    yk_particle* d_particles = nullptr;    // device copy of the particles
    // device allocations
    yk::d4* d_part = nullptr;
    float4* d_c32 = nullptr;
    float* d_r32 = nullptr;
    int* d_counter = nullptr;
    yk::PairList lists[4];                 // residual split, gradient split, all, cut-off
    yk::PairList sym[7];                   // symmetric FP32 far field: inner operator, split,
                                           //   normal-derivative split, FMM near field,
                                           //   cut-off: value split, derivative split, all
    int* d_shape_of = nullptr;
    double2* d_shape_ab = nullptr;
    double* d_x = nullptr;
    double* d_y = nullptr;
    double* d_nx = nullptr;
    double* d_ny = nullptr;
    double* d_w = nullptr;
    double* d_speed = nullptr;
    float2* d_xi = nullptr;
    double* d_cval = nullptr;
    double* d_cgrad = nullptr;
    double* d_glx = nullptr;      // GL nodes [ngl]
    double* d_glw = nullptr;      // GL weights [ngl]
    double* d_interp = nullptr;   // Lagrange interpolation [os*ngl][ngl]
    double* d_diff = nullptr;     // Lagrange differentiation [ngl][ngl]
    double* d_fine_x = nullptr;   // fine reference nodes [os*ngl]
    double* d_fine_w = nullptr;   // fine reference weights [os*ngl]
    double* d_minv = nullptr;     // block preconditioner: inverse self block per shape,
                                  // transposed, [shape][col j][row i]
    float* d_minv32 = nullptr;    // the same in FP32
    bool use_self = false;        // own-particle far pairs by the blocks below
    double* d_self = nullptr;     // far part of the self block per shape (value),
                                  // transposed, [shape][col j][row i]
    double* d_self_grad = nullptr;  // the same for the normal derivative
    float* d_self32 = nullptr;    // d_self rounded to FP32 (inner operator)
    yk::Workspace ws;
    yk::GeomView view() const;
};

namespace yk {

// geometry.cu
int build_geometry(yk_geom* g);
int update_nodes(yk_geom* g);
int launch_label(yk_geom* g, int kind, double param, double* f);
int build_preconditioner(yk_geom* g);
int apply_preconditioner(yk_geom* g, const double* x, double* y, bool fp32);

// p2p.cu
enum class Prec { F64 = 0, F32 = 1, SPLIT = 2 };
int matvec(yk_geom* g, const double* sigma, double* y, Prec prec);
// launch shape of the symmetric FP32 far field (kind 0: inner operator)
struct SymParams {
    const int2* tasks = nullptr;
    int ntasks = 0, qch = 0, ipb = 1, blocks = 0;
    int nw = 4;            // warps holding a chunk of P's nodes (64 per warp)
    double kscale = 0.0;
};
int sym_params(yk_geom* g, int kind, SymParams* p);
int own_apply_f32(yk_geom* g, const double* x, double* y);   // own-particle part, FP32 operator
int normal_derivative(yk_geom* g, const double* sigma, double* un, Prec prec);
int potential(yk_geom* g, const double* sigma, const double* targets, int64_t nt, double* u);
// near.cu
int potential_near(yk_geom* g, const double* sigma, const double* targets, int64_t nt,
                   double* u);
int potential_noalloc(yk_geom* g, const double* sigma, const double* targets, int64_t nt,
                      double* u);

// expansions.cu
constexpr int EXPANSION_TERMS = 41;        // orders 0..40 of the particle expansions
constexpr double EXPANSION_GAP_RADII = 2.0;  // band starts at a gap of 2 bounding radii
int band_expansions(yk_geom* g, const double* sigma, double* out, bool grad);

// fmm.cu
constexpr int FMM_PMAX = 30;      // largest expansion order (one warp lane per order)
constexpr int FMM_FIXED_ORDER = 12;   // the default order, with register-resident P2M/L2P
constexpr int FMM_SEP = 2;        // near field: leaves at most FMM_SEP boxes apart
constexpr int FMM_LMAX = 10;      // deepest leaf level
constexpr double FMM_REACH_TOL = 1e-10;   // FMM interactions bounded below this x max|sigma| are left out
void fmm_root_box(yk_geom* g, double* x0, double* y0, double* side);
int fmm_candidates(yk_geom* g, int* lo, int* hi);
int fmm_build(yk_geom* g, int L);
int fmm_far(yk_geom* g, const double* sigma, double* out);
void fmm_free(yk_geom* g);

// gmres.cu
// A linear operator for the device GMRES: y = A(prec) x on vectors of length
// n, an optional right preconditioner, and the workspace (Krylov basis and
// scratch vectors of length n) it runs in.
struct KrylovOp {
    yk_ctx* ctx = nullptr;
    Workspace* ws = nullptr;
    int64_t n = 0;
    std::function<int(const double*, double*, Prec)> apply;
    std::function<int(const double*, double*, bool)> precond;   // empty: none
    // Optional deflation of the FP32 inner solve (with precond): deflate(v_j,
    // w, j) turns w = A M v_j into the deflated operator's column, and
    // deflate_end(k, y, x) adds the coarse term of the cycle's correction
    // (k basis vectors) to x.
    std::function<int(const double*, double*, int)> deflate;
    std::function<int(int, const double*, double*)> deflate_end;
};
int solve_op(const KrylovOp& op, const yk_params& P, Prec residual, const double* f,
             double* sigma, const double* sigma0, yk_solve_info* info);
int solve(yk_geom* g, const double* f, double* sigma, const double* sigma0, yk_solve_info* info);
double inner_tolerance(const yk_params& P, double rel);
double device_norm2(yk_geom* g, const double* v);
// batch.cu
int solve_batch(yk_geom* const* g, int count, const double* const* f, double* const* sigma,
                yk_solve_info* info);
int alloc_workspace(yk_geom* g);
int alloc_krylov(Workspace& w, int64_t n, int m, cudaStream_t st);
void free_workspace(yk_geom* g);
void free_workspace(Workspace& w, cudaStream_t st);

// coarse.cu
constexpr int COARSE_MAX_PARTICLES = 2048;
constexpr double COARSE_TOL = 1e-9;   // couplings bounded below this x max|sigma| are left out
constexpr size_t COARSE_MAX_W_FLOATS = (size_t)1 << 29;   // 2 GiB of stored couplings at most
int coarse_prepare(yk_geom* g);
size_t coarse_bytes(const yk_particle* parts, int np, const yk_params& P);   // device memory
int coarse_deflate(yk_geom* g, const double* v, double* w, int j);
int coarse_correct(yk_geom* g, int k, const double* y, double* t);
void coarse_free(yk_geom* g);

// forces.cu
int forces_torques(yk_geom* g, const double* sigma, const double* f, const double* un,
                   double* F, double* tau, double* net);
int energy(yk_geom* g, const double* f, const double* un, double* phi, double* total);

// contact.cu
constexpr int CONTACT_MAX_PARTNERS = 16;   // particles within reach of one particle
int contact_apply(yk_geom* g, const double* sigma, double* y, bool grad);
int contact_targets(yk_geom* g, int* ntgt);   // nodes with near-contact entries
void contact_free(yk_geom* g);

// dynamics.cu
int repulsion(yk_geom* g, const yk_particle* d_parts, double c0, int q, double* F, double* tau,
              double* phi);
int repulsion_host(yk_geom* g, double c0, int q, double* F, double* tau, double* phi);
int step(yk_geom* g, const yk_dynamics& d, yk_solve_info* info, double* energy_out);
void dyn_free(yk_geom* g);

// stokes.cu
constexpr int STOKES_TRACTION = YK_STOKES_TRACTION;
constexpr int STOKES_COMPLETED = YK_STOKES_COMPLETED;
constexpr int STOKES_VELOCITY = YK_STOKES_VELOCITY;
int stokes_apply(yk_geom* g, const double* sigma, double* out, Prec prec, int which);
int mobility(yk_geom* g, const double* F, const double* tau, double* v, double* omega,
             double* sigma_out, yk_solve_info* info);
void stokes_free(yk_geom* g);

// serve.cu
int destroy_server(yk_ctx* ctx);

// capi.cu helpers
double cutoff_gap(double rho, double perim, double tol);
bool is_device_ptr(const void* p);
// stream-ordered device allocations (no device-wide synchronisation)
int dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
double* host_status(yk_ctx* ctx);
void keep_pool_memory(int device);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace yk
