// Device-facing types of the yk kernels: the particle record, constants
// and the device view of a discretised configuration (GeomView).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace yk {

// 32-byte aligned quadruple of doubles (one vectorised load)
struct __align__(32) d4 {
    double x, y, z, w;
};
__host__ __device__ inline d4 make_d4(double x, double y, double z, double w) {
    return d4{x, y, z, w};
}

constexpr double PI = 3.14159265358979323846;
constexpr int MAX_NGL = 32;
constexpr int MAX_ORDER = 24;
constexpr int MAX_NEAR_PANELS = 9;      // (2 near_width + 1) <= 9
constexpr int MAX_OVERSAMPLE = 16;
constexpr int SELF_BLOCK_MAX_NODES = 2048;   // nodes per particle with precomputed self blocks

// Device-resident description of a discretised configuration. All arrays
// are device pointers owned by the yk_geom that holds this view.
struct GeomView {
    int np;          // particles
    int npan;        // panels per particle
    int ngl;         // Gauss-Legendre nodes per panel
    int npp;         // nodes per particle = npan * ngl
    int64_t n;       // nodes
    int near_w;      // near panels on each side (cyclic); all panels when 2w+1 >= npan
    int n_near;      // near panels per target
    double rho;
    double eta;      // coupling of the single layer (combined representation), else 0
    // per particle
    const yk::d4* part;   // (cx, cy, bounding radius, perimeter)
    const float4* c32;    // centre as FP32 hi/lo pairs (hx, hy, lx, ly)
    const float* r32;     // bounding radius, FP32
    const int* shape_of;   // index of the particle's shape block
    // per node
    const double* x;
    const double* y;
    const double* nx;
    const double* ny;
    const double* w;
    const double* speed;
    const float2* xi;      // FP32 offset from the particle centre
    // QBX near rows per shape: [shape][local node][n_near * ngl]
    const double* cval;
    const double* cgrad;
};

}  // namespace yk
