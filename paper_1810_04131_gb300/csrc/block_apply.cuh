// y_P (+)= B[shape(P)] x_P for every particle P, with one npp x npp block per
// particle shape stored transposed ([col j][row i]): the self blocks of the
// operators and the block preconditioner.
//
// A CTA of 256 threads takes 32 rows of one particle's block: lane l of warp
// s sums row r0 + l over the columns j = s, s + 8, ... (each warp reads 32
// consecutive entries of a column), and the eight partial sums of a row are
// added in shared memory. Grid = (particles, ceil(npp / 32)), so that a
// system of a few particles still spreads its blocks over the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace yk {

constexpr int BAPPLY_ROWS = 32;
constexpr int BAPPLY_SLICES = 8;   // 256 threads

// One CTA's tile: rows [r0, r0 + 32) of particle P's block; smem holds npp
// values of T plus 256 partial sums.
template <typename T, bool ACC>
__device__ __forceinline__ void blocks_apply_tile(int npp, const int* __restrict__ shape_of,
                                                  const T* __restrict__ B,
                                                  const double* __restrict__ x,
                                                  double* __restrict__ y, int P, int r0,
                                                  unsigned char* smem) {
    T* xs = reinterpret_cast<T*>(smem);                         // npp
    T* part = xs + ((npp + 1) & ~1);                             // [slices][rows]
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int64_t base = (int64_t)P * npp;
    for (int j = threadIdx.x; j < npp; j += blockDim.x) xs[j] = (T)x[base + j];
    __syncthreads();
    const int i = r0 + lane;
    T acc = 0;
    if (i < npp) {
        const T* M = B + (int64_t)shape_of[P] * npp * npp;
        for (int j = slice; j < npp; j += BAPPLY_SLICES) acc += M[(int64_t)j * npp + i] * xs[j];
    }
    part[slice * BAPPLY_ROWS + lane] = acc;
    __syncthreads();
    if (slice == 0 && i < npp) {
        T s = part[lane];
#pragma unroll
        for (int k = 1; k < BAPPLY_SLICES; ++k) s += part[k * BAPPLY_ROWS + lane];
        if (ACC) y[base + i] += (double)s;
        else y[base + i] = (double)s;
    }
}

template <typename T, bool ACC>
__global__ void __launch_bounds__(BAPPLY_ROWS * BAPPLY_SLICES)
k_blocks_apply(int npp, const int* __restrict__ shape_of, const T* __restrict__ B,
               const double* __restrict__ x, double* __restrict__ y) {
    extern __shared__ unsigned char bapply_smem[];
    blocks_apply_tile<T, ACC>(npp, shape_of, B, x, y, blockIdx.x, blockIdx.y * BAPPLY_ROWS,
                              bapply_smem);
}

template <typename T>
inline size_t blocks_apply_smem(int npp) {
    return sizeof(T) * (((npp + 1) & ~1) + BAPPLY_ROWS * BAPPLY_SLICES);
}

}  // namespace yk
