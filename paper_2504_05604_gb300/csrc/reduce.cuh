// Deterministic grid-wide reductions used by the solver, energy and OC kernels.
//
// Each block reduces its values (warp shuffles, then shared memory), writes
// one partial per value to a fixed slot, and bumps a counter; the block that
// arrives last sums the partials in a fixed order.  The result therefore does
// not depend on block scheduling, and no second kernel launch is needed.
#pragma once
#include "internal.cuh"

namespace to3d {

__device__ __forceinline__ int flat_block() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}
__device__ __forceinline__ int flat_nblocks() { return gridDim.x * gridDim.y * gridDim.z; }
__device__ __forceinline__ int flat_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int flat_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block sum of NV values; result valid in thread 0.  `sh` holds >= 32*NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
    const int t = flat_tid(), lane = t & 31, warp = t >> 5, nw = (flat_nthreads() + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nw ? sh[k * 32 + lane] : 0.0;
            v[k] = warp_sum(s);
        }
    }
}

// Grid sum: returns true in every thread of the last block, where out[k]
// (in shared memory, NV entries) holds the grid totals.  `ismax` marks
// values reduced with max instead of sum (block and grid level).
template <int NV>
__device__ bool grid_sum(const Reducer red, double (&v)[NV], double* sh, double* out,
                         unsigned ismax = 0u) {
    const int t = flat_tid(), lane = t & 31, warp = t >> 5, nw = (flat_nthreads() + 31) >> 5;
    __shared__ int s_last;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = ((ismax >> k) & 1u) ? warp_max(v[k]) : warp_sum(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = v[k];
    }
    __syncthreads();
    const int b = flat_block(), nb = flat_nblocks();
    if (t == 0) {
        for (int k = 0; k < NV; ++k) {
            double s = ((ismax >> k) & 1u) ? -1e300 : 0.0;
            for (int w = 0; w < nw; ++w)
                s = ((ismax >> k) & 1u) ? fmax(s, sh[k * 32 + w]) : s + sh[k * 32 + w];
            red.partials[(size_t)k * kMaxBlocks + b] = s;
        }
        __threadfence();
        unsigned ticket = atomicAdd(red.counter, 1u);
        s_last = (ticket == (unsigned)nb - 1u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const bool mx = (ismax >> k) & 1u;
        double s = mx ? -1e300 : 0.0;
        for (int i = t; i < nb; i += flat_nthreads()) {
            double pv = __ldcg(&red.partials[(size_t)k * kMaxBlocks + i]);
            s = mx ? fmax(s, pv) : s + pv;
        }
        acc[k] = mx ? warp_max(s) : warp_sum(s);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = acc[k];
    }
    __syncthreads();
    if (t == 0) {
        for (int k = 0; k < NV; ++k) {
            const bool mx = (ismax >> k) & 1u;
            double s = mx ? -1e300 : 0.0;
            for (int w = 0; w < nw; ++w) s = mx ? fmax(s, sh[k * 32 + w]) : s + sh[k * 32 + w];
            out[k] = s;
        }
        *red.counter = 0u;
    }
    __syncthreads();
    return true;
}

}  // namespace to3d
