// Device-side helpers shared by the kernel files of libbchar.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace bchar {

template <class real> struct Real;
template <> struct Real<double> {
    static __device__ __forceinline__ const double *w(const MeshView &m, int a) { return m.wd[a]; }
    static __device__ __forceinline__ double phi(const MeshView &m, int64_t k) { return m.phi[k]; }
    static __device__ __forceinline__ double rad(const MeshView &m, int64_t k) { return m.rad[k]; }
    static __device__ __forceinline__ double rhophi(const MeshView &m, int64_t k) { return m.rhophi[k]; }
    static __device__ __forceinline__ const double *u(const VelView &v, int a) { return v.u[a]; }
};
template <> struct Real<float> {
    static __device__ __forceinline__ const float *w(const MeshView &m, int a) { return m.wf[a]; }
    static __device__ __forceinline__ float phi(const MeshView &m, int64_t k) { return m.phif[k]; }
    static __device__ __forceinline__ float rad(const MeshView &m, int64_t k) { return m.radf[k]; }
    static __device__ __forceinline__ float rhophi(const MeshView &m, int64_t k) { return m.rhophif[k]; }
    static __device__ __forceinline__ const float *u(const VelView &v, int a) { return v.uf[a]; }
};

__device__ __forceinline__ void split_cell(const MeshView &m, int64_t k, int c[3]) {
    c[0] = static_cast<int>(k % m.n[0]);
    c[1] = static_cast<int>((k / m.n[0]) % m.n[1]);
    c[2] = static_cast<int>(k / (static_cast<int64_t>(m.n[0]) * m.n[1]));
}

__device__ __forceinline__ int64_t flat_cell(const MeshView &m, const int c[3]) {
    return c[0] + static_cast<int64_t>(m.n[0]) * (c[1] + static_cast<int64_t>(m.n[1]) * c[2]);
}

__device__ __forceinline__ void unpack_counts(int32_t p, int c[3]) {
    c[0] = p & 255;
    c[1] = (p >> 8) & 255;
    c[2] = (p >> 16) & 255;
}

// Largest of non-negative doubles through their bit patterns (order-free).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *slot, double v) {
    atomicMax(slot, static_cast<unsigned long long>(__double_as_longlong(v)));
}

// Programmatic dependent launch: wait until the kernel before this one in the
// stream has completed and its writes are visible (a no-op when this kernel
// was launched without the attribute), then allow the next kernel's blocks to
// be scheduled while this one runs; they wait the same way before reading.
__device__ __forceinline__ void dep_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Deterministic block sum: warp shuffles, then one warp over the warp sums.
// Every thread of the block must call it; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_sums[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_sums[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? warp_sums[lane] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double warp_max[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_max[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? warp_max[lane] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace bchar
