// fe_vec.cuh -- shared pieces of the vector / reduction kernels.
#pragma once
#include "fe_apply_kernel.cuh"

#define RED_BLOCKS 608  // 4 CTAs per SM on 152 SMs; fixed, so reductions are reproducible
#define RED_THREADS 256
#define RED_SLOTS 8
#define RED_U 4  // elements per thread whose loads are issued together in the reduction loops

fe_status fe_ensure_reduction(const fe_mesh* m);

__device__ __forceinline__ dw dw_shfl_down(dw v, int off) {
  return {__shfl_down_sync(0xffffffffu, v.h, off), __shfl_down_sync(0xffffffffu, v.l, off)};
}

// CTA-wide double-word sum in a fixed shuffle tree; result valid in thread 0
__device__ __forceinline__ dw block_reduce_dw(dw v, dw* sh /* [32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = dw_add(v, dw_shfl_down(v, off));
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : dw{0.0f, 0.0f};
  if (wid == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = dw_add(v, dw_shfl_down(v, off));
  }
  __syncthreads();
  return v;
}

template <class S>
__device__ __forceinline__ dw to_dw(S v);
template <>
__device__ __forceinline__ dw to_dw<double>(double v) { return dw_from_double(v); }
template <>
__device__ __forceinline__ dw to_dw<float>(float v) { return {v, 0.0f}; }

// CTA-wide binary64 sum in a fixed shuffle tree; result valid in thread 0
__device__ __forceinline__ double block_reduce_f64(double v, double* sh /* [32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  }
  __syncthreads();
  return v;
}
