// panel_common.cuh -- device helpers shared by the panel-method kernels.
//
// Geometry conventions follow Section 2 of the paper: airfoil b has n nodes
// x_0..x_{n-1} (x_0 at the trailing edge, counter-clockwise), the closing node
// x_n = x_0 is implied, panel i runs from x_i to x_{i+1}, and the control
// point of panel j is x_{j+1/2} = (x_j + x_{j+1}) / 2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "../../include/panel.h"

namespace panel {

constexpr double kPiF64 = 3.1415926535897932384626433832795;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kInvTwoPi = 0.15915494309189533576888376337251;
// Node coordinates must be finite and below this magnitude (the split of
// coordinates into float32 triples in the mixed path relies on it).
constexpr double kCoordLimit = 1024.0;

// Launch-side view of a batch.  All pointers are device memory.
struct Batch {
  int B;
  int n_max;
  const double* nodes;         // [sum n][2]
  const int64_t* node_off;     // [B+1]
  const int64_t* mat_off;      // [B+1]
  const int32_t* order;        // [B]
};

__device__ __forceinline__ int airfoil_n(const Batch& bt, int b) {
  return (int)(bt.node_off[b + 1] - bt.node_off[b]);
}
__device__ __forceinline__ int64_t vec_off(const Batch& bt, int b) { return bt.node_off[b] + b; }

// Warp-wide sums.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of one double; `scratch` holds >= 32 doubles.  All threads
// of the block must call it; every thread gets the result.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// Block-wide max of a non-negative double (same contract as block_sum).
__device__ __forceinline__ double block_max(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_max(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// Geometry validation of one airfoil (Section 2 node conventions), by one
// block.  Loads the nodes into xs/ys (shared, >= n entries each) and returns
// 0 or a PANEL_INFO_* code, identical in every thread.
__device__ __forceinline__ int load_and_check_geometry(const double* nodes, int n, double* xs,
                                                       double* ys, double* scratch) {
  if (n < 3) return PANEL_INFO_FEW_NODES;
  double bad = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double x = nodes[2 * k], y = nodes[2 * k + 1];
    xs[k] = x;
    ys[k] = y;
    if (!(fabs(x) < kCoordLimit) || !(fabs(y) < kCoordLimit)) bad = 1.0;  // also NaN/inf
  }
  if (block_max(bad, scratch) > 0.0) return PANEL_INFO_NONFINITE;  // (syncs)
  double zero = 0.0, area = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int k1 = (k + 1 == n) ? 0 : k + 1;
    double hx = xs[k1] - xs[k], hy = ys[k1] - ys[k];
    if (hx == 0.0 && hy == 0.0) zero = 1.0;
    area += xs[k] * ys[k1] - xs[k1] * ys[k];
  }
  if (block_max(zero, scratch) > 0.0) return PANEL_INFO_ZERO_PANEL;
  area = block_sum(area, scratch);
  if (!(area > 0.0)) return PANEL_INFO_ORIENTATION;
  return 0;
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than any earlier one on the current device: after a warm-up call no
// attribute is set any more, so later calls can be captured into CUDA graphs.
// The attribute is set even below 48 KB: a kernel's static shared memory
// counts against the default 48 KB as well.
inline cudaError_t ensure_smem_impl(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> granted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[std::make_pair(dev, kernel)];
  if (bytes <= g) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g = bytes;
  return e;
}
template <typename K>
inline cudaError_t ensure_smem(K kernel, size_t bytes) {
  return ensure_smem_impl(reinterpret_cast<const void*>(kernel), bytes);
}

// Streaming multiprocessors of the current device (queried once per device;
// 0 if the query fails).
inline int sm_count() {
  static std::mutex mu;
  static std::map<int, int> count;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = count.find(dev);
  if (it != count.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 0;
  count[dev] = n;
  return n;
}

}  // namespace panel
