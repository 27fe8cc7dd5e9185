// Thread groups that solve one linear system together, shared by the 2-D
// and 3-D solver kernels (internal header).
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"

namespace mlmc {

namespace cg = cooperative_groups;

// Cooperating threads that solve one system: a whole thread block, or one
// warp (small grids, no block barriers at all).
struct BlockGroup {
  static constexpr int kU = 1;  // cells per thread per batch in the cell loops
  static constexpr bool kStaged = false;  // runs the shared-memory staged half sweeps
  static constexpr bool kQuads = true;    // FP32 half sweeps over quads of 16-byte accesses
  __device__ __forceinline__ bool local_leader() const { return threadIdx.x == 0; }
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  // the group's blocks (one here) and this thread's place in its own block
  __device__ __forceinline__ int nblocks() const { return 1; }
  __device__ __forceinline__ int block_index() const { return 0; }
  __device__ __forceinline__ int lrank() const { return threadIdx.x; }
  __device__ __forceinline__ int lsize() const { return blockDim.x; }
  __device__ __forceinline__ void lsync() const { __syncthreads(); }
  template <typename T>
  __device__ __forceinline__ T sum(T v, T* red, int& par) const {
    return block_sum(v, red, par);
  }
};

struct WarpGroup {
  static constexpr int kU = 1;
  static constexpr bool kStaged = false;
  static constexpr bool kQuads = true;
  __device__ __forceinline__ bool local_leader() const { return (threadIdx.x & 31) == 0; }
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ int nblocks() const { return 1; }
  __device__ __forceinline__ int block_index() const { return 0; }
  __device__ __forceinline__ int lrank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int lsize() const { return 32; }
  __device__ __forceinline__ void lsync() const { __syncwarp(); }
  template <typename T>
  __device__ __forceinline__ T sum(T v, T*, int&) const {
    return warp_sum(v);
  }
};

// All threads of a thread-block cluster (large grids: the system's
// workspace is shared by the cluster's blocks through global memory / L2).
// sync() is the hardware cluster barrier (release / acquire at cluster
// scope, so global writes of one block are visible to the others after it);
// sum() reduces in each block, then every thread adds the blocks' partials
// in block-rank order through distributed shared memory, so all blocks hold
// bit-identical sums and take identical branches.
struct ClusterGroup {
  static constexpr int kU = 1;
  static constexpr bool kStaged = true;
  static constexpr bool kQuads = true;
  unsigned nblk, brank;
  double* part;  // two double slots in this block's shared memory
  __device__ __forceinline__ bool local_leader() const { return threadIdx.x == 0; }
  __device__ __forceinline__ int rank() const { return (int)(brank * blockDim.x + threadIdx.x); }
  __device__ __forceinline__ int size() const { return (int)(nblk * blockDim.x); }
  __device__ __forceinline__ void sync() const { cg::this_cluster().sync(); }
  __device__ __forceinline__ int nblocks() const { return (int)nblk; }
  __device__ __forceinline__ int block_index() const { return (int)brank; }
  __device__ __forceinline__ int lrank() const { return threadIdx.x; }
  __device__ __forceinline__ int lsize() const { return blockDim.x; }
  __device__ __forceinline__ void lsync() const { __syncthreads(); }
  template <typename T>
  __device__ __forceinline__ T sum(T v, T* red, int& par) const {
    const int slot = par;  // block_sum toggles par; the partial slot follows it
    const T b = block_sum(v, red, par);
    if (threadIdx.x == 0) part[slot] = (double)b;
    cg::this_cluster().sync();
    double t = 0.0;
    for (unsigned r = 0; r < nblk; ++r) t += *cg::this_cluster().map_shared_rank(part + slot, r);
    return (T)t;
  }
};

}  // namespace mlmc
