// Counting sort of the particles by mesh cell, so that a block's particles gather from and deposit into
// neighbouring cells also after clustering has scattered lattice neighbours over many lines.  The particles keep
// their Lagrangian displacements; a slot -> lattice index map (order) says which lattice site each storage slot
// holds.
//
// Keys are z-row segments of 32 cells.  Row order (the default): key = (ix n + iy) ceil(n / 32) + iz / 32.
// Brick order (asked for by the tiled kick-drift-deposit, mesh sides that particle_bricks_ok accepts): the mesh
// is cut into bricks of 8 x 8 x 32 cells, walked with bz slowest, then bx, then by, and a brick's 64 keys are
// its (x, y) rows, key = brick * 64 + 8 (ix mod 8) + (iy mod 8); after the sort the particles of brick b occupy
// the slots [offset(64 b), offset(64 b + 64)), which the tiled kick-drift-deposit takes as its block's range.  A particle's rank within its key comes from an
// atomic counter, the key offsets from an exclusive scan of the counters (three passes: block sums, one-block
// scan of the block sums, block scans plus offsets).  Each destination offset + rank then learns its source
// slot, and a gather moves displacements, momenta and the lattice index there (coalesced writes).  The order
// within a key depends on the atomics.
#include <cuda_runtime.h>

#include "common.h"
#include "mesh_kernels.h"

namespace hrt {

namespace {

constexpr int kSeg = 32;           // cells per key along z
constexpr int kScanThreads = 256;  // threads per scan block, 4 counters each
constexpr int kScanItems = 4 * kScanThreads;

__device__ __forceinline__ int cell_of(int q_node, float d_cells, int n) {
  int i = q_node + static_cast<int>(floorf(d_cells));
  if (static_cast<unsigned>(i) >= static_cast<unsigned>(n)) {
    i %= n;
    if (i < 0) i += n;
  }
  return i;
}

// Key and rank of every particle.  Particles already in cell order (every re-sort) put runs of equal keys in a
// warp, so the lanes of a warp with the same key take their ranks from one atomic of the group's size (lanes
// found by __match_any_sync, ranked by lane within the group).  Every lane of a warp runs the matching, so the
// kernel keeps out-of-range threads until then.
__global__ void sort_key_kernel(const float* __restrict__ disp, const int32_t* __restrict__ order, int64_t np,
                                int n_side, int lns, int ratio, int n, int nseg, int bricks, float inv_cell,
                                int32_t* __restrict__ counts, int32_t* __restrict__ keys, int32_t* __restrict__ ranks) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const bool valid = i < np;
  int32_t key = -1;
  if (valid) {
    const unsigned lag = order ? static_cast<unsigned>(__ldg(order + i)) : static_cast<unsigned>(i);
    int qi, qj, qk;
    if (lns >= 0) {  // n_side a power of two: the lattice site by shifts
      const unsigned mask = (1u << lns) - 1u;
      qk = static_cast<int>(lag & mask);
      qj = static_cast<int>((lag >> lns) & mask);
      qi = static_cast<int>(lag >> (2 * lns));
    } else {
      const unsigned ns = static_cast<unsigned>(n_side);
      qk = static_cast<int>(lag % ns);
      qj = static_cast<int>((lag / ns) % ns);
      qi = static_cast<int>(lag / ns / ns);
    }
    const int ix = cell_of(qi * ratio, __ldg(disp + i) * inv_cell, n);
    const int iy = cell_of(qj * ratio, __ldg(disp + np + i) * inv_cell, n);
    const int iz = cell_of(qk * ratio, __ldg(disp + 2 * np + i) * inv_cell, n);
    if (bricks) {
      const int nb = n / kBrickXY;
      key = (((iz / kSeg) * nb + ix / kBrickXY) * nb + iy / kBrickXY) * kBrickKeys + (ix % kBrickXY) * kBrickXY +
            iy % kBrickXY;
    } else {
      key = (ix * n + iy) * nseg + iz / kSeg;
    }
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(full, key);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (valid && lane == leader) base = atomicAdd(counts + key, __popc(peers));
  base = __shfl_sync(full, base, leader);
  if (valid) {
    keys[i] = key;
    ranks[i] = base + __popc(peers & ((1u << lane) - 1u));
  }
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
  // warp-level inclusive scan, then the warp totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh[lane] = w;
  }
  __syncthreads();
  total = sh[(blockDim.x >> 5) - 1];
  const int before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(const int32_t* __restrict__ counts, int64_t T,
                                                                 int32_t* __restrict__ block_sums) {
  __shared__ int sh[32];
  const int64_t base = blockIdx.x * static_cast<int64_t>(kScanItems) + 4 * threadIdx.x;
  int v = 0;
  for (int k = 0; k < 4; ++k)
    if (base + k < T) v += counts[base + k];
  int total;
  block_exclusive_scan(v, sh, total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums in place (each thread a contiguous chunk).
__global__ void __launch_bounds__(1024) scan_block_sums_kernel(int32_t* __restrict__ sums, int nb) {
  __shared__ int sh[32];
  const int chunk = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * chunk, hi = min(nb, lo + chunk);
  int v = 0;
  for (int i = lo; i < hi; ++i) v += sums[i];
  int total;
  int run = block_exclusive_scan(v, sh, total);
  for (int i = lo; i < hi; ++i) {
    const int c = sums[i];
    sums[i] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(int32_t* __restrict__ counts, int64_t T,
                                                                  const int32_t* __restrict__ block_sums) {
  __shared__ int sh[32];
  const int64_t base = blockIdx.x * static_cast<int64_t>(kScanItems) + 4 * threadIdx.x;
  int c[4], v = 0;
  for (int k = 0; k < 4; ++k) {
    c[k] = base + k < T ? counts[base + k] : 0;
    v += c[k];
  }
  int total;
  int run = block_exclusive_scan(v, sh, total) + block_sums[blockIdx.x];
  for (int k = 0; k < 4; ++k)
    if (base + k < T) {
      counts[base + k] = run;
      run += c[k];
    }
}

// Destination slot of every particle, stored as the source of every destination (a 4-byte scattered write per
// particle), so that the move below writes its six arrays coalesced and reads them scattered.
__global__ void sort_invert_kernel(int64_t np, const int32_t* __restrict__ offsets, const int32_t* __restrict__ keys,
                                   const int32_t* __restrict__ ranks, int32_t* __restrict__ src) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= np) return;
  src[static_cast<int64_t>(offsets[keys[i]]) + ranks[i]] = static_cast<int32_t>(i);
}

__global__ void sort_gather_kernel(const float* __restrict__ disp, const float* __restrict__ mom,
                                   const int32_t* __restrict__ order, int64_t np, const int32_t* __restrict__ src,
                                   float* __restrict__ disp_out, float* __restrict__ mom_out,
                                   int32_t* __restrict__ order_out) {
  const int64_t d = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (d >= np) return;
  const int64_t i = src[d];
  for (int c = 0; c < 3; ++c) {
    disp_out[c * np + d] = __ldg(disp + c * np + i);
    mom_out[c * np + d] = __ldg(mom + c * np + i);
  }
  order_out[d] = order ? __ldg(order + i) : static_cast<int32_t>(i);
}

__global__ void unsort_kernel(const float* __restrict__ in, const int32_t* __restrict__ order, int64_t np,
                              float* __restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= np) return;
  const int64_t p = order[i];
  for (int c = 0; c < 3; ++c) out[c * np + p] = in[c * np + i];
}

}  // namespace

hrt_status launch_particle_sort(const float* disp, const float* mom, const int32_t* order, int64_t n_side, int64_t n,
                                double box, float* disp_out, float* mom_out, int32_t* order_out, int32_t* counts,
                                int32_t* keys, int32_t* ranks, int32_t* src, cudaStream_t s, bool bricks) {
  const int64_t np = n_side * n_side * n_side;
  if (np == 0) return HRT_OK;
  if (np > INT32_MAX) return fail(HRT_ERR_INVALID_ARG, "too many particles for the sort");
  const int nseg = static_cast<int>((n + kSeg - 1) / kSeg);
  const int64_t T = n * n * nseg;
  const int64_t nb = (T + kScanItems - 1) / kScanItems;
  // counters, then the block sums after them
  HRT_CUDA(cudaMemsetAsync(counts, 0, static_cast<size_t>(T) * sizeof(int32_t), s));
  int lns = 0;
  while ((int64_t{1} << lns) < n_side) ++lns;
  if ((int64_t{1} << lns) != n_side) lns = -1;
  sort_key_kernel<<<blocks_for(np, 256), 256, 0, s>>>(disp, order, np, static_cast<int>(n_side), lns,
                                                      static_cast<int>(n / n_side), static_cast<int>(n), nseg,
                                                      bricks && particle_bricks_ok(n) ? 1 : 0, static_cast<float>(n / box),
                                                      counts, keys, ranks);
  HRT_LAUNCHED("sort_key_kernel");
  int32_t* sums = counts + T;
  scan_sums_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(counts, T, sums);
  HRT_LAUNCHED("scan_sums_kernel");
  scan_block_sums_kernel<<<1, 1024, 0, s>>>(sums, static_cast<int>(nb));
  HRT_LAUNCHED("scan_block_sums_kernel");
  scan_apply_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(counts, T, sums);
  HRT_LAUNCHED("scan_apply_kernel");
  sort_invert_kernel<<<blocks_for(np, 256), 256, 0, s>>>(np, counts, keys, ranks, src);
  HRT_LAUNCHED("sort_invert_kernel");
  sort_gather_kernel<<<blocks_for(np, 256), 256, 0, s>>>(disp, mom, order, np, src, disp_out, mom_out, order_out);
  HRT_LAUNCHED("sort_gather_kernel");
  return HRT_OK;
}

int64_t particle_sort_counts(int64_t n) {
  const int64_t T = n * n * ((n + kSeg - 1) / kSeg);
  return T + (T + kScanItems - 1) / kScanItems;
}

hrt_status launch_unsort(const float* in, const int32_t* order, int64_t np, float* out, cudaStream_t s) {
  if (np == 0) return HRT_OK;
  unsort_kernel<<<blocks_for(np, 256), 256, 0, s>>>(in, order, np, out);
  HRT_LAUNCHED("unsort_kernel");
  return HRT_OK;
}

}  // namespace hrt
