// ragged.cuh -- the sweeps of a ragged batch (mixed precision) in one
// persistent launch.
//
// k_group has sorted the instances into size classes, longest horizon first
// inside a class (perm).  k_ragged_items turns that order into work items --
// up to 8 instances of one warp-sweep size (one warp each) or one instance
// of a CTA-sweep size -- and orders the items by an estimate of their chain
// length (horizon x a per-stage cost of the size class), longest first.
// k_ragged_sweep then runs one CTA of 256 threads per SM; each CTA takes the
// next item from an atomic counter until none is left: a warp-size item
// runs the warp sweep of sweep32.cuh on each of its warps, a CTA-size item
// the CTA sweep of seqx.cuh.  No CTA waits on another (the counter is the
// only shared state), so the launch cannot deadlock whatever the order in
// which CTAs start.  Sizes: the exact classes with an FP32 warp sweep of
// even m ((4,2), (6,2), (12,4)) or a CTA sweep ((24,8), (32,8), (48,16)).
#pragma once

#include "common.cuh"
#include "seqx.cuh"
#include "sweep32.cuh"

namespace rlqr {

// Per-stage chain cost of a class (relative units, from the measured
// per-stage times of its sweep): orders the items.
__host__ __device__ inline int ragged_stage_cost(int cls) {
  switch (cls) {
    case 0: return 12;
    case 2: return 18;
    case 3: return 45;
    case 4: return 100;
    case 5: return 160;
    case 6: return 240;
    default: return 0;
  }
}

constexpr int kRaggedWarps = 8;  // instances per warp-size item (= warps of the CTA)
constexpr int kRaggedBuckets = 256;

// Work items (class, first perm index, instances) into items, their number
// into meta[0] and the item counter meta[1] = 0.  One block.
__global__ void k_ragged_items(RaggedPlan P, const int32_t *perm, const int32_t *dN, int4 *items,
                               int32_t *meta) {
  __shared__ int start[kRaggedClasses + 1];
  __shared__ int hist[kRaggedBuckets];
  const int tid = threadIdx.x, T = blockDim.x;
  if (tid == 0) {
    int acc = 0;
    for (int c = 0; c < kRaggedClasses; ++c) {
      start[c] = acc;
      const int k = ragged_kind(c);
      if (k == 1) acc += (P.cnt[c] + kRaggedWarps - 1) / kRaggedWarps;
      else if (k == 2) acc += P.cnt[c];
    }
    start[kRaggedClasses] = acc;
  }
  for (int h = tid; h < kRaggedBuckets; h += T) hist[h] = 0;
  __syncthreads();
  const int total = start[kRaggedClasses];
  // bucket of an item: finer for longer chains, longest first
  auto decode = [&](int j, int4 &w) -> int {
    int c = 0;
    while (c + 1 < kRaggedClasses && start[c + 1] <= j) ++c;
    const int loc = j - start[c];
    const int g = ragged_kind(c) == 1 ? kRaggedWarps : 1;
    const int first = P.off[c] + loc * g;
    const int cnt = min(g, P.cnt[c] - loc * g);
    w = make_int4(c, first, cnt, 0);
    const float cost = (float)dN[perm[first]] * (float)ragged_stage_cost(c);
    const int lb = (int)(8.0f * log2f(fmaxf(cost, 1.0f)));
    return kRaggedBuckets - 1 - min(kRaggedBuckets - 1, lb);
  };
  for (int j = tid; j < total; j += T) {
    int4 w;
    atomicAdd(&hist[decode(j, w)], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int h = 0; h < kRaggedBuckets; ++h) {
      const int v = hist[h];
      hist[h] = acc;
      acc += v;
    }
    meta[0] = total;
    meta[1] = 0;
  }
  __syncthreads();
  for (int j = tid; j < total; j += T) {
    int4 w;
    const int h = decode(j, w);
    items[atomicAdd(&hist[h], 1)] = w;
  }
}

template <int NX, int NU>
__device__ __forceinline__ void ragged_warp_item(const BatchArgs &a, const int32_t *perm, int4 w,
                                                 unsigned char *smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < w.z)
    sweep32_body<NX, NU, true>(a, perm[w.y + warp], smem + (size_t)warp * sizeof(Sw32<NX, NU>),
                               lane);
}

__host__ __device__ constexpr size_t ragged_max(size_t x, size_t y) { return x > y ? x : y; }

// Shared memory of a persistent-sweep CTA: the largest item's.
constexpr size_t kRaggedSmem = ragged_max(
    ragged_max(kRaggedWarps * sizeof(Sw32<4, 2>), kRaggedWarps * sizeof(Sw32<6, 2>)),
    ragged_max(ragged_max(kRaggedWarps * sizeof(Sw32<12, 4>), sizeof(SxSmem<float, 24, 8>)),
               ragged_max(sizeof(SxSmem<float, 32, 8>), sizeof(SxSmem<float, 48, 16>))));

__global__ void __launch_bounds__(scan::kTH, 1)
    k_ragged_sweep(BatchArgs a, const int32_t *perm, const int4 *items, int32_t *meta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  const int nitems = __ldcg(meta);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(meta + 1, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;  // uniform over the block
    const int4 w = items[it];
    switch (w.x) {
      case 0: ragged_warp_item<4, 2>(a, perm, w, smem_raw); break;
      case 2: ragged_warp_item<6, 2>(a, perm, w, smem_raw); break;
      case 3: ragged_warp_item<12, 4>(a, perm, w, smem_raw); break;
      case 4: seqx_body<float, 24, 8, true>(a, perm[w.y], smem_raw); break;
      case 5: seqx_body<float, 32, 8, true>(a, perm[w.y], smem_raw); break;
      case 6: seqx_body<float, 48, 16, true>(a, perm[w.y], smem_raw); break;
      default: break;
    }
    __syncthreads();  // shared memory and s_item free for the next item
  }
}

}  // namespace rlqr
