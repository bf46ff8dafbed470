// rlqr_api.cu -- C ABI of the B300 dual-regularized LQR library (include/rlqr.h).
//
// Host side: argument validation, workspace layout, kernel selection by the
// instance dimensions, and the launch sequences of the factor / solve /
// residual / batched entry points.  Every step of the solve runs in the
// kernels of seq.cuh and refine.cuh; nothing here touches problem data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "common.cuh"
#include "cross.cuh"
#include "escalate.cuh"
#include "launch.cuh"
#include "residual.cuh"
#include "residual_grid.cuh"
#include "scan.cuh"

namespace rlqr {

Instr g_instr;

// One warp per stage; as many warps per CTA (<= 8) as the dense stage blocks
// of the largest instance fit in shared memory.
static cudaError_t launch_residual(const BatchArgs &a, int rs_max, int store, double *res_out,
                                   double *norms_out, int recompute, int standalone,
                                   cudaStream_t s, int cert_g = 0, int do_residual = 1) {
  const size_t per_warp = residual_warp_bytes(rs_max);
  int warps = (int)std::min<size_t>(8, (200u * 1024u) / per_warp);
  warps = std::max(warps, 1);
  const size_t bytes = per_warp * warps;
  auto kern = k_residual;
  cudaError_t e = set_smem(kern, bytes);
  if (e != cudaSuccess) return e;
  LaunchScope ls(!do_residual ? "k_cert_fp64" : "k_residual_fp64", s);
  kern<<<a.count, 32 * warps, bytes, s>>>(a, store, res_out, norms_out, recompute, standalone,
                                         rs_max, cert_g, do_residual);
  return cudaGetLastError();
}

// Stage-parallel first residual over every instance of `a` (residual_grid.cuh):
// spre is the work-item prefix sum of a batch (null for one instance), items
// the number of work items (sum of N_b + 1).  Mixed: the residual is stored
// for the refinement and, when cert_g, the control pivots are certified.
static cudaError_t launch_grid_residual(const BatchArgs &a, const int64_t *spre, int64_t items,
                                        bool mixed, int cert_g, cudaStream_t s) {
  BatchArgs ab = a;
  ab.perm = nullptr;
  ab.goff = 0;
  LaunchScope ls("k_residual_grid", s);  // FP64 products in both precisions
  const int cb = (int)std::min<int64_t>((ab.count + 255) / 256, 148 * 16);
  k_resb_reset<<<cb, 256, 0, s>>>(ab);
  if (mixed && cert_g)
    k_certb<<<(int)std::min<int64_t>((items + 255) / 256, 148 * 16), 256, 0, s>>>(ab, spre, items);
  k_resb<<<(int)std::min<int64_t>((items + 7) / 8, 148 * 16), 256, 0, s>>>(ab, spre, items,
                                                                           mixed ? 1 : 0);
  k_resb_final<<<cb, 256, 0, s>>>(ab);
  return cudaGetLastError();
}

// FP64 certificate with margin of every stored FP32 control pivot of a batch
// (k_certb), without a residual: the fused route's first refinement pass
// computes that.
static cudaError_t launch_cert_g(const BatchArgs &a, const int64_t *spre, int64_t items,
                                 cudaStream_t s) {
  BatchArgs ab = a;
  ab.perm = nullptr;
  ab.goff = 0;
  LaunchScope ls("k_cert_g", s);
  k_certb<<<(int)std::min<int64_t>((items + 255) / 256, 148 * 16), 256, 0, s>>>(ab, spre, items);
  return cudaGetLastError();
}

// First residual of a uniform launch group (or one instance): stored for the
// refinement and certifying the control pivots when cert_g (mixed), or the
// FP64 backward error only.  The sizes of the FP32 warp sweeps take the
// float-float warp residual (mixed) or the generic FP64 one; the rest take
// the stage-parallel grid residual.
static bool warp_res32_size(int n, int m) {
  return ((n == 4 || n == 6) && (m == 1 || m == 2)) || (n == 12 && (m == 3 || m == 4));
}

// Residual route of a uniform launch group of a warp size: 0 = by size (the
// warp residual), 1 = the warp residual, 2 = the stage-parallel grid
// residual, 5 = (mixed, with refinement) no separate first residual: the
// first refinement pass computes it.  Batches record the autotuner's choice (rlqr_autotune_batched)
// per (nx, nu, precision, floor(log2 max N), floor(log2 count)).
static std::mutex g_route_mu;
static std::map<uint64_t, int> g_res_route;

static int ilog2(int v) {
  int l = 0;
  while (l < 30 && (1 << (l + 1)) <= v) ++l;
  return l;
}

static uint64_t route_key(int N, int n, int m, int tsize, int count) {
  return ((uint64_t)n << 40) | ((uint64_t)m << 32) | ((uint64_t)tsize << 24) |
         ((uint64_t)ilog2(N) << 8) | (uint64_t)ilog2(count);
}

// Sweep route of a ragged batch: 3 = one launch per size class on
// concurrent streams (the default), 4 = one persistent launch (ragged.cuh);
// recorded per (set of size classes, precision, floor(log2 max N),
// floor(log2 count)).
static uint64_t ragged_key(int mask, int N, int tsize, int count) {
  return (1ull << 63) | ((uint64_t)mask << 32) | ((uint64_t)tsize << 24) |
         ((uint64_t)ilog2(N) << 8) | (uint64_t)ilog2(count);
}

static int ragged_route(int mask, int N, int tsize, int count) {
  std::lock_guard<std::mutex> lock(g_route_mu);
  const auto it = g_res_route.find(ragged_key(mask, N, tsize, count));
  return it == g_res_route.end() ? 3 : it->second;
}

static int residual_route(int N, int n, int m, int tsize, int count) {
  std::lock_guard<std::mutex> lock(g_route_mu);
  const auto it = g_res_route.find(route_key(N, n, m, tsize, count));
  return it == g_res_route.end() ? 0 : it->second;
}

static cudaError_t launch_first_residual(const BatchArgs &a, int n, int m, bool mixed, int cert_g,
                                         const int64_t *spre, int64_t items, cudaStream_t s,
                                         int route = 0) {
  if (!warp_res32_size(n, m) || (route == 2 && spre))
    return launch_grid_residual(a, spre, items, mixed, cert_g, s);
  if (mixed) return launch_residual32<float>(n, m, true, a, cert_g, s);
  return launch_residual(a, 2 * n + m, 0, nullptr, nullptr, 1, 0, s);
}

// FP64 re-decision of the pivot certificate (k_escalate) for the instances
// of `a` whose FP32-computed pivots a margin test could not decide; the
// other instances' blocks return at once.  solved: the call also produced a
// solution (the status output then reflects convergence too); scan: the
// factor came from the associative scan.
static cudaError_t launch_escalate(const BatchArgs &a, int nmax, int mmax, int solved, int scan,
                                   cudaStream_t s) {
  const size_t bytes = escalate_smem_bytes(nmax, mmax);
  cudaError_t e = set_smem(k_escalate, bytes);
  if (e != cudaSuccess) return e;
  BatchArgs ab = a;
  ab.perm = nullptr;
  ab.goff = 0;
  LaunchScope ls("k_escalate", s);
  k_escalate<<<ab.count, kEscThreads, bytes, s>>>(ab, solved, scan);
  return cudaGetLastError();
}

// After a refinement pass: the full residual, recomputed in FP64 accuracy for
// the instances whose convergence the pass's rounding bound could not
// certify (the others return at once).  The next pass then starts from an
// exact residual, and a certified backward error never rests on the bound.
static cudaError_t launch_recheck(const BatchArgs &a, int n, int m, const int64_t *spre,
                                  int64_t items, cudaStream_t s, int route = 0,
                                  bool uniform = true) {
  BatchArgs ar = a;
  ar.recheck = 1;
  return uniform ? launch_first_residual(ar, n, m, true, 0, spre, items, s, route)
                 : launch_grid_residual(ar, spre, items, true, 0, s);
}

// ---- ragged batches: size classes and the launch order
// Class of an instance: its exact (n, m) when that size has specialized
// kernels (warp-per-instance or compile-time CTA), else its bucket.
constexpr int kNumExact = 7, kNumClasses = kNumExact + 4;
constexpr int kNBuckets = 64;  // horizon buckets for the longest-first order

__host__ __device__ inline int size_class(int n, int m) {
  if (n == 4 && m == 2) return 0;
  if (n == 6 && m == 1) return 1;
  if (n == 6 && m == 2) return 2;
  if (n == 12 && m == 4) return 3;
  if (n == 24 && m == 8) return 4;
  if (n == 32 && m == 8) return 5;
  if (n == 48 && m == 16) return 6;
  const int bk = n <= 8 && m <= 4 ? 0 : (n <= 16 && m <= 8 ? 1 : (n <= 32 && m <= 16 ? 2 : 3));
  return kNumExact + bk;
}

struct ClassOffsets {
  int off[kNumClasses];
};

// perm: instances grouped by class (class c starts at off[c]), longest
// horizon first within a class (counting sort over horizon buckets of
// width q).  One block.
__global__ void k_group(int count, const int32_t *dN, const int32_t *dn, const int32_t *dm,
                        int q, ClassOffsets co, int32_t *perm) {
  __shared__ int cnt[kNumClasses * kNBuckets];
  for (int i = threadIdx.x; i < kNumClasses * kNBuckets; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    const int cls = size_class(dn[b], dm[b]);
    const int nb = kNBuckets - 1 - min(kNBuckets - 1, dN[b] / q);
    atomicAdd(&cnt[cls * kNBuckets + nb], 1);
  }
  __syncthreads();
  if (threadIdx.x < kNumClasses) {
    const int c = threadIdx.x;
    int acc = co.off[c];
    for (int j = 0; j < kNBuckets; ++j) {
      const int v = cnt[c * kNBuckets + j];
      cnt[c * kNBuckets + j] = acc;
      acc += v;
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    const int cls = size_class(dn[b], dm[b]);
    const int nb = kNBuckets - 1 - min(kNBuckets - 1, dN[b] / q);
    perm[atomicAdd(&cnt[cls * kNBuckets + nb], 1)] = b;
  }
}

// Streams of the size classes of a ragged batch: one non-blocking stream per
// class and device, created on first use and kept; the classes' launch
// sequences are forked from the caller's stream and joined back with events
// (which also places them in a graph when the caller's stream is being
// captured).  The mutex orders the fork/join enqueues of concurrent callers.
struct ClassStreams {
  bool ok = false;
  cudaStream_t st[kNumClasses];
  cudaEvent_t fork, join[kNumClasses];
  // the FP64 re-decision of escalated certificates, concurrent with the
  // refinement passes
  cudaStream_t esc;
  cudaEvent_t esc_fork, esc_join;
};
constexpr int kMaxClassDevices = 64;
static ClassStreams g_class_streams[kMaxClassDevices];
static std::mutex g_class_mu;

static ClassStreams *class_streams_locked() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxClassDevices) return nullptr;
  ClassStreams &cs = g_class_streams[dev];
  if (!cs.ok) {
    for (int c = 0; c < kNumClasses; ++c) {
      if (cudaStreamCreateWithFlags(&cs.st[c], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&cs.join[c], cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    }
    if (cudaEventCreateWithFlags(&cs.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs.esc, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&cs.esc_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cs.esc_join, cudaEventDisableTiming) != cudaSuccess)
      return nullptr;
    cs.ok = true;
  }
  return &cs;
}

// Header of a batch's workspace: per-instance byte offsets (int64), the
// launch permutation of a ragged batch (int32), the exclusive prefix sum of
// N_b + 1 (int64, count + 1 entries: the residual's work items), then the
// persistent ragged sweep's work items (int4, at most count) and its item
// count and counter (two int32).
__host__ __device__ inline size_t batch_header_items(int count) {
  return align_up((size_t)count * sizeof(int64_t)) + align_up((size_t)count * sizeof(int32_t)) +
         align_up((size_t)(count + 1) * sizeof(int64_t));
}
__host__ __device__ inline size_t batch_header_bytes(int count) {
  return batch_header_items(count) + align_up((size_t)count * sizeof(int4)) +
         align_up(2 * sizeof(int32_t));
}

// Per-instance workspace offsets of a batch (exclusive prefix sum of
// ws_layout(...).total after the header) and the work-item prefix sum.
__global__ void k_plan(int count, const int32_t *dN, const int32_t *dn, const int32_t *dm,
                       int tsize, int64_t *ows) {
  __shared__ int64_t part[1024], part2[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (count + T - 1) / T;
  const int lo = min(count, t * per), hi = min(count, lo + per);
  int64_t s = 0, s2 = 0;
  for (int b = lo; b < hi; ++b) {
    s += (int64_t)ws_layout(dN[b], dn[b], dm[b], tsize).total;
    s2 += (int64_t)dN[b] + 1;
  }
  // exclusive prefix sums of the per-thread partials over the block: an
  // inclusive shuffle scan in each warp, then one over the warp totals
  // (blockDim.x a multiple of 32, at most 1024)
  __shared__ int64_t wsum[32], wsum2[32];
  const int lane = t & 31, wid = t >> 5, nw = T >> 5;
  int64_t in = s, in2 = s2;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, in, o), u2 = __shfl_up_sync(0xffffffffu, in2, o);
    if (lane >= o) {
      in += u;
      in2 += u2;
    }
  }
  if (lane == 31) {
    wsum[wid] = in;
    wsum2[wid] = in2;
  }
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < nw ? wsum[lane] : 0, w2 = lane < nw ? wsum2[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, w, o), u2 = __shfl_up_sync(0xffffffffu, w2, o);
      if (lane >= o) {
        w += u;
        w2 += u2;
      }
    }
    wsum[lane] = w;  // inclusive over warps 0..lane
    wsum2[lane] = w2;
  }
  __syncthreads();
  const int64_t before = wid > 0 ? wsum[wid - 1] : 0, before2 = wid > 0 ? wsum2[wid - 1] : 0;
  part[t] = (int64_t)batch_header_bytes(count) + before + in - s;
  part2[t] = before2 + in2 - s2;
  __syncthreads();
  int64_t *spre = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(ows) +
                                              align_up((size_t)count * sizeof(int64_t)) +
                                              align_up((size_t)count * sizeof(int32_t)));
  int64_t acc = part[t], acc2 = part2[t];
  for (int b = lo; b < hi; ++b) {
    ows[b] = acc;
    spre[b] = acc2;
    acc += (int64_t)ws_layout(dN[b], dn[b], dm[b], tsize).total;
    acc2 += (int64_t)dN[b] + 1;
  }
  if (hi == count && lo < hi) spre[count] = acc2;
  if (count == 0 && t == 0) spre[0] = 0;
}

static bool valid_opts(const rlqr_opts *o) {
  if (!o) return false;
  if (o->prec != RLQR_FP64 && o->prec != RLQR_MIXED) return false;
  if (o->algo != RLQR_ALGO_AUTO && o->algo != RLQR_ALGO_SEQ && o->algo != RLQR_ALGO_SCAN)
    return false;
  if (o->max_refine < 0 || o->max_refine > 64) return false;
  if (!(o->tol > 0.0) || !std::isfinite(o->tol)) return false;
  if (o->flags & ~RLQR_OPT_SYNC) return false;
  return true;
}

// RLQR_OPT_SYNC: wait for the stream and turn the instance state at the
// start of `ws` into the host return (factor: the pivot status; solve: the
// status the device writes, convergence included for the mixed path).
static rlqr_status sync_status(const rlqr_opts *o, const void *ws, bool solved, bool mixed,
                               cudaStream_t s) {
  if (!(o->flags & RLQR_OPT_SYNC)) return RLQR_OK;
  InstState st;
  if (cudaMemcpyAsync(&st, ws, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RLQR_ERR_CUDA;
  if (st.pivot_status == RLQR_ERR_SINGULAR) return RLQR_ERR_SINGULAR;
  if (solved && mixed && !st.converged) return RLQR_ERR_NOT_CONVERGED;
  return static_cast<rlqr_status>(st.pivot_status);
}

static bool valid_dims(int N, int n, int m) {
  return N >= 1 && n >= 1 && m >= 1 && bucket_of(n, m) >= 0 && N < (1 << 28);
}

static bool valid_problem(const rlqr_problem *p) {
  if (!p || !valid_dims(p->N, p->nx, p->nu)) return false;
  if (!(p->delta >= 0.0) || !std::isfinite(p->delta)) return false;
  return p->Q && p->M && p->R && p->q && p->r && p->A && p->B && p->c;
}

static BatchArgs single_args(const rlqr_problem *p, const rlqr_opts *o, void *ws) {
  BatchArgs a{};
  a.count = 1;
  a.single = 1;
  a.N = p->N;
  a.n = p->nx;
  a.m = p->nu;
  a.delta = p->delta;
  a.Q = p->Q; a.M = p->M; a.R = p->R; a.q = p->q; a.r = p->r; a.A = p->A; a.B = p->B; a.c = p->c;
  a.ws = static_cast<char *>(ws);
  a.tsize = (o && o->prec == RLQR_MIXED) ? 4 : 8;
  a.tol = o ? o->tol : 1e-9;
  a.max_refine = o ? o->max_refine : 0;
  return a;
}

static rlqr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA; }

// ---- algorithm selection for one instance
// The scan path has kernels for these sizes; it needs delta > 0 and every
// R_i invertible (the elimination of the controls).
static bool scan_sizes(int n, int m) {
  return (n == 4 && m == 2) || (n == 6 && m == 2) || (n == 12 && m == 4) || (n == 32 && m == 8);
}
constexpr int kScanAutoN = 4096;  // AUTO takes the scan from this horizon on

// Whether the workspace must hold the scan arrays (delta is not known here).
static bool scan_sized(int N, int n, int m, const rlqr_opts *o) {
  if (o->algo == RLQR_ALGO_SCAN) return true;
  return o->algo == RLQR_ALGO_AUTO && N >= kScanAutoN && scan_sizes(n, m);
}

// 1: scan, 0: sequential, -1: SCAN requested where it does not apply.
static int use_scan(const rlqr_problem *p, const rlqr_opts *o) {
  const bool ok = scan_sizes(p->nx, p->nu) && p->delta > 0.0;
  if (o->algo == RLQR_ALGO_SCAN) return ok ? 1 : -1;
  if (o->algo == RLQR_ALGO_AUTO) return (ok && p->N >= kScanAutoN) ? 1 : 0;
  return 0;
}

// ---- scan tiles: the chunk of stages one CTA folds.  Default: about 444
// chunks (three CTAs per SM on 148 SMs), at least 8 stages.  The autotuner
// (rlqr_autotune_scan) times chunk counts that are multiples of the SM count
// and records the fastest per (nx, nu, precision, floor(log2 N)); later
// factorizations of that shape use it.  Workspaces are sized for the largest
// candidate count, so every recorded choice fits.
constexpr int kScanChunkCandidates[] = {148, 296, 444, 592, 888};
constexpr int kScanChunkMax = 888;
std::mutex g_tune_mu;
std::map<uint64_t, int> g_scan_chunks;

static uint64_t tune_key(int N, int n, int m, int tsize) {
  int lg = 0;
  while (lg < 30 && (1 << (lg + 1)) <= N) ++lg;
  return ((uint64_t)n << 40) | ((uint64_t)m << 32) | ((uint64_t)tsize << 24) | (uint64_t)lg;
}

static int chunk_len_of_count(int N, int chunks) { return std::max(8, (N + chunks - 1) / chunks); }

static int scan_len_for(int N, int n, int m, int tsize) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const auto it = g_scan_chunks.find(tune_key(N, n, m, tsize));
  return it == g_scan_chunks.end() ? scan_chunk_len(N) : chunk_len_of_count(N, it->second);
}

static ScanLayout scan_args(const rlqr_problem *p, const rlqr_opts *o, size_t *sbase) {
  const int tsize = o->prec == RLQR_MIXED ? 4 : 8;
  *sbase = ws_layout(p->N, p->nx, p->nu, tsize).total;
  return scan_layout(p->N, p->nx, scan_len_for(p->N, p->nx, p->nu, tsize), tsize);
}

}  // namespace rlqr

using namespace rlqr;

extern "C" {

rlqr_opts rlqr_default_opts(void) {
  rlqr_opts o;
  o.max_refine = 3;
  o.tol = 1e-9;
  o.algo = RLQR_ALGO_AUTO;
  o.prec = RLQR_FP64;
  o.flags = 0;
  return o;
}

const char *rlqr_version(void) { return "rlqr-b300 0.1 (sm_103a)"; }

const char *rlqr_status_string(rlqr_status s) {
  switch (s) {
    case RLQR_OK: return "ok";
    case RLQR_NOT_PD: return "solved; a pivot is not positive-definite";
    case RLQR_ERR_ARG: return "invalid argument";
    case RLQR_ERR_SINGULAR: return "zero or non-finite pivot";
    case RLQR_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
    case RLQR_ERR_TIMEOUT: return "device wait timed out";
    case RLQR_ERR_WORKSPACE: return "workspace too small or misaligned";
    case RLQR_ERR_CUDA: return "CUDA error";
  }
  return "unknown status";
}

size_t rlqr_workspace_bytes(int32_t N, int32_t nx, int32_t nu, const rlqr_opts *opts) {
  if (!valid_dims(N, nx, nu) || !valid_opts(opts)) return 0;
  int tsize = opts->prec == RLQR_MIXED ? 4 : 8;
  size_t tot = ws_layout(N, nx, nu, tsize).total;
  if (scan_sized(N, nx, nu, opts))
    tot += scan_layout(N, nx, chunk_len_of_count(N, kScanChunkMax), tsize).total;
  return tot;
}

rlqr_status rlqr_factor(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                        size_t ws_bytes, uint8_t *pivot_pd, int32_t *status,
                        rlqr_stream_t stream) {
  if (!valid_problem(prob) || !valid_opts(opts) || !pivot_pd) return RLQR_ERR_ARG;
  size_t need = rlqr_workspace_bytes(prob->N, prob->nx, prob->nu, opts);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  BatchArgs a = single_args(prob, opts, ws);
  a.flags = pivot_pd;
  a.status = status;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = prob->nx, m = prob->nu;
  const int scan = use_scan(prob, opts);
  if (scan < 0) return RLQR_ERR_ARG;
  if (scan) {
    size_t sbase;
    const ScanLayout SL = scan_args(prob, opts, &sbase);
    const bool mixed = opts->prec == RLQR_MIXED;
    cudaError_t e = mixed ? launch_scan_factor<float>(n, m, a, SL, sbase, s)
                          : launch_scan_factor<double>(n, m, a, SL, sbase, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
    // mixed: FP64 certificate of the stored control pivots; status out
    e = mixed ? launch_scan_residual<float>(n, m, a, 1, 0, s)
              : launch_scan_residual<double>(n, m, a, 0, 0, s);
    if (e == cudaSuccess && mixed) e = launch_escalate(a, n, m, 0, 1, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
    return sync_status(opts, ws, false, mixed, s);
  }
  if (opts->prec == RLQR_MIXED) {
    cudaError_t e = launch_seq<float, false>(n, m, true, a, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
    // FP64 certificate of the control pivots stored by the FP32 sweep, then
    // the FP64 decision of whatever lacked its margin
    e = launch_residual(a, 2 * n + m, 0, nullptr, nullptr, 0, 0, s, 1, 0);
    if (e == cudaSuccess) e = launch_escalate(a, n, m, 0, 0, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
    return sync_status(opts, ws, false, true, s);
  }
  if (launch_seq<double, false>(n, m, true, a, s) != cudaSuccess) return RLQR_ERR_CUDA;
  return sync_status(opts, ws, false, false, s);
}

rlqr_status rlqr_solve(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                       size_t ws_bytes, double *x, double *u, double *y, double *rel_resid,
                       int32_t *iters, int32_t *status, rlqr_stream_t stream) {
  if (!valid_problem(prob) || !valid_opts(opts) || !x || !u || !y) return RLQR_ERR_ARG;
  size_t need = rlqr_workspace_bytes(prob->N, prob->nx, prob->nu, opts);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  BatchArgs a = single_args(prob, opts, ws);
  a.x = x;
  a.u = u;
  a.y = y;
  a.rel = rel_resid;
  a.iters = iters;
  a.status = status;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = prob->nx, m = prob->nu;
  const bool mixed = opts->prec == RLQR_MIXED;
  const int scan = use_scan(prob, opts);
  if (scan < 0) return RLQR_ERR_ARG;
  if (scan) {
    size_t sbase;
    const ScanLayout SL = scan_args(prob, opts, &sbase);
    cudaError_t e = mixed ? launch_scan_solve<float>(n, m, false, a, SL, sbase, s)
                          : launch_scan_solve<double>(n, m, false, a, SL, sbase, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
    const int with_res = (mixed || rel_resid) ? 1 : 0;
    e = mixed ? launch_scan_residual<float>(n, m, a, 0, with_res, s)
              : launch_scan_residual<double>(n, m, a, 0, with_res, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
    if (mixed)
      for (int it = 0; it < opts->max_refine; ++it) {
        e = launch_scan_solve<float>(n, m, true, a, SL, sbase, s);
        if (e == cudaSuccess) e = launch_scan_norms<float>(a, s);
        if (e != cudaSuccess) return RLQR_ERR_CUDA;
      }
    return sync_status(opts, ws, true, mixed, s);
  }
  cudaError_t e = mixed ? launch_solve<float, false>(n, m, true, a, s)
                        : launch_solve<double, false>(n, m, true, a, s);
  if (e != cudaSuccess) return RLQR_ERR_CUDA;
  if (mixed || rel_resid) {
    e = launch_first_residual(a, n, m, mixed, 0, nullptr, (int64_t)prob->N + 1, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
  }
  if (mixed)
    for (int it = 0; it < opts->max_refine; ++it) {
      a.rpass = it;
      e = launch_solve<float, true>(n, m, true, a, s);
      if (e == cudaSuccess) e = launch_recheck(a, n, m, nullptr, (int64_t)prob->N + 1, s);
      if (e != cudaSuccess) return RLQR_ERR_CUDA;
    }
  return sync_status(opts, ws, true, mixed, s);
}

rlqr_status rlqr_residual(const rlqr_problem *prob, const double *x, const double *u,
                          const double *y, double *res, double *norms, rlqr_stream_t stream) {
  if (!valid_problem(prob) || !x || !u || !y || !norms) return RLQR_ERR_ARG;
  BatchArgs a = single_args(prob, nullptr, nullptr);
  a.x = const_cast<double *>(x);
  a.u = const_cast<double *>(u);
  a.y = const_cast<double *>(y);
  a.tol = 1e-9;
  return cuda_status(launch_residual(a, 2 * prob->nx + prob->nu, 0, res, norms, 1, 1,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

size_t rlqr_batched_workspace_bytes(const rlqr_batch *batch, const rlqr_opts *opts) {
  if (!batch || batch->count < 1 || !batch->h_N || !batch->h_nx || !batch->h_nu ||
      !valid_opts(opts))
    return 0;
  int tsize = opts->prec == RLQR_MIXED ? 4 : 8;
  size_t tot = batch_header_bytes(batch->count);
  for (int b = 0; b < batch->count; ++b) {
    if (!valid_dims(batch->h_N[b], batch->h_nx[b], batch->h_nu[b])) return 0;
    tot += ws_layout(batch->h_N[b], batch->h_nx[b], batch->h_nu[b], tsize).total;
  }
  return tot;
}

rlqr_status rlqr_solve_batched(const rlqr_batch *batch, const rlqr_opts *opts, void *ws,
                               size_t ws_bytes, int32_t *status, double *rel_resid,
                               int32_t *iters, rlqr_stream_t stream) {
  if (!batch || batch->count < 1 || !valid_opts(opts)) return RLQR_ERR_ARG;
  if (opts->algo == RLQR_ALGO_SCAN) return RLQR_ERR_ARG;  // batches use the sequential recursion
  const rlqr_batch &B = *batch;
  if (!B.N || !B.nx || !B.nu || !B.delta || !B.off_Q || !B.off_M || !B.off_R || !B.off_q ||
      !B.off_r || !B.off_A || !B.off_B || !B.off_c || !B.off_x || !B.off_u || !B.off_y ||
      !B.off_flag || !B.Q || !B.M || !B.R || !B.q || !B.r || !B.A || !B.B || !B.c || !B.x ||
      !B.u || !B.y || !B.pivot_pd)
    return RLQR_ERR_ARG;
  size_t need = rlqr_batched_workspace_bytes(batch, opts);
  if (need == 0) return RLQR_ERR_ARG;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  int nmax = 0, mmax = 0, rs_max = 0;
  bool uniform = true;
  for (int b = 0; b < B.count; ++b) {
    nmax = std::max(nmax, B.h_nx[b]);
    mmax = std::max(mmax, B.h_nu[b]);
    rs_max = std::max(rs_max, 2 * B.h_nx[b] + B.h_nu[b]);
    uniform = uniform && B.h_nx[b] == B.h_nx[0] && B.h_nu[b] == B.h_nu[0];
  }
  const bool mixed = opts->prec == RLQR_MIXED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BatchArgs a{};
  a.count = B.count;
  a.single = 0;
  a.dN = B.N; a.dn = B.nx; a.dm = B.nu; a.ddelta = B.delta;
  a.oQ = B.off_Q; a.oM = B.off_M; a.oR = B.off_R; a.oq = B.off_q; a.or_ = B.off_r;
  a.oA = B.off_A; a.oB = B.off_B; a.oc = B.off_c; a.ox = B.off_x; a.ou = B.off_u;
  a.oy = B.off_y; a.of = B.off_flag;
  a.Q = B.Q; a.M = B.M; a.R = B.R; a.q = B.q; a.r = B.r; a.A = B.A; a.B = B.B; a.c = B.c;
  a.x = B.x; a.u = B.u; a.y = B.y; a.flags = B.pivot_pd;
  a.ws = static_cast<char *>(ws);
  a.ows = reinterpret_cast<const int64_t *>(ws);
  a.tsize = mixed ? 4 : 8;
  a.status = status;
  a.rel = rel_resid;
  a.iters = iters;
  a.tol = opts->tol;
  a.max_refine = opts->max_refine;
  cudaError_t e;
  {
    LaunchScope ls("k_plan", s);
    k_plan<<<1, 1024, 0, s>>>(B.count, B.N, B.nx, B.nu, a.tsize,
                              reinterpret_cast<int64_t *>(ws));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return RLQR_ERR_CUDA;
  // one launch sequence per size class (the whole batch when uniform)
  struct Group {
    int n, m, rs, count, off;
    bool exact;
  };
  Group groups[kNumClasses];
  int ng = 0;
  int sweep_route = 3;  // ragged batches: class streams (3) or the persistent sweep (4)
  RaggedPlan rplan{};
  if (uniform) {
    groups[ng++] = Group{nmax, mmax, rs_max, B.count, 0, true};
  } else {
    int cnt[kNumClasses] = {}, gn[kNumClasses] = {}, gm[kNumClasses] = {}, grs[kNumClasses] = {};
    int nmaxN = 1;
    for (int b = 0; b < B.count; ++b) {
      const int c = size_class(B.h_nx[b], B.h_nu[b]);
      ++cnt[c];
      gn[c] = std::max(gn[c], B.h_nx[b]);
      gm[c] = std::max(gm[c], B.h_nu[b]);
      grs[c] = std::max(grs[c], 2 * B.h_nx[b] + B.h_nu[b]);
      nmaxN = std::max(nmaxN, B.h_N[b]);
    }
    ClassOffsets co{};
    int acc = 0;
    for (int c = 0; c < kNumClasses; ++c) {
      co.off[c] = acc;
      if (cnt[c]) groups[ng++] = Group{gn[c], gm[c], grs[c], cnt[c], acc, c < kNumExact};
      acc += cnt[c];
    }
    int32_t *perm = reinterpret_cast<int32_t *>(static_cast<char *>(ws) +
                                                align_up((size_t)B.count * sizeof(int64_t)));
    {
      LaunchScope ls("k_group", s);
      k_group<<<1, 1024, 0, s>>>(B.count, B.N, B.nx, B.nu, (nmaxN + kNBuckets - 1) / kNBuckets,
                                 co, perm);
      if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
    }
    a.perm = perm;
    if (mixed) {
      bool covered = true;
      int mask = 0;
      for (int c = 0; c < kNumClasses; ++c) {
        if (!cnt[c]) continue;
        mask |= 1 << c;
        if (c >= kRaggedClasses || !ragged_kind(c)) {
          covered = false;
        } else {
          rplan.off[c] = co.off[c];
          rplan.cnt[c] = cnt[c];
        }
      }
      if (covered) sweep_route = ragged_route(mask, nmaxN, a.tsize, B.count);
    }
  }
  auto group_args = [&](int g) {
    BatchArgs ag = a;
    ag.count = groups[g].count;
    ag.goff = groups[g].off;
    return ag;
  };
  // several classes: each on its own stream, concurrently
  std::unique_lock<std::mutex> lock(g_class_mu, std::defer_lock);
  ClassStreams *cs = nullptr;
  if (ng > 1) {
    lock.lock();
    cs = class_streams_locked();
  }
  auto gstream = [&](int g) { return cs ? cs->st[g] : s; };
  bool esc_pending = false;  // k_escalate running on cs->esc
  auto fork = [&]() -> bool {
    if (!cs) return true;
    if (cudaEventRecord(cs->fork, s) != cudaSuccess) return false;
    for (int g = 0; g < ng; ++g)
      if (cudaStreamWaitEvent(cs->st[g], cs->fork, 0) != cudaSuccess) return false;
    return true;
  };
  auto join = [&]() -> bool {
    if (!cs) return true;
    for (int g = 0; g < ng; ++g)
      if (cudaEventRecord(cs->join[g], cs->st[g]) != cudaSuccess ||
          cudaStreamWaitEvent(s, cs->join[g], 0) != cudaSuccess)
        return false;
    return true;
  };
  if (sweep_route == 4) {
    // one persistent launch for every class's sweep, then the CTA classes'
    // deferred certificates
    char *hdr = static_cast<char *>(ws) + batch_header_items(B.count);
    int4 *items = reinterpret_cast<int4 *>(hdr);
    int32_t *meta = reinterpret_cast<int32_t *>(hdr + align_up((size_t)B.count * sizeof(int4)));
    e = launch_ragged_sweep(a, rplan, a.perm, items, meta, s);
    for (int g = 0; g < ng && e == cudaSuccess; ++g)
      e = launch_seq_cert(groups[g].n, groups[g].m, group_args(g), s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
  } else {
    if (!fork()) return RLQR_ERR_CUDA;
    for (int g = 0; g < ng; ++g) {
      const Group &G = groups[g];
      const BatchArgs ag = group_args(g);
      e = mixed ? launch_seq<float, true>(G.n, G.m, G.exact, ag, gstream(g))
                : launch_seq<double, true>(G.n, G.m, G.exact, ag, gstream(g));
      if (e != cudaSuccess) return RLQR_ERR_CUDA;
    }
    if (!join()) return RLQR_ERR_CUDA;
  }
  if (mixed || rel_resid) {
    // uniform: the group's first residual; ragged: one stage-parallel
    // residual over every instance
    const int64_t *spre = reinterpret_cast<const int64_t *>(
        static_cast<char *>(ws) + align_up((size_t)B.count * sizeof(int64_t)) +
        align_up((size_t)B.count * sizeof(int32_t)));
    int64_t items = 0;
    int nmaxN = 1;
    for (int b = 0; b < B.count; ++b) {
      items += (int64_t)B.h_N[b] + 1;
      nmaxN = std::max(nmaxN, B.h_N[b]);
    }
    const int route = uniform ? residual_route(nmaxN, nmax, mmax, a.tsize, B.count) : 0;
    if (route == 6 || route == 7) a.refine_warps = 2;
    else if (route != 0) a.refine_warps = 1;
    if (mixed && uniform && (route == 5 || route == 7) && opts->max_refine > 0 &&
        warp_res32_size(nmax, mmax)) {
      // fused route: the control-pivot certificate alone here; the first
      // refinement pass computes the residual as it goes
      a.fused_res = 1;
      e = launch_cert_g(a, spre, items, s);
    } else {
      e = uniform ? launch_first_residual(a, nmax, mmax, mixed, 1, spre, items, s, route)
                  : launch_grid_residual(a, spre, items, mixed, 1, s);
    }
    if (e == cudaSuccess && mixed) {
      if (cs && opts->max_refine > 0) {
        // the FP64 re-decision changes only flags and pivot status, which
        // the refinement does not read: it runs beside the refinement
        // passes on its own stream (joined, with the status of the
        // escalated instances, after the last pass)
        if (cudaEventRecord(cs->esc_fork, s) != cudaSuccess ||
            cudaStreamWaitEvent(cs->esc, cs->esc_fork, 0) != cudaSuccess)
          return RLQR_ERR_CUDA;
        e = launch_escalate(a, nmax, mmax, 2, 0, cs->esc);
        if (e == cudaSuccess && cudaEventRecord(cs->esc_join, cs->esc) != cudaSuccess)
          e = cudaErrorUnknown;
        esc_pending = true;
      } else {
        e = launch_escalate(a, nmax, mmax, 1, 0, s);
      }
    }
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
  }
  if (mixed) {
    const int64_t *spre = reinterpret_cast<const int64_t *>(
        static_cast<char *>(ws) + align_up((size_t)B.count * sizeof(int64_t)) +
        align_up((size_t)B.count * sizeof(int32_t)));
    int64_t items = 0;
    int nmaxN = 1;
    for (int b = 0; b < B.count; ++b) {
      items += (int64_t)B.h_N[b] + 1;
      nmaxN = std::max(nmaxN, B.h_N[b]);
    }
    const int route = uniform ? residual_route(nmaxN, nmax, mmax, a.tsize, B.count) : 0;
    for (int it = 0; it < opts->max_refine; ++it) {
      if (!fork()) return RLQR_ERR_CUDA;
      for (int g = 0; g < ng; ++g) {
        const Group &G = groups[g];
        BatchArgs ag = group_args(g);
        ag.rpass = it;
        e = launch_solve<float, true>(G.n, G.m, G.exact, ag, gstream(g));
        if (e != cudaSuccess) return RLQR_ERR_CUDA;
      }
      if (!join()) return RLQR_ERR_CUDA;
      e = launch_recheck(a, nmax, mmax, spre, items, s, route, uniform);
      if (e != cudaSuccess) return RLQR_ERR_CUDA;
    }
  }
  if (esc_pending) {
    if (cudaStreamWaitEvent(s, cs->esc_join, 0) != cudaSuccess) return RLQR_ERR_CUDA;
    LaunchScope ls("k_escalate", s);
    k_escalate_status<<<(B.count + 255) / 256, 256, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  }
  return RLQR_OK;
}

// ---- allocation-free entry point
// The scratch of rlqr_solve_noalloc: a file-scope device array, so that the
// call itself never allocates.  Host code only sees a host-side stand-in for
// the symbol; the device address comes from cudaGetSymbolAddress, taken once
// per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RLQR_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

rlqr_status rlqr_solve_noalloc(const rlqr_problem *prob, const rlqr_opts *opts, double *x,
                               double *u, double *y, uint8_t *pivot_pd, double *rel_resid,
                               int32_t *status, rlqr_stream_t stream) {
  if (!valid_problem(prob) || !valid_opts(opts) || !x || !u || !y || !pivot_pd)
    return RLQR_ERR_ARG;
  if (opts->algo == RLQR_ALGO_SCAN) return RLQR_ERR_ARG;  // sequential recursion only
  const size_t need = ws_layout(prob->N, prob->nx, prob->nu,
                                opts->prec == RLQR_MIXED ? 4 : 8).total;
  if (need > RLQR_NOALLOC_SCRATCH_BYTES) return RLQR_ERR_WORKSPACE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RLQR_ERR_CUDA;
  void *ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RLQR_ERR_CUDA;
      g_noalloc_ptr[dev] = p;
    }
    ws = g_noalloc_ptr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the per-instance state at the start of the scratch starts from zero
  if (cudaMemsetAsync(ws, 0, sizeof(InstState), s) != cudaSuccess) return RLQR_ERR_CUDA;
  BatchArgs a = single_args(prob, opts, ws);
  a.x = x;
  a.u = u;
  a.y = y;
  a.flags = pivot_pd;
  a.status = status;
  a.rel = rel_resid;
  const bool mixed = opts->prec == RLQR_MIXED;
  const int n = prob->nx, m = prob->nu;
  cudaError_t e = mixed ? launch_seq<float, true>(n, m, true, a, s)
                        : launch_seq<double, true>(n, m, true, a, s);
  if (e != cudaSuccess) return RLQR_ERR_CUDA;
  if (mixed || rel_resid) {
    e = launch_first_residual(a, n, m, mixed, 1, nullptr, (int64_t)prob->N + 1, s);
    if (e == cudaSuccess && mixed) e = launch_escalate(a, n, m, 1, 0, s);
    if (e != cudaSuccess) return RLQR_ERR_CUDA;
  }
  if (mixed)
    for (int it = 0; it < opts->max_refine; ++it) {
      a.rpass = it;
      e = launch_solve<float, true>(n, m, true, a, s);
      if (e == cudaSuccess) e = launch_recheck(a, n, m, nullptr, (int64_t)prob->N + 1, s);
      if (e != cudaSuccess) return RLQR_ERR_CUDA;
    }
  return sync_status(opts, ws, true, mixed, s);
}

// ---- horizon shards of one long instance
static bool shard_ok(const rlqr_problem *p, const rlqr_opts *o) {
  return valid_problem(p) && valid_opts(o) && o->prec == RLQR_FP64 &&
         o->algo == RLQR_ALGO_SCAN && scan_sizes(p->nx, p->nu) && p->delta > 0.0;
}

rlqr_status rlqr_shard_element(const rlqr_problem *shard, const rlqr_opts *opts, void *ws,
                               size_t ws_bytes, double *elem, rlqr_stream_t stream) {
  if (!shard_ok(shard, opts) || !elem) return RLQR_ERR_ARG;
  const size_t need = rlqr_workspace_bytes(shard->N, shard->nx, shard->nu, opts);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  size_t sbase;
  const ScanLayout SL = scan_args(shard, opts, &sbase);
  const BatchArgs a = single_args(shard, opts, ws);
  return cuda_status(launch_shard_element(shard->nx, shard->nu, a, SL, sbase, elem,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

rlqr_status rlqr_shard_boundary(int32_t G, int32_t g, int32_t nx, int32_t nu,
                                const double *elems, const double *QN, double *P_end,
                                double *P_start, rlqr_stream_t stream) {
  if (G < 1 || g < 0 || g >= G || !scan_sizes(nx, nu) || !elems || !QN || !P_end)
    return RLQR_ERR_ARG;
  return cuda_status(launch_shard_boundary(nx, nu, G, g, elems, QN, P_end, P_start,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

rlqr_status rlqr_shard_pmap(const rlqr_problem *shard, const rlqr_opts *opts, const void *ws,
                            size_t ws_bytes, double *Phi, double *phi, rlqr_stream_t stream) {
  if (!shard_ok(shard, opts) || !Phi || !phi) return RLQR_ERR_ARG;
  const size_t need = rlqr_workspace_bytes(shard->N, shard->nx, shard->nu, opts);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  size_t sbase;
  const ScanLayout SL = scan_args(shard, opts, &sbase);
  const BatchArgs a = single_args(shard, opts, const_cast<void *>(ws));
  return cuda_status(launch_shard_pmap(shard->nx, shard->nu, a, SL, sbase, Phi, phi,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

rlqr_status rlqr_shard_p_end(int32_t G, int32_t g, int32_t nx, const double *Phis,
                             const double *phis, const double *qN, double *p_end,
                             rlqr_stream_t stream) {
  if (G < 1 || g < 0 || g >= G || nx < 1 || nx > 64 || !Phis || !phis || !qN || !p_end)
    return RLQR_ERR_ARG;
  return cuda_status(launch_shard_p_end(G, g, nx, Phis, phis, qN, p_end,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

rlqr_status rlqr_shard_x_offset(int32_t nx, const double *Phi, const double *x_first,
                                const double *x_last, double *psi, rlqr_stream_t stream) {
  if (nx < 1 || nx > 64 || !Phi || !x_first || !x_last || !psi) return RLQR_ERR_ARG;
  return cuda_status(launch_shard_x_offset(nx, Phi, x_first, x_last, psi,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

rlqr_status rlqr_shard_x_start(int32_t g, int32_t nx, const double *Phis, const double *psis,
                               double *x_start, rlqr_stream_t stream) {
  if (g < 1 || nx < 1 || nx > 64 || !Phis || !psis || !x_start) return RLQR_ERR_ARG;
  return cuda_status(launch_shard_x_start(g, nx, Phis, psis, x_start,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

rlqr_status rlqr_shard_entry(int32_t nx, double delta, const double *P_start,
                             const double *x_start, const double *x_first, double *c0,
                             rlqr_stream_t stream) {
  if (nx < 1 || nx > 64 || !(delta >= 0.0) || !P_start || !x_start || !x_first || !c0)
    return RLQR_ERR_ARG;
  return cuda_status(launch_shard_entry(nx, delta, P_start, x_start, x_first, c0,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

// ---- cross-stage variables (Section "Cross-Stage Variables")
// Scratch: V and z_b (p + 1 columns of length L), the dot-product partials,
// p + 2 status slots (the p + 1 solves, then the combined status), and one
// copy of the factored workspace per solve, so that the p + 1 solves run
// concurrently on their own streams.
static size_t cross_len(int N, int n, int m) { return (size_t)(N + 1) * n * 2 + (size_t)N * m; }

struct CrossScratch {
  size_t V, part, st, ws, ws_each, total;
};

static CrossScratch cross_scratch(int N, int n, int m, int p, const rlqr_opts *o) {
  CrossScratch c{};
  const size_t L = cross_len(N, n, m);
  c.ws_each = align_up(rlqr_workspace_bytes(N, n, m, o));
  size_t off = 0;
  c.V = off;
  off += align_up((size_t)(p + 1) * L * sizeof(double));
  c.part = off;
  off += align_up((size_t)kCrossBlocks * p * (p + 1) * sizeof(double));
  c.st = off;
  off += align_up((size_t)(p + 2) * sizeof(int32_t));
  c.ws = off;
  off += (size_t)(p + 1) * c.ws_each;
  c.total = off;
  return c;
}

// Streams of the concurrent solves (per device, created once, like the
// size-class streams).
struct CrossStreams {
  bool ok = false;
  cudaStream_t st[kCrossMaxP + 1];
  cudaEvent_t fork, join[kCrossMaxP + 1];
};
static CrossStreams g_cross_streams[kMaxClassDevices];
static std::mutex g_cross_mu;

static CrossStreams *cross_streams_locked() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxClassDevices) return nullptr;
  CrossStreams &cs = g_cross_streams[dev];
  if (!cs.ok) {
    for (int j = 0; j <= kCrossMaxP; ++j)
      if (cudaStreamCreateWithFlags(&cs.st[j], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&cs.join[j], cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    if (cudaEventCreateWithFlags(&cs.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    cs.ok = true;
  }
  return &cs;
}

size_t rlqr_cross_scratch_bytes(int32_t N, int32_t nx, int32_t nu, int32_t p,
                                const rlqr_opts *opts) {
  if (!valid_dims(N, nx, nu) || p < 1 || p > kCrossMaxP || !valid_opts(opts)) return 0;
  return cross_scratch(N, nx, nu, p, opts).total;
}

rlqr_status rlqr_solve_cross(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                             size_t ws_bytes, int32_t p, const double *J, const double *H,
                             const double *r_theta, void *scratch, size_t scratch_bytes,
                             double *x, double *u, double *y, double *dtheta, int32_t *status,
                             rlqr_stream_t stream) {
  if (!valid_problem(prob) || !valid_opts(opts) || p < 1 || p > kCrossMaxP || !J || !H ||
      !r_theta || !x || !u || !y || !dtheta)
    return RLQR_ERR_ARG;
  const int N = prob->N, n = prob->nx, m = prob->nu;
  const CrossScratch C = cross_scratch(N, n, m, p, opts);
  const size_t need = rlqr_workspace_bytes(N, n, m, opts);
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  if (!scratch || scratch_bytes < C.total || (reinterpret_cast<uintptr_t>(scratch) % kAlign) != 0)
    return RLQR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t L = cross_len(N, n, m);
  const int64_t nX = (int64_t)(N + 1) * n, nU = (int64_t)N * m;
  char *sc = static_cast<char *>(scratch);
  double *V = reinterpret_cast<double *>(sc + C.V);  // columns 0..p-1: V, column p: z_b
  double *part = reinterpret_cast<double *>(sc + C.part);
  int32_t *sst = reinterpret_cast<int32_t *>(sc + C.st);
  rlqr_opts o = *opts;
  o.flags &= ~RLQR_OPT_SYNC;  // the inner solves stay stream-ordered
  // status slots start at RLQR_OK (a solve that takes no decision leaves its
  // slot alone; the factor's pivot status comes from the instance state);
  // every solve gets its own copy of the factored workspace
  if (cudaMemsetAsync(sst, 0, (size_t)(p + 2) * sizeof(int32_t), s) != cudaSuccess)
    return RLQR_ERR_CUDA;
  for (int j = 0; j <= p; ++j)
    if (cudaMemcpyAsync(sc + C.ws + (size_t)j * C.ws_each, ws, need, cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
      return RLQR_ERR_CUDA;
  std::unique_lock<std::mutex> lock(g_cross_mu);
  CrossStreams *cs = cross_streams_locked();
  auto tstream = [&](int j) { return cs ? cs->st[j] : s; };
  if (cs) {
    if (cudaEventRecord(cs->fork, s) != cudaSuccess) return RLQR_ERR_CUDA;
    for (int j = 0; j <= p; ++j)
      if (cudaStreamWaitEvent(cs->st[j], cs->fork, 0) != cudaSuccess) return RLQR_ERR_CUDA;
  }
  // column j < p: V_j = -K^{-1} J_j; column p: z_b = -K^{-1} b
  for (int j = 0; j <= p; ++j) {
    rlqr_problem pj = *prob;
    if (j < p) {
      pj.q = J + (size_t)j * L;
      pj.r = pj.q + nX;
      pj.c = pj.r + nU;
    }
    double *xj = V + (size_t)j * L;
    const rlqr_status st =
        rlqr_solve(&pj, &o, sc + C.ws + (size_t)j * C.ws_each, C.ws_each, xj, xj + nX,
                   xj + nX + nU, nullptr, nullptr, sst + j,
                   reinterpret_cast<rlqr_stream_t>(tstream(j)));
    if (st != RLQR_OK) return st;
  }
  if (cs) {
    for (int j = 0; j <= p; ++j)
      if (cudaEventRecord(cs->join[j], cs->st[j]) != cudaSuccess ||
          cudaStreamWaitEvent(s, cs->join[j], 0) != cudaSuccess)
        return RLQR_ERR_CUDA;
  }
  lock.unlock();
  {
    const double *zb = V + (size_t)p * L;
    LaunchScope ls("k_cross", s);
    k_cross_dots<<<kCrossBlocks, 256, 0, s>>>(p, (int64_t)L, nX, nU, J, V, zb, zb + nX,
                                             zb + nX + nU, part);
    k_cross_theta<<<1, 1024, 0, s>>>(p, kCrossBlocks, H, r_theta, part,
                                     reinterpret_cast<const InstState *>(ws), sst, dtheta,
                                     sst + p + 1);
    k_cross_combine<<<(int)std::min<size_t>((L + 255) / 256, 148 * 8), 256, 0, s>>>(
        p, (int64_t)L, nX, nU, V, dtheta, x, u, y);
    if (status && cudaMemcpyAsync(status, sst + p + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  s) != cudaSuccess)
      return RLQR_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return RLQR_ERR_CUDA;
  }
  if (opts->flags & RLQR_OPT_SYNC) {
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, sst + p + 1, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return RLQR_ERR_CUDA;
    return static_cast<rlqr_status>(h);
  }
  return RLQR_OK;
}

rlqr_status rlqr_instrument(int enable) {
  g_instr.on = enable != 0;
  g_instr.n = 0;
  return RLQR_OK;
}

int rlqr_instrument_report(int max, const char **names, int64_t *launches, double *ms) {
  const int timed = std::min(g_instr.n, Instr::kMax);
  int k = 0;
  for (int i = 0; i < timed; ++i) {
    if (cudaEventSynchronize(g_instr.ev[2 * i + 1]) != cudaSuccess) return -1;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_instr.ev[2 * i], g_instr.ev[2 * i + 1]) != cudaSuccess)
      return -1;
    int j = 0;
    while (j < k && std::strcmp(names[j], g_instr.name[i]) != 0) ++j;
    if (j == k) {
      if (k >= max) continue;
      names[k] = g_instr.name[i];
      launches[k] = 0;
      ms[k] = 0.0;
      ++k;
    }
    launches[j] += 1;
    ms[j] += t;
  }
  return k;
}

}  // extern "C"

// ---- scan tile autotuning
extern "C" {

rlqr_status rlqr_tune_scan_set(int32_t N, int32_t nx, int32_t nu, const rlqr_opts *opts,
                               int32_t chunks) {
  if (!valid_dims(N, nx, nu) || !valid_opts(opts)) return RLQR_ERR_ARG;
  if (chunks != 0 && (chunks < 1 || chunks > kScanChunkMax)) return RLQR_ERR_ARG;
  const int tsize = opts->prec == RLQR_MIXED ? 4 : 8;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (chunks == 0)
    g_scan_chunks.erase(tune_key(N, nx, nu, tsize));
  else
    g_scan_chunks[tune_key(N, nx, nu, tsize)] = chunks;
  return RLQR_OK;
}

rlqr_status rlqr_tune_reset(void) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_scan_chunks.clear();
  }
  std::lock_guard<std::mutex> lock(g_route_mu);
  g_res_route.clear();
  return RLQR_OK;
}

// The tuning key of a batch and whether it is ragged: a uniform batch of a
// warp-residual size (residual routes 1, 2) or a ragged mixed-precision
// batch whose classes the persistent sweep covers (sweep routes 3, 4).
static bool batch_tune_key(const rlqr_batch *batch, const rlqr_opts *opts, uint64_t *key,
                           bool *ragged) {
  if (!batch || batch->count < 1 || !batch->h_N || !batch->h_nx || !batch->h_nu ||
      !valid_opts(opts))
    return false;
  int nmaxN = 1, mask = 0;
  bool uniform = true;
  for (int b = 0; b < batch->count; ++b) {
    if (batch->h_nx[b] != batch->h_nx[0] || batch->h_nu[b] != batch->h_nu[0]) uniform = false;
    nmaxN = std::max(nmaxN, batch->h_N[b]);
    mask |= 1 << size_class(batch->h_nx[b], batch->h_nu[b]);
  }
  const int tsize = opts->prec == RLQR_MIXED ? 4 : 8;
  if (uniform) {
    if (!warp_res32_size(batch->h_nx[0], batch->h_nu[0])) return false;
    *key = route_key(nmaxN, batch->h_nx[0], batch->h_nu[0], tsize, batch->count);
    *ragged = false;
    return true;
  }
  if (tsize != 4) return false;
  for (int c = 0; c < kNumClasses; ++c)
    if ((mask >> c & 1) && (c >= kRaggedClasses || !ragged_kind(c))) return false;
  *key = ragged_key(mask, nmaxN, tsize, batch->count);
  *ragged = true;
  return true;
}

rlqr_status rlqr_tune_batched_set(const rlqr_batch *batch, const rlqr_opts *opts, int32_t route) {
  uint64_t key;
  bool ragged = false;
  if (!batch_tune_key(batch, opts, &key, &ragged) || route < 0) return RLQR_ERR_ARG;
  if (route != 0 && (ragged ? (route < 3 || route > 4)
                            : !(route == 1 || route == 2 ||
                                (route >= 5 && route <= 7 && opts->prec == RLQR_MIXED))))
    return RLQR_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_route_mu);
  if (route == 0)
    g_res_route.erase(key);
  else
    g_res_route[key] = route;
  return RLQR_OK;
}

rlqr_status rlqr_autotune_batched(const rlqr_batch *batch, const rlqr_opts *opts, void *ws,
                                  size_t ws_bytes, int32_t *status, int32_t *best_route,
                                  double *best_ms, rlqr_stream_t stream) {
  uint64_t key;
  bool ragged = false;
  if (!batch_tune_key(batch, opts, &key, &ragged)) return RLQR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rlqr_opts o = *opts;
  o.flags = 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RLQR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RLQR_ERR_CUDA;
  }
  rlqr_status err = RLQR_OK;
  int best = 0;
  float best_t = 0.0f;
  const int reps = 3;
  int cand[5], nc = 0;
  if (ragged) {
    cand[nc++] = 3;
    cand[nc++] = 4;
  } else {
    cand[nc++] = 1;
    cand[nc++] = 2;
    if (opts->prec == RLQR_MIXED && opts->max_refine > 0) {
      cand[nc++] = 5;
      cand[nc++] = 6;
      cand[nc++] = 7;
    }
  }
  for (int ci = 0; ci < nc && err == RLQR_OK; ++ci) {
    const int route = cand[ci];
    err = rlqr_tune_batched_set(batch, opts, route);
    float t = 0.0f;
    for (int r = 0; r <= reps && err == RLQR_OK; ++r) {  // r = 0: warm-up
      if (r == 1 && cudaEventRecord(e0, s) != cudaSuccess) err = RLQR_ERR_CUDA;
      if (err == RLQR_OK)
        err = rlqr_solve_batched(batch, &o, ws, ws_bytes, status, nullptr, nullptr, stream);
    }
    if (err != RLQR_OK) break;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      err = RLQR_ERR_CUDA;
      break;
    }
    t /= reps;
    if (best == 0 || t < best_t) {
      best = route;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != RLQR_OK) {
    rlqr_tune_batched_set(batch, opts, 0);
    return err;
  }
  rlqr_tune_batched_set(batch, opts, best);
  if (best_route) *best_route = best;
  if (best_ms) *best_ms = best_t;
  return RLQR_OK;
}

rlqr_status rlqr_autotune_scan(const rlqr_problem *prob, const rlqr_opts *opts, void *ws,
                               size_t ws_bytes, double *x, double *u, double *y,
                               uint8_t *pivot_pd, int32_t *best_chunks, double *best_ms,
                               rlqr_stream_t stream) {
  if (!valid_problem(prob) || !valid_opts(opts) || !x || !u || !y || !pivot_pd)
    return RLQR_ERR_ARG;
  if (use_scan(prob, opts) != 1) return RLQR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rlqr_opts o = *opts;
  o.flags = 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RLQR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RLQR_ERR_CUDA;
  }
  rlqr_status err = RLQR_OK;
  int best = 0;
  float best_t = 0.0f;
  const int reps = 3;
  for (int c : kScanChunkCandidates) {
    err = rlqr_tune_scan_set(prob->N, prob->nx, prob->nu, opts, c);
    if (err != RLQR_OK) break;
    float t = 0.0f;
    for (int r = 0; r <= reps && err == RLQR_OK; ++r) {  // r = 0: warm-up
      if (r == 1 && cudaEventRecord(e0, s) != cudaSuccess) err = RLQR_ERR_CUDA;
      if (err == RLQR_OK) err = rlqr_factor(prob, &o, ws, ws_bytes, pivot_pd, nullptr, stream);
      if (err == RLQR_OK)
        err = rlqr_solve(prob, &o, ws, ws_bytes, x, u, y, nullptr, nullptr, nullptr, stream);
    }
    if (err != RLQR_OK) break;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      err = RLQR_ERR_CUDA;
      break;
    }
    t /= reps;
    if (best == 0 || t < best_t) {
      best = c;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != RLQR_OK) {
    rlqr_tune_scan_set(prob->N, prob->nx, prob->nu, opts, 0);
    return err;
  }
  rlqr_tune_scan_set(prob->N, prob->nx, prob->nu, opts, best);
  if (best_chunks) *best_chunks = best;
  if (best_ms) *best_ms = best_t;
  return RLQR_OK;
}

}  // extern "C"
