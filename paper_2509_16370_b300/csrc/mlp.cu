// mlp.cu -- the warm-start network of the nonlinear IPM (include/rlqr_mlp.h):
// BF16 x BF16 -> FP32 tensor-core GEMMs (one warp per 16 x 16 output tile,
// WMMA fragments: these layers are a few hundred rows by 256 columns, so the
// time is launch latency, not tensor throughput), the bias / ReLU / BF16
// epilogues, the loss gradient, column sums for the bias gradients and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <cstdint>
#include <type_traits>

#include "../../include/rlqr.h"
#include "../../include/rlqr_mlp.h"

namespace rlqr {
namespace mlp {

using bf16 = __nv_bfloat16;
namespace wm = nvcuda::wmma;

struct Off {
  size_t W1, b1, W2, b2, W3, b3, total;
  int npad;
};

inline Off offsets(const rlqr_mlp_dims &d) {
  Off o{};
  o.npad = (d.n_out + 15) / 16 * 16;
  const size_t W = d.width;
  o.W1 = 0;
  o.b1 = o.W1 + W * 16;
  o.W2 = o.b1 + W;
  o.b2 = o.W2 + W * W;
  o.W3 = o.b2 + W;
  o.b3 = o.W3 + (size_t)o.npad * W;
  o.total = o.b3 + o.npad;
  return o;
}

inline bool valid(const rlqr_mlp_dims *d) {
  return d && d->n_in >= 1 && d->n_in <= 16 && d->width >= 16 && d->width <= 1024 &&
         d->width % 16 == 0 && d->n_out >= 1 && d->n_out <= (1 << 20) && d->max_rows >= 16 &&
         d->max_rows % 16 == 0;
}

inline size_t up(size_t v) { return (v + 255) / 256 * 256; }

struct Ws {
  size_t a0, h1, h2, c, y, dy, dz2, dz1, dh, part, total;
};

inline Ws ws_layout(const rlqr_mlp_dims &d) {
  const Off o = offsets(d);
  const size_t R = d.max_rows, W = d.width, P = o.npad;
  Ws w{};
  size_t at = 0;
  auto take = [&](size_t b) {
    const size_t r = at;
    at = up(at + b);
    return r;
  };
  w.a0 = take(R * 16 * 2);
  w.h1 = take(R * W * 2);
  w.h2 = take(R * W * 2);
  w.c = take(R * W * 4);
  w.y = take(R * P * 4);
  w.dy = take(R * P * 2);
  w.dz2 = take(R * W * 2);
  w.dz1 = take(R * W * 2);
  w.dh = take(R * W * 4);
  w.part = take((R + 1) * 4);
  w.total = at;
  return w;
}

// C[M][N] (FP32, row-major, ldc = N) = sum_k A(m, k) B(k, n) with
//   A(m, k) = AT ? A[k lda + m] : A[m lda + k],
//   B(k, n) = BT ? B[n ldb + k] : B[k ldb + n];  M, N, K multiples of 16.
template <bool AT, bool BT>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16 *A, int lda,
                                              const bf16 *B, int ldb, float *C) {
  using LA = typename std::conditional<AT, wm::col_major, wm::row_major>::type;
  using LB = typename std::conditional<BT, wm::col_major, wm::row_major>::type;
  const int tile = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int tn = N / 16;
  if (tile >= (M / 16) * tn) return;
  const int m0 = (tile / tn) * 16, n0 = (tile % tn) * 16;
  wm::fragment<wm::matrix_a, 16, 16, 16, bf16, LA> fa;
  wm::fragment<wm::matrix_b, 16, 16, 16, bf16, LB> fb;
  wm::fragment<wm::accumulator, 16, 16, 16, float> acc;
  wm::fill_fragment(acc, 0.0f);
  for (int k0 = 0; k0 < K; k0 += 16) {
    wm::load_matrix_sync(fa, AT ? A + (size_t)k0 * lda + m0 : A + (size_t)m0 * lda + k0, lda);
    wm::load_matrix_sync(fb, BT ? B + (size_t)n0 * ldb + k0 : B + (size_t)k0 * ldb + n0, ldb);
    wm::mma_sync(acc, fa, fb, acc);
  }
  wm::store_matrix_sync(C + (size_t)m0 * N + n0, acc, N, wm::mem_row_major);
}

// Row indices of a batch: idx, advanced by *counter batches when counter is
// given (a graph-replayed training step reads its batch on the device).
__device__ __forceinline__ const int32_t *batch_rows(const int32_t *idx, const int32_t *counter,
                                                     int rows) {
  return (idx && counter) ? idx + (size_t)(*counter) * rows : idx;
}

__global__ void k_input(const float *x, const int32_t *idx0, const int32_t *counter, int rows,
                        int n_in, bf16 *a0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * 16) return;
  const int r = e >> 4, c = e & 15;
  const int32_t *idx = batch_rows(idx0, counter, rows);
  const int64_t src = idx ? idx[r] : r;
  a0[e] = __float2bfloat16_rn(c < n_in ? x[src * n_in + c] : 0.0f);
}

__global__ void k_bias_relu(const float *C, const bf16 *b, int rows, int W, bf16 *h) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * W) return;
  h[e] = __float2bfloat16_rn(fmaxf(0.0f, C[e] + __bfloat162float(b[e % W])));
}

__global__ void k_bias_out(const float *C, const bf16 *b, int rows, int npad, int n_out,
                           float *y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * n_out) return;
  const int r = e / n_out, c = e - r * n_out;
  y[e] = C[(size_t)r * npad + c] + __bfloat162float(b[c]);
}

// dy = bf16(2 (y - t) / (rows n_out)) on the real columns (0 on the padding),
// per-row partial sums of (y - t)^2 (one block per row).
__global__ void __launch_bounds__(256) k_loss_grad(const float *C, const bf16 *b, const float *t,
                                                   const int32_t *idx0, const int32_t *counter,
                                                   int rows, int npad, int n_out, bf16 *dy,
                                                   float *part) {
  __shared__ float sh[8];
  const int r = blockIdx.x;
  const int32_t *idx = batch_rows(idx0, counter, rows);
  const float scale = 2.0f / ((float)rows * (float)n_out);
  float acc = 0.0f;
  for (int c = threadIdx.x; c < npad; c += blockDim.x) {
    float g = 0.0f;
    if (c < n_out) {
      const int64_t src = idx ? idx[r] : r;
      const float d = C[(size_t)r * npad + c] + __bfloat162float(b[c]) - t[src * n_out + c];
      acc += d * d;
      g = scale * d;
    }
    dy[(size_t)r * npad + c] = __float2bfloat16_rn(g);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int i = 0; i < 8; ++i) s += sh[i];
    part[blockIdx.x] = s;
  }
}

// Sum of the per-row partials by one warp in a fixed order (deterministic).
__global__ void k_loss_final(const float *part, int nblk, int rows, int n_out, float *loss) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 32) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *loss = (float)(s / ((double)rows * (double)n_out));
}

__global__ void k_relu_back(const float *dh, const bf16 *h, int n, bf16 *dz) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  dz[e] = __float2bfloat16_rn(__bfloat162float(h[e]) > 0.0f ? dh[e] : 0.0f);
}

// out[c] = sum_r src[r][c] (FP32): block (32, 8) per 32 columns, thread
// (c, j) sums rows j, j + 8, ... (coalesced across c), then the 8 partial
// sums in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_colsum(const bf16 *src, int rows, int cols, float *out) {
  __shared__ float sh[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.0f;
  if (c < cols)
    for (int r = threadIdx.y; r < rows; r += 8) s += __bfloat162float(src[(size_t)r * cols + c]);
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    float t = 0.0f;
    for (int j = 0; j < 8; ++j) t += sh[j][threadIdx.x];
    out[c] = t;
  }
}

__global__ void k_to_bf16(const float *p, size_t n, bf16 *q) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < n) q[e] = __float2bfloat16_rn(p[e]);
}

// Adam; with sched / counter given, lr, c1, c2 = sched[3 s .. 3 s + 2] for
// s = *counter instead of the arguments.
__global__ void k_adam(float *p, bf16 *q, float *m, float *v, const float *g, size_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2, const float *sched,
                       const int32_t *counter) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (sched) {
    const float *sc = sched + 3 * (size_t)(*counter);
    lr = sc[0];
    c1 = sc[1];
    c2 = sc[2];
  }
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.0f - b1) * gg;
  const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  const float pn = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  p[e] = pn;
  q[e] = __float2bfloat16_rn(pn);
}

__global__ void k_counter_inc(int32_t *counter) { *counter += 1; }

template <bool AT, bool BT>
cudaError_t gemm(int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, float *C,
                 cudaStream_t s) {
  const int tiles = (M / 16) * (N / 16);
  k_gemm<AT, BT><<<(tiles + 3) / 4, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C);
  return cudaGetLastError();
}

inline int blocks(size_t n, int t = 256) { return (int)((n + t - 1) / t); }

// Forward pass of `rows` rows into the workspace (h1, h2 and the output
// pre-bias product in w.y); returns the first CUDA error.
cudaError_t forward(const rlqr_mlp_dims &d, const bf16 *q, const float *x, const int32_t *idx,
                    const int32_t *counter, int rows, char *ws, cudaStream_t s) {
  const Off o = offsets(d);
  const Ws w = ws_layout(d);
  const int W = d.width, P = o.npad;
  bf16 *a0 = reinterpret_cast<bf16 *>(ws + w.a0), *h1 = reinterpret_cast<bf16 *>(ws + w.h1);
  bf16 *h2 = reinterpret_cast<bf16 *>(ws + w.h2);
  float *c = reinterpret_cast<float *>(ws + w.c), *y = reinterpret_cast<float *>(ws + w.y);
  k_input<<<blocks((size_t)rows * 16), 256, 0, s>>>(x, idx, counter, rows, d.n_in, a0);
  cudaError_t e = gemm<false, true>(rows, W, 16, a0, 16, q + o.W1, 16, c, s);
  if (e != cudaSuccess) return e;
  k_bias_relu<<<blocks((size_t)rows * W), 256, 0, s>>>(c, q + o.b1, rows, W, h1);
  if ((e = gemm<false, true>(rows, W, W, h1, W, q + o.W2, W, c, s)) != cudaSuccess) return e;
  k_bias_relu<<<blocks((size_t)rows * W), 256, 0, s>>>(c, q + o.b2, rows, W, h2);
  if ((e = gemm<false, true>(rows, P, W, h2, W, q + o.W3, W, y, s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace rlqr

using namespace rlqr::mlp;

// The loss and gradient of a batch (rows of x, t selected by idx, advanced on
// the device by *counter batches when counter is given).
static cudaError_t grad_impl(const rlqr_mlp_dims &d, const bf16 *q, const float *x, const float *t,
                             const int32_t *idx, const int32_t *counter, int rows, float *loss,
                             float *grad, char *w, cudaStream_t s) {
  if (cudaError_t e = forward(d, q, x, idx, counter, rows, w, s)) return e;
  const Off o = offsets(d);
  const Ws L = ws_layout(d);
  const int W = d.width, P = o.npad;
  bf16 *a0 = reinterpret_cast<bf16 *>(w + L.a0), *h1 = reinterpret_cast<bf16 *>(w + L.h1);
  bf16 *h2 = reinterpret_cast<bf16 *>(w + L.h2), *dy = reinterpret_cast<bf16 *>(w + L.dy);
  bf16 *dz2 = reinterpret_cast<bf16 *>(w + L.dz2), *dz1 = reinterpret_cast<bf16 *>(w + L.dz1);
  float *dh = reinterpret_cast<float *>(w + L.dh), *part = reinterpret_cast<float *>(w + L.part);
  k_loss_grad<<<rows, 256, 0, s>>>(reinterpret_cast<float *>(w + L.y), q + o.b3, t, idx, counter,
                                   rows, P, d.n_out, dy, part);
  k_loss_final<<<1, 32, 0, s>>>(part, rows, rows, d.n_out, loss);
  if (cudaError_t e = gemm<true, false>(P, W, rows, dy, P, h2, W, grad + o.W3, s)) return e;
  k_colsum<<<(P + 31) / 32, dim3(32, 8), 0, s>>>(dy, rows, P, grad + o.b3);
  if (cudaError_t e = gemm<false, false>(rows, W, P, dy, P, q + o.W3, W, dh, s)) return e;
  k_relu_back<<<blocks((size_t)rows * W), 256, 0, s>>>(dh, h2, rows * W, dz2);
  if (cudaError_t e = gemm<true, false>(W, W, rows, dz2, W, h1, W, grad + o.W2, s)) return e;
  k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, s>>>(dz2, rows, W, grad + o.b2);
  if (cudaError_t e = gemm<false, false>(rows, W, W, dz2, W, q + o.W2, W, dh, s)) return e;
  k_relu_back<<<blocks((size_t)rows * W), 256, 0, s>>>(dh, h1, rows * W, dz1);
  if (cudaError_t e = gemm<true, false>(W, 16, rows, dz1, W, a0, 16, grad + o.W1, s)) return e;
  k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, s>>>(dz1, rows, W, grad + o.b1);
  return cudaGetLastError();
}

extern "C" {

size_t rlqr_mlp_param_count(const rlqr_mlp_dims *d) { return valid(d) ? offsets(*d).total : 0; }

size_t rlqr_mlp_workspace_bytes(const rlqr_mlp_dims *d) {
  return valid(d) ? ws_layout(*d).total : 0;
}

rlqr_status rlqr_mlp_sync_bf16(const rlqr_mlp_dims *d, const float *params, uint16_t *params_bf16,
                               rlqr_stream_t stream) {
  if (!valid(d) || !params || !params_bf16) return RLQR_ERR_ARG;
  const size_t n = offsets(*d).total;
  k_to_bf16<<<blocks(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      params, n, reinterpret_cast<bf16 *>(params_bf16));
  return cudaGetLastError() == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA;
}

static bool ws_ok(const rlqr_mlp_dims *d, void *ws, size_t ws_bytes) {
  return ws && ws_bytes >= ws_layout(*d).total && reinterpret_cast<uintptr_t>(ws) % 256 == 0;
}

rlqr_status rlqr_mlp_forward(const rlqr_mlp_dims *d, const uint16_t *params_bf16, const float *x,
                             int32_t rows, float *y, void *ws, size_t ws_bytes,
                             rlqr_stream_t stream) {
  if (!valid(d) || !params_bf16 || !x || !y || rows < 16 || rows % 16 || rows > d->max_rows ||
      reinterpret_cast<uintptr_t>(params_bf16) % 32)
    return RLQR_ERR_ARG;
  if (!ws_ok(d, ws, ws_bytes)) return RLQR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char *w = static_cast<char *>(ws);
  const bf16 *q = reinterpret_cast<const bf16 *>(params_bf16);
  if (forward(*d, q, x, nullptr, nullptr, rows, w, s) != cudaSuccess) return RLQR_ERR_CUDA;
  const Off o = offsets(*d);
  const Ws L = ws_layout(*d);
  k_bias_out<<<blocks((size_t)rows * d->n_out), 256, 0, s>>>(
      reinterpret_cast<float *>(w + L.y), q + o.b3, rows, o.npad, d->n_out, y);
  return cudaGetLastError() == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA;
}

rlqr_status rlqr_mlp_grad(const rlqr_mlp_dims *d, const uint16_t *params_bf16, const float *x,
                          const float *t, const int32_t *idx, int32_t rows, float *loss,
                          float *grad, void *ws, size_t ws_bytes, rlqr_stream_t stream) {
  // the tensor-core tiles load and store 32-byte aligned fragments
  if (!valid(d) || !params_bf16 || !x || !t || !loss || !grad || rows < 16 || rows % 16 ||
      rows > d->max_rows || reinterpret_cast<uintptr_t>(params_bf16) % 32 ||
      reinterpret_cast<uintptr_t>(grad) % 32)
    return RLQR_ERR_ARG;
  if (!ws_ok(d, ws, ws_bytes)) return RLQR_ERR_WORKSPACE;
  return grad_impl(*d, reinterpret_cast<const bf16 *>(params_bf16), x, t, idx, nullptr, rows, loss,
                   grad, static_cast<char *>(ws), reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? RLQR_OK
             : RLQR_ERR_CUDA;
}

rlqr_status rlqr_mlp_adam(const rlqr_mlp_dims *d, float *params, uint16_t *params_bf16,
                          float *m, float *v, const float *grad, int32_t step, float lr,
                          float beta1, float beta2, float eps, rlqr_stream_t stream) {
  if (!valid(d) || !params || !params_bf16 || !m || !v || !grad || step < 1 || !(lr > 0) ||
      !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return RLQR_ERR_ARG;
  const size_t n = offsets(*d).total;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_adam<<<blocks(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      params, reinterpret_cast<bf16 *>(params_bf16), m, v, grad, n, lr, beta1, beta2, eps, c1,
      c2, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA;
}

rlqr_status rlqr_mlp_train_step(const rlqr_mlp_dims *d, float *params, uint16_t *params_bf16,
                                float *m, float *v, float *grad, const float *x, const float *t,
                                const int32_t *idx_all, int32_t rows, int32_t *counter,
                                const float *sched, float beta1, float beta2, float eps,
                                float *loss, void *ws, size_t ws_bytes, rlqr_stream_t stream) {
  if (!valid(d) || !params || !params_bf16 || !m || !v || !grad || !x || !t || !idx_all ||
      !counter || !sched || !loss || rows < 16 || rows % 16 || rows > d->max_rows ||
      reinterpret_cast<uintptr_t>(params_bf16) % 32 || reinterpret_cast<uintptr_t>(grad) % 32 ||
      !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return RLQR_ERR_ARG;
  if (!ws_ok(d, ws, ws_bytes)) return RLQR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (grad_impl(*d, reinterpret_cast<const bf16 *>(params_bf16), x, t, idx_all, counter, rows,
                loss, grad, static_cast<char *>(ws), s) != cudaSuccess)
    return RLQR_ERR_CUDA;
  const size_t n = offsets(*d).total;
  k_adam<<<blocks(n), 256, 0, s>>>(params, reinterpret_cast<bf16 *>(params_bf16), m, v, grad, n,
                                   0.0f, beta1, beta2, eps, 1.0f, 1.0f, sched, counter);
  k_counter_inc<<<1, 1, 0, s>>>(counter);
  return cudaGetLastError() == cudaSuccess ? RLQR_OK : RLQR_ERR_CUDA;
}

}  // extern "C"
