// Test-only probe of the device helpers in the package's common.cuh: the
// integer FP64 <-> FP32 conversions, the float-float split and dot product,
// the pivot reciprocal, the FP32 Gershgorin test and the FP32 Cholesky proof
// of positive definiteness.  Compiled by the GPU
// tests with nvcc; every entry point takes device pointers, runs on the
// default stream and returns the CUDA error code after synchronizing.
#include <cuda_runtime.h>

#include "../../paper_2509_16370_b300/csrc/common.cuh"

using namespace rlqr;

__global__ void k_conv(const double *v, float *rz, float *hi, float *lo, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rz[i] = f64_to_f32_rz(v[i]);
  const float2 s = split_f64(v[i]);
  hi[i] = s.x;
  lo[i] = s.y;
}

__global__ void k_widen(const float *f, double *w, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = f32_to_f64(f[i]);
}

__global__ void k_ffdot(const double *a, const double *z, const double *b, int rows, int len,
                        double *out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float sh = 0.f, sl = 0.f;
  ff_add(sh, sl, split_f64(b[r]));
  for (int j = 0; j < len; ++j) ff_fma(sh, sl, split_f64(a[(size_t)r * len + j]), split_f64(z[j]));
  out[r] = f32_to_f64(sh) + f32_to_f64(sl);
}

__global__ void k_recip(const float *d, float *r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = recip_pivot(d[i]);
}

// one row per thread: off = sum_{j != i} |P_ij| with round-up additions, as
// the sweep kernels accumulate it
__global__ void k_gersh(const float *P, int rows, int n, double delta, int *pass) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int i = r % n;
  const float *row = P + (size_t)r * n;
  float off = 0.f;
  for (int j = 0; j < n; ++j)
    if (j != i) off = __fadd_ru(off, fabsf(row[j]));
  pass[r] = gershgorin_row_pd(row[i], off, __double2float_ru(delta)) ? 1 : 0;
}

// one warp per matrix: the FP32 proof that I + delta P_k - tau D is PD
template <int NX>
__global__ void k_pdproof(const float *P, int count, double delta, float tau, int *pass) {
  const int k = blockIdx.x;
  if (k >= count) return;
  const int r = warp_pd_proof_f32<NX>(P + (size_t)k * NX * NX, delta, tau);
  if (threadIdx.x == 0) pass[k] = r;
}

static int finish() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

extern "C" int probe_conv(const double *v, float *rz, float *hi, float *lo, int n) {
  k_conv<<<(n + 127) / 128, 128>>>(v, rz, hi, lo, n);
  return finish();
}
extern "C" int probe_widen(const float *f, double *w, int n) {
  k_widen<<<(n + 127) / 128, 128>>>(f, w, n);
  return finish();
}
extern "C" int probe_ffdot(const double *a, const double *z, const double *b, int rows, int len,
                           double *out) {
  k_ffdot<<<(rows + 127) / 128, 128>>>(a, z, b, rows, len, out);
  return finish();
}
extern "C" int probe_recip(const float *d, float *r, int n) {
  k_recip<<<(n + 127) / 128, 128>>>(d, r, n);
  return finish();
}
extern "C" int probe_gersh(const float *P, int rows, int n, double delta, int *pass) {
  k_gersh<<<(rows + 127) / 128, 128>>>(P, rows, n, delta, pass);
  return finish();
}

extern "C" int probe_pdproof(const float *P, int count, int n, double delta, float tau,
                             int *pass) {
  if (n == 12) k_pdproof<12><<<count, 32>>>(P, count, delta, tau, pass);
  else if (n == 24) k_pdproof<24><<<count, 32>>>(P, count, delta, tau, pass);
  else if (n == 48) k_pdproof<48><<<count, 32>>>(P, count, delta, tau, pass);
  else return -1;
  return finish();
}
