// shard.cu -- launch sequences of the horizon-shard building blocks (FP64).
#include "launch.cuh"
#include "scan.cuh"
#include "shard.cuh"

namespace rlqr {

namespace {

template <int NX, int NU>
cudaError_t shard_element_sz(const BatchArgs &a, const ScanLayout &SL, size_t sbase,
                             double *elem, cudaStream_t s) {
  using CS = scan::CombSmem<double, NX, NU>;
  cudaError_t e;
  if ((e = cudaMemsetAsync(&reinterpret_cast<InstState *>(a.ws)->r_singular, 0, sizeof(int32_t),
                           s)) != cudaSuccess)
    return e;
  {
    auto k = k_scan_reduce<double, NX, NU>;
    if ((e = set_smem(k, sizeof(CS))) != cudaSuccess) return e;
    LaunchScope ls("k_scan_reduce", s);
    k<<<SL.C + 1, scan::kTH, sizeof(CS), s>>>(a, SL, sbase, 1, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int from1 = 0;
  {
    auto k = k_scan_level<double, NX, NU>;
    if ((e = set_smem(k, sizeof(CS))) != cudaSuccess) return e;
    for (int d = 1; d <= SL.C; d <<= 1) {
      LaunchScope ls("k_scan_level", s);
      k<<<SL.C + 1, scan::kTH, sizeof(CS), s>>>(a, SL, sbase, d, from1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      from1 ^= 1;
    }
  }
  const double *S = reinterpret_cast<const double *>(a.ws + sbase + (from1 ? SL.S1 : SL.S0));
  LaunchScope ls("k_shard_elem_out", s);
  k_shard_elem_out<NX><<<1, 256, 0, s>>>(S, elem);
  return cudaGetLastError();
}

template <int NX, int NU>
cudaError_t shard_boundary_sz(int G, int g, const double *elems, const double *QN,
                              double *P_end, double *P_start, cudaStream_t s) {
  using CS = scan::CombSmem<double, NX, NU>;
  auto k = k_shard_boundary<NX, NU>;
  cudaError_t e = set_smem(k, sizeof(CS));
  if (e != cudaSuccess) return e;
  LaunchScope ls("k_shard_boundary", s);
  k<<<1, scan::kTH, sizeof(CS), s>>>(G, g, elems, QN, P_end, P_start);
  return cudaGetLastError();
}

template <int NX, int NU>
cudaError_t shard_pmap_sz(const BatchArgs &a, const ScanLayout &SL, size_t sbase, double *Phi,
                          double *phi, cudaStream_t s) {
  const WsLayout L = ws_layout(a.N, a.n, a.m, 8);
  const double *Phic = reinterpret_cast<const double *>(a.ws + sbase + SL.Phi);
  const double *pv = reinterpret_cast<const double *>(a.ws + L.pv);
  LaunchScope ls("k_shard_pmap", s);
  k_shard_pmap<NX><<<1, scan::kTH, 0, s>>>(Phic, SL.C, pv, Phi, phi);
  return cudaGetLastError();
}

#define RLQR_SHARD_SIZES(X) \
  X(4, 2)                   \
  X(6, 2)                   \
  X(12, 4)                  \
  X(32, 8)

}  // namespace

cudaError_t launch_shard_element(int n, int m, const BatchArgs &a, const ScanLayout &SL,
                                 size_t sbase, double *elem, cudaStream_t s) {
#define RLQR_SHARD_E(NX, NU) \
  if (n == NX && m == NU) return shard_element_sz<NX, NU>(a, SL, sbase, elem, s);
  RLQR_SHARD_SIZES(RLQR_SHARD_E)
#undef RLQR_SHARD_E
  return cudaErrorNotSupported;
}

cudaError_t launch_shard_boundary(int n, int m, int G, int g, const double *elems,
                                  const double *QN, double *P_end, double *P_start,
                                  cudaStream_t s) {
#define RLQR_SHARD_B(NX, NU) \
  if (n == NX && m == NU) return shard_boundary_sz<NX, NU>(G, g, elems, QN, P_end, P_start, s);
  RLQR_SHARD_SIZES(RLQR_SHARD_B)
#undef RLQR_SHARD_B
  return cudaErrorNotSupported;
}

cudaError_t launch_shard_pmap(int n, int m, const BatchArgs &a, const ScanLayout &SL,
                              size_t sbase, double *Phi, double *phi, cudaStream_t s) {
#define RLQR_SHARD_P(NX, NU) \
  if (n == NX && m == NU) return shard_pmap_sz<NX, NU>(a, SL, sbase, Phi, phi, s);
  RLQR_SHARD_SIZES(RLQR_SHARD_P)
#undef RLQR_SHARD_P
  return cudaErrorNotSupported;
}

cudaError_t launch_shard_p_end(int G, int g, int n, const double *Phis, const double *phis,
                               const double *qN, double *p_end, cudaStream_t s) {
  LaunchScope ls("k_shard_p_end", s);
  k_shard_p_end<<<1, 32, 0, s>>>(G, g, n, Phis, phis, qN, p_end);
  return cudaGetLastError();
}

cudaError_t launch_shard_x_start(int g, int n, const double *Phis, const double *psis,
                                 double *x_start, cudaStream_t s) {
  LaunchScope ls("k_shard_x_start", s);
  k_shard_x_start<<<1, 32, 0, s>>>(g, n, Phis, psis, x_start);
  return cudaGetLastError();
}

cudaError_t launch_shard_x_offset(int n, const double *Phi, const double *x_first,
                                  const double *x_last, double *psi, cudaStream_t s) {
  LaunchScope ls("k_shard_x_offset", s);
  k_shard_x_offset<<<1, 32, 0, s>>>(n, Phi, x_first, x_last, psi);
  return cudaGetLastError();
}

cudaError_t launch_shard_entry(int n, double delta, const double *P_start,
                               const double *x_start, const double *x_first, double *c0,
                               cudaStream_t s) {
  LaunchScope ls("k_shard_entry", s);
  k_shard_entry<<<1, 32, 0, s>>>(n, delta, P_start, x_start, x_first, c0);
  return cudaGetLastError();
}

}  // namespace rlqr
