// shard.cuh -- horizon shards of one long instance, FP64.
//
// A horizon [0, N] split into G contiguous shards [s_g, e_g] is solved by G
// independent sub-problems once three sets of boundary values are known,
// each from small summaries that the shards exchange (Section "Parallel
// Algorithm": the interval elements of contiguous stage ranges compose with
// the associative rule of eq. lqr-gpu-combo; Corollary p-recurrence and
// Section "Composing Affine Functions" for the vector maps):
//   1. the interval element (P, A, C) of every shard's stages -> P at each
//      shard's end and start (k_shard_boundary);
//   2. every shard's p map p_{s} = Phi p_{e} + phi (k_shard_pmap after the
//      shard's factor and a solve with p_e = 0) -> p at each shard's end
//      (k_shard_p_end);
//   3. every shard's x map x_{e} = Phi^T x_{s} + psi (k_shard_x_offset) ->
//      x at each shard's start (k_shard_x_start) and the shard's initial term
//      c_0 that reproduces it (k_shard_entry).
// The sub-problem of shard g is the LQR over its stages with terminal cost
// (P_{e}, p_{e}) and the initial term c_0 (dynamic programming cut).
#pragma once

#include "common.cuh"
#include "scan.cuh"

namespace rlqr {

// The first entry of a finished suffix scan (a shard's interval element).
template <int NX>
__global__ void k_shard_elem_out(const double *S, double *out) {
  for (int e = threadIdx.x; e < 3 * NX * NX; e += blockDim.x) out[e] = S[e];
}

// P at the end of shard g: the composition of the interval elements of
// shards g+1 .. G-1 and the terminal element (Q_N, 0, 0) of eq.
// lqr-gpu-init-terminal; P at its start: shard g's element in front of
// that.  elems: G x (P, A, C), each n x n row-major.  One CTA.
template <int NX, int NU>
__global__ void __launch_bounds__(scan::kTH) k_shard_boundary(int G, int g, const double *elems,
                                                              const double *QN, double *P_end,
                                                              double *P_start) {
  using SM = scan::CombSmem<double, NX, NU>;
  constexpr int n = NX, nn = n * n, LD = SM::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n, o = r * LD + c;
    s.P2[o] = __ldg(QN + (r <= c ? e : c * n + r));
    s.A2[o] = 0.0;
    s.C2[o] = 0.0;
  }
  for (int h = G - 1; h >= g; --h) {
    __syncthreads();
    if (h == g) {
      for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        P_end[e] = s.P2[r * LD + c];
      }
      if (!P_start) return;
    }
    scan::load_elem<double, NX>(elems + (size_t)h * 3 * nn, s.P1, s.A1, s.C1, LD);
    scan::combine<double, NX, NU>(s);  // (Pn, An, Cn) = element h (+) accumulator
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int r = e / n, c = e - r * n, o = r * LD + c;
      s.P2[o] = s.Pn[o];
      s.A2[o] = s.An[o];
      s.C2[o] = s.Cn[o];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    P_start[e] = s.P2[r * LD + c];
  }
}

// A factored and solved shard's p map: Phi = Phi_0 Phi_1 ... Phi_{C-1} over
// its chunk maps (p_s = Phi p_e + phi) and phi = its current p_0.  One CTA.
template <int NX>
__global__ void __launch_bounds__(scan::kTH) k_shard_pmap(const double *Phic, int C,
                                                          const double *pv, double *Phi,
                                                          double *phi) {
  constexpr int n = NX, nn = n * n, LD = NX + 2;
  __shared__ double acc[NX * LD], cur[NX * LD], res[NX * LD];
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    acc[r * LD + c] = Phic[(size_t)(C - 1) * nn + e];
  }
  for (int ch = C - 2; ch >= 0; --ch) {
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      cur[r * LD + c] = Phic[(size_t)ch * nn + e];
    }
    __syncthreads();
    scan::mmt<double, NX, NX, NX, false, false>(res, LD, cur, LD, acc, LD, nullptr, 0, 1.0);
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      acc[r * LD + c] = res[r * LD + c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    Phi[e] = acc[r * LD + c];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) phi[i] = pv[i];
}

// v <- M v + b (TRANS: M^T v + b) for an n x n row-major M, one warp, n <= 64.
__device__ __forceinline__ void warp_affine(double *v, const double *M, const double *b, int n,
                                            bool trans) {
  const int lane = threadIdx.x & 31;
  double t0 = 0.0, t1 = 0.0;
  __syncwarp();
  for (int l = 0; l < n; ++l) {
    const double vl = v[l];
    if (lane < n) t0 = fma(trans ? M[l * n + lane] : M[lane * n + l], vl, t0);
    if (lane + 32 < n) t1 = fma(trans ? M[l * n + lane + 32] : M[(lane + 32) * n + l], vl, t1);
  }
  __syncwarp();
  if (lane < n) v[lane] = t0 + (b ? b[lane] : 0.0);
  if (lane + 32 < n) v[lane + 32] = t1 + (b ? b[lane + 32] : 0.0);
  __syncwarp();
}

// p at the end of shard g from p_N = q_N: v <- Phi_h v + phi_h for
// h = G-1 .. g+1.  One warp.
__global__ void k_shard_p_end(int G, int g, int n, const double *Phis, const double *phis,
                              const double *qN, double *p_end) {
  __shared__ double v[64];
  for (int i = threadIdx.x; i < n; i += 32) v[i] = qN[i];
  for (int h = G - 1; h > g; --h)
    warp_affine(v, Phis + (size_t)h * n * n, phis + (size_t)h * n, n, false);
  __syncwarp();
  for (int i = threadIdx.x; i < n; i += 32) p_end[i] = v[i];
}

// x at the start of shard g >= 1: v = psi_0 (shard 0's last state), then
// v <- Phi_h^T v + psi_h for h = 1 .. g-1.  One warp.
__global__ void k_shard_x_start(int g, int n, const double *Phis, const double *psis,
                                double *x_start) {
  __shared__ double v[64];
  for (int i = threadIdx.x; i < n; i += 32) v[i] = psis[i];
  for (int h = 1; h < g; ++h)
    warp_affine(v, Phis + (size_t)h * n * n, psis + (size_t)h * n, n, true);
  __syncwarp();
  for (int i = threadIdx.x; i < n; i += 32) x_start[i] = v[i];
}

// psi = x_last - Phi^T x_first: the offset of a shard's x map from one of
// its trajectories.  One warp.
__global__ void k_shard_x_offset(int n, const double *Phi, const double *x_first,
                                 const double *x_last, double *psi) {
  __shared__ double v[64];
  for (int i = threadIdx.x; i < n; i += 32) v[i] = -x_first[i];
  warp_affine(v, Phi, x_last, n, true);
  for (int i = threadIdx.x; i < n; i += 32) psi[i] = v[i];
}

// c_0 = (I + delta P_s)(x_start - x_first): the initial term that moves a
// shard's first state from x_first (its solve with c_0 = 0) to x_start
// (x_0 = (I + delta P_0)^{-1} (c_0 - delta p_0), eq. recover-x0).  One warp.
__global__ void k_shard_entry(int n, double delta, const double *P_start, const double *x_start,
                              const double *x_first, double *c0) {
  __shared__ double d[64];
  const int lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) d[i] = x_start[i] - x_first[i];
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    double t = 0.0;
    for (int l = 0; l < n; ++l) t = fma(P_start[i * n + l], d[l], t);
    c0[i] = fma(delta, t, d[i]);
  }
}

}  // namespace rlqr
