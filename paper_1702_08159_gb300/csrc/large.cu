// Multi-pass forms of the feature map and its adjoint, for the dimensions the
// one-pass kernels do not hold on chip: features at 2^15 < d <= 2^20 and the
// adjoint at 2^11 <= d <= 2^20. The same arithmetic as the fused kernels, one
// step per pass over an HBM scratch of the rows in flight (Eq. etn:mckernel,
// Eq. etn:mcfeatures):
//
//   forward   U = B x-hat;  U = H U;  V = G (Pi U);  V = H V;  phi = [cos | sin](Cs V)
//   adjoint   (recompute u = H B x-hat, v = Pi u, h = H G v), then
//             dz = -sin z dphi_cos + cos z dphi_sin    dCs += h dz    dh = Cs dz
//             dw = H dh                                dG  += v dw    dv = G dw
//             du = Pi^T dv (scatter)   du0 = H du      dx = sum_e B_e du0   dB += x-hat du0
//
// H runs through the library's transform (launch_fwht: warp, chunked,
// cluster or two-pass regime by d). Rows go in chunks sized to a fixed
// scratch budget. Sums over the batch (dCs, dG, dB) are taken by one thread
// per (e, k) looping over the chunk's rows in order, written by the first
// chunk and added by the later ones, so results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace mck {
namespace {

constexpr int kT = 256;

unsigned grid_for(int64_t n, int num_sms) {
  const int64_t want = (n + kT - 1) / kT;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 16));
}

__device__ __forceinline__ float bsign(const uint32_t* __restrict__ bits, int64_t words, int e,
                                       int64_t k) {
  return (__ldg(bits + (int64_t)e * words + (k >> 5)) >> (k & 31)) & 1u ? -1.f : 1.f;
}

// U[(r, e), k] = B_e[k] x[r0 + r][k] (k < in_dim), else 0.
__global__ void k_mp_sign(const float* __restrict__ x, int64_t ldx, int64_t in_dim,
                          const uint32_t* __restrict__ bits, int64_t words, int64_t d, int E,
                          int64_t r0, int64_t rows, float* __restrict__ U) {
  const int64_t total = rows * E * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t % d, re = t / d;
    const int e = (int)(re % E);
    const int64_t r = re / E;
    const float xv = k < in_dim ? __ldg(x + (r0 + r) * ldx + k) : 0.f;
    U[t] = bsign(bits, words, e, k) * xv;
  }
}

// V = G (Pi U) per (r, e); Vp (optional) = Pi U, the v of the adjoint.
__global__ void k_mp_gather(const float* __restrict__ U, const uint32_t* __restrict__ perm,
                            const float* __restrict__ G, int64_t d, int E, int64_t rows,
                            float* __restrict__ V, float* __restrict__ Vp) {
  const int64_t total = rows * E * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t % d, re = t / d;
    const int64_t ek = (re % E) * d + k;
    const float v = U[re * d + __ldg(perm + ek)];
    if (Vp) Vp[t] = v;
    V[t] = __ldg(G + ek) * v;
  }
}

// phi[r0 + r][e 2d + k] = cos(Cs_e[k] h), phi[...][e 2d + d + k] = sin(...).
__global__ void k_mp_features(const float* __restrict__ H, const float* __restrict__ Cs, int64_t d,
                              int E, int64_t r0, int64_t rows, float* __restrict__ phi) {
  const int64_t total2 = rows * E * d / 2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total2;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 2 * t, k = i % d, re = i / d;
    const int64_t e = re % E, r = re / E;
    const float2 h = *reinterpret_cast<const float2*>(H + i);
    const float2 cs = *reinterpret_cast<const float2*>(Cs + e * d + k);
    float2 c, s;
    cos_sin2(cs, h, c, s);
    float* o = phi + (r0 + r) * 2 * E * d + 2 * e * d + k;
    __stcs(reinterpret_cast<float2*>(o), c);
    __stcs(reinterpret_cast<float2*>(o + d), s);
  }
}

// One thread per (e, k): over the chunk's rows, z = Cs h, dz from dphi (given,
// or formed as dlogits W), dCs sum of h dz; H becomes dh = Cs dz; phi_out (if
// given) receives the recomputed features.
__global__ void k_mp_dz(float* __restrict__ H, const float* __restrict__ Cs,
                        const float* __restrict__ dphi, const float* __restrict__ dl,
                        const float* __restrict__ W, int C, int64_t d, int E, int64_t r0,
                        int64_t rows, float* __restrict__ dCs, bool first,
                        float* __restrict__ phi_out) {
  const int64_t ed = (int64_t)E * d, F = 2 * ed;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ed;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / d, k = t % d;
    const float cs = __ldg(Cs + t);
    const int64_t fc = 2 * e * d + k, fs = fc + d;
    float wc[MCK_MAX_CLASSES], ws[MCK_MAX_CLASSES];
    if (dl) {
#pragma unroll
      for (int c = 0; c < MCK_MAX_CLASSES; ++c) {
        wc[c] = c < C ? __ldg(W + c * F + fc) : 0.f;
        ws[c] = c < C ? __ldg(W + c * F + fs) : 0.f;
      }
    }
    float acc = 0.f;
    for (int64_t r = 0; r < rows; ++r) {
      float* hp = H + r * ed + t;
      const float h = *hp;
      float c, s;
      cos_sin(cs * h, c, s);
      float gc, gs;
      if (dl) {
        gc = 0.f;
        gs = 0.f;
        const float* dr = dl + (r0 + r) * C;
#pragma unroll
        for (int q = 0; q < MCK_MAX_CLASSES; ++q) {
          if (q < C) {
            const float g = __ldg(dr + q);
            gc = fmaf(g, wc[q], gc);
            gs = fmaf(g, ws[q], gs);
          }
        }
      } else {
        gc = __ldg(dphi + (r0 + r) * F + fc);
        gs = __ldg(dphi + (r0 + r) * F + fs);
      }
      const float dz = fmaf(-s, gc, c * gs);
      acc = fmaf(h, dz, acc);
      *hp = cs * dz;
      if (phi_out) {
        phi_out[(r0 + r) * F + fc] = c;
        phi_out[(r0 + r) * F + fs] = s;
      }
    }
    if (dCs) dCs[t] = first ? acc : dCs[t] + acc;
  }
}

// One thread per (e, k): dG sum of v dw over the chunk's rows; D becomes dv = G dw.
__global__ void k_mp_dg(float* __restrict__ D, const float* __restrict__ Vp,
                        const float* __restrict__ G, int64_t d, int E, int64_t rows,
                        float* __restrict__ dG, bool first) {
  const int64_t ed = (int64_t)E * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ed;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float g = __ldg(G + t);
    float acc = 0.f;
    for (int64_t r = 0; r < rows; ++r) {
      float* p = D + r * ed + t;
      const float dw = *p;
      acc = fmaf(Vp[r * ed + t], dw, acc);
      *p = g * dw;
    }
    if (dG) dG[t] = first ? acc : dG[t] + acc;
  }
}

// du = Pi^T dv: U[(r, e), pi_e(k)] = D[(r, e), k] (a permutation: no collisions).
__global__ void k_mp_scatter(const float* __restrict__ D, const uint32_t* __restrict__ perm,
                             int64_t d, int E, int64_t rows, float* __restrict__ U) {
  const int64_t total = rows * E * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t % d, re = t / d;
    U[re * d + __ldg(perm + (re % E) * d + k)] = D[t];
  }
}

// dx[r0 + r][k] = sum over e (in order) of B_e[k] du0[(r, e), k], k < in_dim.
__global__ void k_mp_dx(const float* __restrict__ U, const uint32_t* __restrict__ bits,
                        int64_t words, int64_t d, int E, int64_t in_dim, int64_t ldx, int64_t r0,
                        int64_t rows, float* __restrict__ dx) {
  const int64_t total = rows * in_dim;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / in_dim, k = t % in_dim;
    float acc = 0.f;
    for (int e = 0; e < E; ++e) acc = fmaf(bsign(bits, words, e, k), U[(r * E + e) * d + k], acc);
    dx[(r0 + r) * ldx + k] = acc;
  }
}

// One thread per (e, k): dB sum of x-hat du0 over the chunk's rows.
__global__ void k_mp_db(const float* __restrict__ U, const float* __restrict__ x, int64_t ldx,
                        int64_t in_dim, int64_t d, int E, int64_t r0, int64_t rows,
                        float* __restrict__ dB, bool first) {
  const int64_t ed = (int64_t)E * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ed;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t % d;
    float acc = 0.f;
    if (k < in_dim)
      for (int64_t r = 0; r < rows; ++r) acc = fmaf(__ldg(x + (r0 + r) * ldx + k), U[r * ed + t], acc);
    dB[t] = first ? acc : dB[t] + acc;
  }
}

// logits[r0 + r][c] = b[c] + sum_f phi[r][f] W[c][f]: one block per row, a
// fixed-order reduction over the block.
__global__ void __launch_bounds__(kT) k_mp_logits(const float* __restrict__ phi,
                                                  const float* __restrict__ W,
                                                  const float* __restrict__ b, int C, int64_t F,
                                                  int64_t r0, float* __restrict__ logits) {
  __shared__ float red[kT / 32][MCK_MAX_CLASSES];
  const int64_t r = blockIdx.x;
  const float* pr = phi + r * F;
  float acc[MCK_MAX_CLASSES];
#pragma unroll
  for (int c = 0; c < MCK_MAX_CLASSES; ++c) acc[c] = 0.f;
  for (int64_t f = threadIdx.x; f < F; f += kT) {
    const float p = pr[f];
#pragma unroll
    for (int c = 0; c < MCK_MAX_CLASSES; ++c)
      if (c < C) acc[c] = fmaf(p, __ldg(W + c * F + f), acc[c]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < MCK_MAX_CLASSES; ++c) {
    float t = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp][c] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < C) {
    float t = 0.f;
    for (int w = 0; w < kT / 32; ++w) t += red[w][threadIdx.x];
    logits[(r0 + r) * C + threadIdx.x] = t + (b ? b[threadIdx.x] : 0.f);
  }
}

// Rows per chunk for a scratch of `bufs` buffers of rows x E x d floats (plus
// `extra` floats per row) within kScratchFloats.
constexpr int64_t kScratchFloats = (int64_t)1 << 26;  // 256 MiB

int64_t chunk_rows(int64_t n, int64_t ed, int bufs, int64_t extra) {
  const int64_t per = bufs * ed + extra;
  return std::max<int64_t>(1, std::min<int64_t>(n, kScratchFloats / per));
}

#define MP_TRY(expr)                                \
  do {                                              \
    const cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return _e;               \
  } while (0)

// u = H B x-hat into U, then V = G Pi u (Vp = Pi u if given), then h = H V.
cudaError_t forward_chunk(const FeatureArgs& a, int64_t r0, int64_t rows, float* U, float* V,
                          float* Vp, cudaStream_t s) {
  const int64_t d = (int64_t)1 << a.L, words = (d + 31) / 32, tot = rows * a.E * d;
  const unsigned g = grid_for(tot, a.num_sms);
  k_mp_sign<<<g, kT, 0, s>>>(a.x, a.ldx, a.in_dim, a.B_bits, words, d, a.E, r0, rows, U);
  MP_TRY(cudaGetLastError());
  MP_TRY(launch_fwht(U, rows * a.E, a.L, a.num_sms, s));
  k_mp_gather<<<g, kT, 0, s>>>(U, a.perm, a.G, d, a.E, rows, V, Vp);
  MP_TRY(cudaGetLastError());
  return launch_fwht(V, rows * a.E, a.L, a.num_sms, s);
}

}  // namespace

int64_t multipass_scratch_floats(int L, int64_t n, int E, int C, bool backward) {
  if (n <= 0) return 0;
  const int64_t d = (int64_t)1 << L, ed = (int64_t)E * d;
  if (backward) return chunk_rows(n, ed, 3, 0) * 3 * ed;
  const int64_t extra = C > 0 ? 2 * ed : 0;  // fused logits: the chunk's features
  return chunk_rows(n, ed, 2, extra) * (2 * ed + extra);
}

cudaError_t launch_features_multipass(const FeatureArgs& a, float* phi, const float* W,
                                      const float* b, int C, float* logits, float* scratch,
                                      cudaStream_t s) {
  const int64_t d = (int64_t)1 << a.L, ed = (int64_t)a.E * d;
  const bool fused = logits != nullptr;
  const int64_t rows_max = chunk_rows(a.n, ed, 2, fused ? 2 * ed : 0);
  float* U = scratch;
  float* V = U + rows_max * ed;
  float* ph = fused ? V + rows_max * ed : nullptr;
  for (int64_t r0 = 0; r0 < a.n; r0 += rows_max) {
    const int64_t rows = std::min<int64_t>(rows_max, a.n - r0);
    MP_TRY(forward_chunk(a, r0, rows, U, V, nullptr, s));
    const unsigned g = grid_for(rows * ed / 2, a.num_sms);
    if (fused) {
      k_mp_features<<<g, kT, 0, s>>>(V, a.Cs, d, a.E, 0, rows, ph);
      MP_TRY(cudaGetLastError());
      k_mp_logits<<<(unsigned)rows, kT, 0, s>>>(ph, W, b, C, 2 * ed, r0, logits);
    } else {
      k_mp_features<<<g, kT, 0, s>>>(V, a.Cs, d, a.E, r0, rows, phi);
    }
    MP_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t launch_backward_multipass(const BackwardArgs& b, float* scratch, cudaStream_t s) {
  const FeatureArgs& a = b.f;
  const int64_t d = (int64_t)1 << a.L, ed = (int64_t)a.E * d, words = (d + 31) / 32;
  const int64_t rows_max = chunk_rows(a.n, ed, 3, 0);
  float* U = scratch;
  float* Vp = U + rows_max * ed;
  float* H = Vp + rows_max * ed;
  for (int64_t r0 = 0; r0 < a.n; r0 += rows_max) {
    const int64_t rows = std::min<int64_t>(rows_max, a.n - r0);
    const bool first = r0 == 0;
    MP_TRY(forward_chunk(a, r0, rows, U, H, Vp, s));  // H = h, Vp = v
    const unsigned ge = grid_for(ed, a.num_sms), gt = grid_for(rows * ed, a.num_sms);
    k_mp_dz<<<ge, kT, 0, s>>>(H, a.Cs, b.dphi, b.dlogits, b.W, b.C, d, a.E, r0, rows, b.dCs, first,
                              b.phi_out);
    MP_TRY(cudaGetLastError());
    MP_TRY(launch_fwht(H, rows * a.E, a.L, a.num_sms, s));  // dw
    k_mp_dg<<<ge, kT, 0, s>>>(H, Vp, a.G, d, a.E, rows, b.dG, first);
    MP_TRY(cudaGetLastError());
    if (!b.dx && !b.dB) continue;
    k_mp_scatter<<<gt, kT, 0, s>>>(H, a.perm, d, a.E, rows, U);
    MP_TRY(cudaGetLastError());
    MP_TRY(launch_fwht(U, rows * a.E, a.L, a.num_sms, s));  // du0
    if (b.dx) {
      k_mp_dx<<<grid_for(rows * a.in_dim, a.num_sms), kT, 0, s>>>(U, a.B_bits, words, d, a.E,
                                                                  a.in_dim, a.ldx, r0, rows, b.dx);
      MP_TRY(cudaGetLastError());
    }
    if (b.dB) {
      k_mp_db<<<ge, kT, 0, s>>>(U, a.x, a.ldx, a.in_dim, d, a.E, r0, rows, b.dB, first);
      MP_TRY(cudaGetLastError());
    }
  }
  return cudaSuccess;
}

}  // namespace mck
