// Plan-time table generation: B, Pi, G and the calibration C of E expansions,
// all recreated from the seed with Philox4x32-10 (Sec. "McKernel": B from
// hash bits, Pi by Fisher-Yates driven by the hash, G by Box-Muller driven by
// the hash, C kernel-dependent; Sec. "API Description": nothing is stored).
//
// Counter layout (c0, c1, c2, c3) = (index, expansion, tag, sub-draw); key =
// the 64-bit seed as two words. This file is compiled with --fmad=false so
// that the double-precision formulas round exactly as written (G and the RBF
// radius then match an IEEE float64 evaluation of the same formulas up to the
// last-place differences of log/cos).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mma_layout.h"
#include "philox.cuh"

namespace mck {
namespace {

constexpr double kTwoM32 = 2.3283064365386962890625e-10;  // 2^-32
constexpr double kPi = 3.141592653589793238462643383279502884;

__device__ __forceinline__ double unit_open0(uint32_t w) { return ((double)w + 1.0) * kTwoM32; }
__device__ __forceinline__ double unit_closed0(uint32_t w) { return (double)w * kTwoM32; }

// Box-Muller (1958), cosine branch: sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ double box_muller_cos(uint32_t w0, uint32_t w1) {
  const double r = sqrt(-2.0 * log(unit_open0(w0)));
  const double a = 2.0 * kPi * unit_closed0(w1);
  return r * cos(a);
}

// B: bit (k mod 32) of word k/32 set where B_e[k] = -1 (bit 0 of Philox word 0).
__global__ void k_plan_B(uint32_t* __restrict__ bits, int64_t d, int64_t words, int32_t E,
                         uint32_t k0, uint32_t k1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= words * E) return;
  const uint32_t e = (uint32_t)(t / words);
  const int64_t w = t % words;
  uint32_t out = 0;
  for (int b = 0; b < 32; ++b) {
    const int64_t k = 32 * w + b;
    if (k < d) out |= (philox4x32_10((uint32_t)k, e, kTagB, 0, k0, k1).x & 1u) << b;
  }
  bits[t] = out;
}

// G_e[k] (float table) and its float64 value (for ||G_e||).
__global__ void k_plan_G(float* __restrict__ G, double* __restrict__ G64, int64_t d, int32_t E,
                         uint32_t k0, uint32_t k1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * E) return;
  const uint32_t e = (uint32_t)(t / d), k = (uint32_t)(t % d);
  const U32x4 w = philox4x32_10(k, e, kTagG, 0, k0, k1);
  const double g = box_muller_cos(w.x, w.y);
  G64[t] = g;
  G[t] = (float)g;
}

// ||G_e||_2 in float64, one block per expansion (fixed summation order).
__global__ void k_plan_norm(const double* __restrict__ G64, double* __restrict__ norm, int64_t d) {
  __shared__ double part[1024];
  const double* g = G64 + (int64_t)blockIdx.x * d;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < d; k += blockDim.x) s += g[k] * g[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) norm[blockIdx.x] = sqrt(part[0]);
}

// RBF radius r ~ chi_d: r^2 = 2 Gamma(d/2, 1) by Marsaglia & Tsang (2000):
// dd = d/2 - 1/3, c = 1/sqrt(9 dd); trial j draws g ~ N(0,1) (words 0, 1) and
// U (word 2) from counter (k, e, 4, j); v = (1 + c g)^3 > 0 is accepted when
// ln U < g^2/2 + dd - dd v + dd ln v; then r^2 = 2 dd v. Cs = r/||G_e||/(sigma sqrt d).
// LAPLACE: the Laplacian kernel exp(-|x - x'|/sigma) has the spherical
// multivariate Cauchy as spectral density, a radius chi_d / |N(0,1)|: r is
// divided by |n|, n the Box-Muller normal (words 0, 1) of counter (k, e, 7, 0),
// floored at 2^-32.
template <bool LAPLACE>
__global__ void k_plan_rbf(float* __restrict__ Cs, const double* __restrict__ norm, int64_t d,
                           int32_t E, double inv_sigma_sqrt_d, uint32_t k0, uint32_t k1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * E) return;
  const uint32_t e = (uint32_t)(t / d), k = (uint32_t)(t % d);
  const double a = (double)d / 2.0;
  const double dd = a - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * dd);
  double r = 0.0;
  for (uint32_t j = 0; j < 64; ++j) {
    const U32x4 w = philox4x32_10(k, e, kTagRbf, j, k0, k1);
    const double g = box_muller_cos(w.x, w.y);
    const double u = unit_open0(w.z);
    double v = 1.0 + c * g;
    if (v <= 0.0) continue;
    v = v * v * v;
    if (log(u) < 0.5 * g * g + dd - dd * v + dd * log(v)) {
      r = sqrt(2.0 * dd * v);
      break;
    }
  }
  if (LAPLACE) {
    const U32x4 w = philox4x32_10(k, e, kTagLaplace, 0, k0, k1);
    r /= fmax(fabs(box_muller_cos(w.x, w.y)), 0x1p-32);
  }
  Cs[t] = (float)((r / norm[e]) * inv_sigma_sqrt_d);
}

// Matern radius (Sec. "Customizing McKernel"): r = || sum_{j=1..t} u_j || with
// u_j = U_j^{1/d} X_j/||X_j||, X_j ~ N(0, I_d) (coordinates 2p, 2p+1 are the
// Box-Muller pair of counter (p, e, 5 + 16k, j)), U_j = (w0+1)/2^32 of
// counter (k, e, 6, j). One block per (e, k) (block index e*d + k); each thread owns up to 16 pairs
// of coordinates of the running sum, which stays in registers. Float32
// coordinates; squared norms summed in float per thread and in float64 across
// threads.
constexpr int kBallPairs = 16;

// KEEP: each thread keeps its coordinates of X_j in registers between the
// norm and the accumulation (up to 512 threads); otherwise X_j is drawn twice.
template <bool KEEP>
__global__ void __launch_bounds__(KEEP ? 512 : 1024) k_plan_matern(float* __restrict__ Cs,
                                                      const double* __restrict__ norm, int64_t d,
                                                      int32_t t_order, double inv_sigma_sqrt_d,
                                                      uint32_t k0, uint32_t k1) {
  __shared__ double red[32];
  __shared__ double bcast;
  const int64_t pairs = d / 2;
  const uint32_t e = (uint32_t)(blockIdx.x / d), k = (uint32_t)(blockIdx.x % d);
  const int tid = threadIdx.x, nt = blockDim.x;
  float s[2 * kBallPairs];
#pragma unroll
  for (int i = 0; i < 2 * kBallPairs; ++i) s[i] = 0.f;

  auto block_sum = [&](double v) -> double {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
      double x = (tid < (nt + 31) / 32) ? red[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (tid == 0) bcast = x;
    }
    __syncthreads();
    const double out = bcast;
    __syncthreads();
    return out;
  };

  auto coords = [&](int64_t p, uint32_t j, float& xc, float& xs) {
    const U32x4 w = philox4x32_10((uint32_t)p, e, kTagBall + 16u * k, j, k0, k1);
    const float u1 = (float)(((double)w.x + 1.0) * kTwoM32);
    const float u2 = (float)((double)w.y * kTwoM32);
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    xc = r * cs;
    xs = r * sn;
  };

  float xk[KEEP ? 2 * kBallPairs : 1];
  for (uint32_t j = 1; j <= (uint32_t)t_order; ++j) {
    // ||X_j||^2: float sums over a thread's (at most 32) coordinates, float64 across threads
    float ssf = 0.f;
#pragma unroll
    for (int i = 0; i < kBallPairs; ++i) {
      const int64_t p = tid + (int64_t)i * nt;
      if (p < pairs) {
        float xc, xs;
        coords(p, j, xc, xs);
        if constexpr (KEEP) {
          xk[2 * i] = xc;
          xk[2 * i + 1] = xs;
        }
        ssf += xc * xc + xs * xs;
      }
    }
    const double xnorm = sqrt(block_sum((double)ssf));
    const U32x4 wr = philox4x32_10(k, e, kTagBallRadius, j, k0, k1);
    const double rho = pow(unit_open0(wr.x), 1.0 / (double)d);
    const float scale = (float)(rho / xnorm);
#pragma unroll
    for (int i = 0; i < kBallPairs; ++i) {
      const int64_t p = tid + (int64_t)i * nt;
      if (p < pairs) {
        float xc, xs;
        if constexpr (KEEP) {
          xc = xk[2 * i];
          xs = xk[2 * i + 1];
        } else {
          coords(p, j, xc, xs);
        }
        s[2 * i] = fmaf(scale, xc, s[2 * i]);
        s[2 * i + 1] = fmaf(scale, xs, s[2 * i + 1]);
      }
    }
  }
  double ss = 0.0;
#pragma unroll
  for (int i = 0; i < kBallPairs; ++i) {
    const int64_t p = tid + (int64_t)i * nt;
    if (p < pairs) ss += (double)s[2 * i] * s[2 * i] + (double)s[2 * i + 1] * s[2 * i + 1];
  }
  const double r = sqrt(block_sum(ss));
  if (tid == 0) Cs[(int64_t)e * d + k] = (float)((r / norm[e]) * inv_sigma_sqrt_d);
}

// Pi_e by Durstenfeld's Fisher-Yates on L = [0..d-1]: for i = d-1 down to 1,
// j = floor(w0 (i+1) / 2^32) from counter (i, e, 2, 0), swap L[i], L[j].
// One block per expansion: the draws of 1024 consecutive steps are computed
// in parallel, then one thread applies the swaps in order (the shuffle is
// sequential by definition). L lives in shared memory (d <= 2^15).
__global__ void k_plan_perm(uint32_t* __restrict__ perm, int64_t d, uint32_t k0, uint32_t k1) {
  extern __shared__ uint32_t sm[];
  uint32_t* Ls = sm;
  uint32_t* J = sm + d;
  const uint32_t e = blockIdx.x;
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) Ls[i] = (uint32_t)i;
  __syncthreads();
  for (int64_t hi = d - 1; hi >= 1; hi -= 1024) {
    const int64_t lo = hi - 1023 > 1 ? hi - 1023 : 1;
    for (int64_t i = lo + threadIdx.x; i <= hi; i += blockDim.x) {
      const U32x4 w = philox4x32_10((uint32_t)i, e, kTagPerm, 0, k0, k1);
      J[i - lo] = __umulhi(w.x, (uint32_t)(i + 1));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int64_t i = hi; i >= lo; --i) {
        const uint32_t j = J[i - lo];
        const uint32_t a = Ls[i];
        Ls[i] = Ls[j];
        Ls[j] = a;
      }
    }
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) perm[(int64_t)e * d + i] = Ls[i];
}

// Lane-ordered copies of Pi, G and B for the warp kernels (see internal.h):
// entry t = (e, m, lam, q) of an expansion's d entries describes element
// k = kB(lam, 4m + q); the mask word (e, lam) has bit j for element kA(lam, j).
template <int L>
__global__ void k_plan_lane_tables(const uint32_t* __restrict__ perm, const float* __restrict__ G,
                                   const uint32_t* __restrict__ bits, uint32_t* __restrict__ permB,
                                   float* __restrict__ GB, uint32_t* __restrict__ maskA, int32_t E) {
  using Y = Lay<L>;
  constexpr int d = Y::d, T = Y::T;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)E * d) return;
  const int64_t e = t / d;
  const int r = (int)(t % d);
  const int q = r & 3, lam = (r >> 2) % T, m = (r >> 2) / T;
  const int k = Y::kB(lam, 4 * m + q);
  permB[t] = 4u * (uint32_t)pad((int)perm[e * d + k]);
  GB[t] = G[e * d + k];
  if (m == 0 && q == 0) {
    uint32_t mask = 0;
    for (int j = 0; j < 32; ++j) {
      const int kk = Y::kA(lam, j);
      mask |= ((bits[e * (d / 32) + (kk >> 5)] >> (kk & 31)) & 1u) << j;
    }
    maskA[e * T + lam] = mask;
  }
}

// The same tables for the chunked block kernels (11 <= L <= 14): vector
// element k = 1024 w + k' belongs to chunk w, and chunk w is laid out as a
// d = 1024 vector (k' = kB10(lam, 4m + q) for entry t = (e, w, m, lam, q)).
// Pi is stored as the word offset of pi(k) in the block's shared memory,
// where chunk i occupies 1056 words from i * 1056 (< 2^16 for L <= 14); the
// mask word (e, w, lam) has bit j for element 1024 w + kA10(lam, j).
template <int L>
__global__ void k_plan_chunk_tables(const uint32_t* __restrict__ perm, const float* __restrict__ G,
                                    const uint32_t* __restrict__ bits, uint32_t* __restrict__ permB,
                                    float* __restrict__ GB, uint32_t* __restrict__ maskA, int32_t E) {
  using Y = Lay<10>;
  constexpr int d = 1 << L;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)E * d) return;
  const int64_t e = t / d;
  const int r = (int)(t % d);
  const int w = r >> 10, rr = r & 1023;
  const int q = rr & 3, lam = (rr >> 2) & 31, m = rr >> 7;
  const int k = 1024 * w + Y::kB(lam, 4 * m + q);
  const int src = (int)perm[e * d + k];
  permB[t] = (uint32_t)((src >> 10) * Y::SLOT + pad(src & 1023));
  GB[t] = G[e * d + k];
  if (m == 0 && q == 0) {
    uint32_t mask = 0;
    for (int j = 0; j < 32; ++j) {
      const int kk = 1024 * w + Y::kA(lam, j);
      mask |= ((bits[e * (d / 32) + (kk >> 5)] >> (kk & 31)) & 1u) << j;
    }
    maskA[e * (d / 32) + w * 32 + lam] = mask;
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Durstenfeld's Fisher-Yates on the host for d > 2^15, exactly as
// k_plan_perm: for i = d-1 .. 1, j = mulhi(w0, i + 1) of Philox counter
// (i, e, 2, 0), swap L[i] and L[j]. Expansions on host threads; the result is
// copied to p->perm on stream s (and waited for).
mck_status_t host_perm(mck_plan_s* p, cudaStream_t s) {
  const int64_t d = p->d, E = p->E;
  const uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
  std::vector<uint32_t> perm((size_t)(d * E));
  auto shuffle = [&](int64_t e) {
    uint32_t* L = perm.data() + e * d;
    for (int64_t i = 0; i < d; ++i) L[i] = (uint32_t)i;
    for (int64_t i = d - 1; i >= 1; --i) {
      const U32x4 w = philox4x32_10((uint32_t)i, (uint32_t)e, kTagPerm, 0, k0, k1);
      const uint32_t j = mulhi_u32(w.x, (uint32_t)(i + 1));
      const uint32_t a = L[i];
      L[i] = L[j];
      L[j] = a;
    }
  };
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(E, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int64_t t = 1; t < nt; ++t)
    pool.emplace_back([&, t] {
      for (int64_t e = t; e < E; e += nt) shuffle(e);
    });
  for (int64_t e = 0; e < E; e += nt) shuffle(e);
  for (auto& th : pool) th.join();
  cudaError_t err = cudaMemcpyAsync(p->perm, perm.data(), sizeof(uint32_t) * perm.size(),
                                    cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "plan: permutation upload");
  return MCK_OK;
}

template <int L>
void launch_chunk_tables(mck_plan_s* p, cudaStream_t s) {
  k_plan_chunk_tables<L><<<blocks_for(p->d * p->E, 256), 256, 0, s>>>(p->perm, p->G, p->B_bits,
                                                                      p->permB, p->GB, p->maskA,
                                                                      p->E);
}

template <int L>
void launch_lane_tables(mck_plan_s* p, cudaStream_t s) {
  k_plan_lane_tables<L><<<blocks_for(p->d * p->E, 256), 256, 0, s>>>(p->perm, p->G, p->B_bits,
                                                                     p->permB, p->GB, p->maskA,
                                                                     p->E);
}

// Signs from real values: bit k of word (e, k / 32) is set (B_e[k] = -1)
// where B[e][k] < 0. One thread per word.
__global__ void k_plan_set_signs(const float* __restrict__ B, uint32_t* __restrict__ bits,
                                 int64_t d, int64_t words, int32_t E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= words * E) return;
  const int64_t e = t / words, w = t % words;
  uint32_t m = 0;
  for (int j = 0; j < 32; ++j) {
    const int64_t k = w * 32 + j;
    if (k < d && B[e * d + k] < 0.f) m |= 1u << j;
  }
  bits[t] = m;
}

// The tensor-core feature kernel's tables at d = 1024 (mma_layout.h orders):
// entry t = (e, m, lane, q) of an expansion's 1024 holds G at the input-order
// element of register j = 4m + q of `lane` and Cs at its output-order element;
// the mask word (e, lane) has bit j where B_e is -1 at the input-order element.
__global__ void k_plan_mma_tables(const float* __restrict__ G, const float* __restrict__ Cs,
                                  const uint32_t* __restrict__ bits, float* __restrict__ mG,
                                  float* __restrict__ mCs, uint32_t* __restrict__ mMask, int32_t E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)E * 1024) return;
  const int64_t e = t / 1024;
  const int rr = (int)(t % 1024);
  const int q = rr & 3, lane = (rr >> 2) & 31, m = rr >> 7, j = 4 * m + q;
  mG[t] = G[e * 1024 + mma_in(lane, j)];
  mCs[t] = Cs[e * 1024 + mma_out(lane, j)];
  if (m == 0 && q == 0) {
    uint32_t mask = 0;
    for (int jj = 0; jj < 32; ++jj) {
      const int k = mma_in(lane, jj);
      mask |= ((bits[e * 32 + (k >> 5)] >> (k & 31)) & 1u) << jj;
    }
    mMask[e * 32 + lane] = mask;
  }
}

// The lane-ordered copies of Pi, G and the B mask (warp and chunked kernels).
cudaError_t launch_layout_tables(mck_plan_s* p, cudaStream_t s) {
  if (p->mmaG) {
    k_plan_mma_tables<<<blocks_for(p->E * 1024, 256), 256, 0, s>>>(p->G, p->Cs, p->B_bits, p->mmaG,
                                                                   p->mmaCs, p->mmaMask, p->E);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (!p->permB) return cudaSuccess;
  switch (p->L) {
    case 5: launch_lane_tables<5>(p, s); break;
    case 6: launch_lane_tables<6>(p, s); break;
    case 7: launch_lane_tables<7>(p, s); break;
    case 8: launch_lane_tables<8>(p, s); break;
    case 9: launch_lane_tables<9>(p, s); break;
    case 10: launch_lane_tables<10>(p, s); break;
    case 11: launch_chunk_tables<11>(p, s); break;
    case 12: launch_chunk_tables<12>(p, s); break;
    case 13: launch_chunk_tables<13>(p, s); break;
    case 14: launch_chunk_tables<14>(p, s); break;
    default: break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t set_signs(mck_plan_s* p, const float* B, cudaStream_t s) {
  k_plan_set_signs<<<blocks_for(p->words * p->E, 128), 128, 0, s>>>(B, p->B_bits, p->d, p->words,
                                                                   p->E);
  const cudaError_t err = cudaGetLastError();
  return err != cudaSuccess ? err : launch_layout_tables(p, s);
}

mck_status_t build_tables(mck_plan_s* p, cudaStream_t s) {
  const uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
  const int64_t d = p->d, E = p->E, n = d * E;
  double* G64 = nullptr;
  double* norm = nullptr;
  cudaError_t err = cudaMallocAsync(&G64, sizeof(double) * n, s);
  if (err == cudaSuccess) err = cudaMallocAsync(&norm, sizeof(double) * E, s);
  if (err != cudaSuccess) {
    if (G64) cudaFreeAsync(G64, s);
    cudaGetLastError();
    return fail(MCK_ENOMEM, "plan: scratch allocation failed");
  }
  k_plan_B<<<blocks_for(p->words * E, 256), 256, 0, s>>>(p->B_bits, d, p->words, p->E, k0, k1);
  k_plan_G<<<blocks_for(n, 256), 256, 0, s>>>(p->G, G64, d, p->E, k0, k1);
  k_plan_norm<<<(unsigned)E, 1024, 0, s>>>(G64, norm, d);
  const double inv = 1.0 / (p->sigma * std::sqrt((double)d));
  if (p->kernel == MCK_RBF) {
    k_plan_rbf<false><<<blocks_for(n, 128), 128, 0, s>>>(p->Cs, norm, d, p->E, inv, k0, k1);
  } else if (p->kernel == MCK_LAPLACE) {
    k_plan_rbf<true><<<blocks_for(n, 128), 128, 0, s>>>(p->Cs, norm, d, p->E, inv, k0, k1);
  } else {
    const int64_t pairs = d / 2;
    int threads = (int)((pairs + kBallPairs - 1) / kBallPairs);
    threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
    if (threads <= 512)
      k_plan_matern<true><<<(unsigned)(d * E), threads, 0, s>>>(p->Cs, norm, d, p->matern_t, inv, k0, k1);
    else
      k_plan_matern<false><<<(unsigned)(d * E), threads, 0, s>>>(p->Cs, norm, d, p->matern_t, inv, k0, k1);
  }
  if (d <= ((int64_t)1 << 15)) {
    const size_t perm_smem = sizeof(uint32_t) * (size_t)(d + 1024);
    err = cudaFuncSetAttribute(k_plan_perm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)perm_smem);
    if (err == cudaSuccess) {
      k_plan_perm<<<(unsigned)E, 1024, perm_smem, s>>>(p->perm, d, k0, k1);
      err = cudaGetLastError();
    }
  } else {
    // The list no longer fits in shared memory: the same shuffle on the host
    // (the same Philox draws and swaps, so the same permutation).
    const mck_status_t st = host_perm(p, s);
    if (st != MCK_OK) {
      cudaFreeAsync(G64, s);
      cudaFreeAsync(norm, s);
      return st;
    }
  }
  if (err == cudaSuccess) err = launch_layout_tables(p, s);
  cudaFreeAsync(G64, s);
  cudaFreeAsync(norm, s);
  if (err != cudaSuccess) return cuda_fail(err, "plan kernels");
  err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "plan kernels");
  return MCK_OK;
}


// ---------------------------------------------------------------------------
// Skewed gather tables for d = 1024 (a memory layout of the forward warp
// kernels; the paper's method is unchanged by it).
//
// The forward kernels hold u = H B x-hat in layout B (lane lam, register j:
// element kB(lam, j)) and gather v_k = u_{pi(k)} for the same layout, one
// shared-memory load per register: load j of lane lam reads element
// pi(kB(lam, j)). With u stored in natural order these 32 reads of a warp hit
// random banks (about 3.5 times the conflict-free cost). Here u is stored with
// register j of lane lam at word base[lam] + 33 j: a store instruction (one j,
// all lanes) then touches banks (base[lam] + j) mod 32, distinct for any
// permutation `base` of 0..31, and the gather's banks become
// (base[lane of the source] + register of the source) mod 32. The bases of
// each expansion are chosen by simulated annealing over swaps, minimising the
// gather's wavefronts (the sum over its 32 loads of the largest number of
// lanes that share a bank); with random permutations this takes the gather
// from ~112 to ~84 wavefronts. The search is seeded by (plan seed,
// expansion), so equal plans get equal tables.
// ---------------------------------------------------------------------------
namespace {

struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Lane and register of element s in layout B at d = 1024.
inline int lane_of(int s) { return (s & 3) | ((s >> 7) << 2); }
inline int reg_of(int s) { return (s >> 2) & 31; }

// Bases (a permutation of 0..31) for one expansion's permutation pi (1024
// entries); returns the gather's wavefront count with them. Load j of lane l
// fills element dest(l, j) of the gather's layout; u element s sits in lane
// src_lane(s), register src_reg(s) of the stored layout.
template <class Dest, class SrcLane, class SrcReg>
int skew_bases(const uint32_t* pi, uint64_t seed, int iters, uint8_t* base, Dest dest,
               SrcLane src_lane, SrcReg src_reg) {
  // The 32 sources read from each lane group a: (load j, register of source).
  int occ_j[32][32], occ_r[32][32], nocc[32] = {0};
  for (int l = 0; l < 32; ++l)
    for (int j = 0; j < 32; ++j) {
      const int src = (int)pi[dest(l, j)];
      const int a = src_lane(src);
      occ_j[a][nocc[a]] = j;
      occ_r[a][nocc[a]] = src_reg(src);
      ++nocc[a];
    }
  int f[32], best_f[32];
  for (int a = 0; a < 32; ++a) f[a] = a;
  // cnt[j][b]: lanes of load j reading bank b; hist[j][c]: banks with count
  // c; mx[j]: the largest count (the load's wavefronts).
  int cnt[32][32], hist[32][34], mx[32];
  std::memset(cnt, 0, sizeof cnt);
  std::memset(hist, 0, sizeof hist);
  for (int a = 0; a < 32; ++a)
    for (int i = 0; i < nocc[a]; ++i) cnt[occ_j[a][i]][(f[a] + occ_r[a][i]) & 31]++;
  for (int j = 0; j < 32; ++j) {
    mx[j] = 0;
    for (int b = 0; b < 32; ++b) {
      hist[j][cnt[j][b]]++;
      if (cnt[j][b] > mx[j]) mx[j] = cnt[j][b];
    }
  }
  auto inc = [&](int j, int b) {
    const int c = cnt[j][b]++;
    hist[j][c]--;
    hist[j][c + 1]++;
    if (c + 1 > mx[j]) mx[j] = c + 1;
  };
  auto dec = [&](int j, int b) {
    const int c = cnt[j][b]--;
    hist[j][c]--;
    hist[j][c - 1]++;
    if (hist[j][mx[j]] == 0) mx[j]--;
  };
  auto total = [&] {
    int t = 0;
    for (int j = 0; j < 32; ++j) t += mx[j];
    return t;
  };
  auto swap_bases = [&](int a, int b) {
    for (int i = 0; i < nocc[a]; ++i) {
      dec(occ_j[a][i], (f[a] + occ_r[a][i]) & 31);
      inc(occ_j[a][i], (f[b] + occ_r[a][i]) & 31);
    }
    for (int i = 0; i < nocc[b]; ++i) {
      dec(occ_j[b][i], (f[b] + occ_r[b][i]) & 31);
      inc(occ_j[b][i], (f[a] + occ_r[b][i]) & 31);
    }
    const int t = f[a];
    f[a] = f[b];
    f[b] = t;
  };
  SplitMix rng{seed};
  int cur = total(), best = cur;
  std::memcpy(best_f, f, sizeof f);
  for (int it = 0; it < iters; ++it) {
    const double T = 2.0 * (1.0 - (double)it / iters) + 0.01;  // linear cooling
    const int a = (int)(rng.next() & 31), b = (int)((rng.next() >> 8) & 31);
    if (a == b) continue;
    swap_bases(a, b);
    const int c = total();
    if (c <= cur || rng.unit() < std::exp((cur - c) / T)) {
      cur = c;
      if (c < best) {
        best = c;
        std::memcpy(best_f, f, sizeof f);
      }
    } else {
      swap_bases(a, b);
    }
  }
  for (int a = 0; a < 32; ++a) base[a] = (uint8_t)best_f[a];
  return best;
}

// Annealing steps for the slots' lane bases. The FP32 feature kernel's slot
// takes 5x more: measured at d = 1024, E = 16 (60000 rows), 20000 steps give
// 1.511 ms per pass, 100000 steps 1.506 ms (400000: the same) for 33 ms more
// plan time; the tensor-core kernel's slot keeps the shorter run.
constexpr int kSkewIters = 20000;
constexpr int kSkewItersFp32 = 100000;

}  // namespace

mck_status_t build_skew_tables(mck_plan_s* p) {
  if (p->L != 10 || !p->permS || !p->ubase) return MCK_OK;
  const int d = 1024;
  const int64_t E = p->E;
  std::vector<uint32_t> pi((size_t)E * d), permS((size_t)E * d / 2), ubase((size_t)E * 32);
  std::vector<uint32_t> mPerm((size_t)E * d / 2), mBase((size_t)E * 32);
  cudaError_t err = cudaMemcpy(pi.data(), p->perm, sizeof(uint32_t) * pi.size(), cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return cuda_fail(err, "plan: skewed gather tables");
  auto pack = [](const uint32_t* pe, const uint8_t* base, int lam, int i, auto dest, auto slane,
                 auto sreg) {
    uint32_t wv = 0;
    for (int h = 0; h < 2; ++h) {
      const int src = (int)pe[dest(lam, 2 * i + h)];
      wv |= (4u * (uint32_t)(base[slane(src)] + 33 * sreg(src))) << (16 * h);
    }
    return wv;
  };
  auto work = [&](int64_t e) {
    const uint32_t* pe = pi.data() + e * d;
    const uint64_t seed = p->seed ^ (0x5851F42D4C957F2Dull * (uint64_t)(e + 1));
    // the tensor-core kernel: gather into the input order, u stored from the output order
    uint8_t mb[32];
    auto min_ = [](int l, int j) { return mma_in(l, j); };
    auto mlane = [](int src) { return mma_out_lane(src); };
    auto mreg = [](int src) { return mma_out_reg(src); };
    skew_bases(pe, seed ^ 0x9E3779B97F4A7C15ull, kSkewIters, mb, min_, mlane, mreg);
    for (int l = 0; l < 32; ++l) mBase[(size_t)e * 32 + l] = mb[l];
    for (int lam = 0; lam < 32; ++lam)
      for (int i = 0; i < 16; ++i)
        mPerm[(size_t)e * (d / 2) + ((size_t)(i >> 2) * 32 + lam) * 4 + (i & 3)] =
            pack(pe, mb, lam, i, min_, mlane, mreg);
    uint8_t base[32];
    skew_bases(pe, seed, kSkewItersFp32, base, [](int l, int j) { return Lay<10>::kB(l, j); },
               [](int src) { return lane_of(src); }, [](int src) { return reg_of(src); });
    for (int l = 0; l < 32; ++l) ubase[(size_t)e * 32 + l] = base[l];
    // Lane lam's 16 packed words: word i holds the byte offsets of its
    // registers 2i (low half) and 2i + 1 (high half); stored as 4 x uint4
    // per lane, uint4 q of lane lam at (q * 32 + lam).
    for (int lam = 0; lam < 32; ++lam)
      for (int i = 0; i < 16; ++i) {
        uint32_t wv = 0;
        for (int h = 0; h < 2; ++h) {
          const int src = (int)pi[(size_t)e * d + Lay<10>::kB(lam, 2 * i + h)];
          const uint32_t off = 4u * (uint32_t)(base[lane_of(src)] + 33 * reg_of(src));
          wv |= off << (16 * h);
        }
        permS[(size_t)e * (d / 2) + ((size_t)(i >> 2) * 32 + lam) * 4 + (i & 3)] = wv;
      }
  };
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(E, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int64_t t = 1; t < nt; ++t)
    pool.emplace_back([&, t] {
      for (int64_t e = t; e < E; e += nt) work(e);
    });
  for (int64_t e = 0; e < E; e += nt) work(e);
  for (auto& th : pool) th.join();
  err = cudaMemcpy(p->permS, permS.data(), sizeof(uint32_t) * permS.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess)
    err = cudaMemcpy(p->ubase, ubase.data(), sizeof(uint32_t) * ubase.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && p->mmaPerm)
    err = cudaMemcpy(p->mmaPerm, mPerm.data(), sizeof(uint32_t) * mPerm.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && p->mmaBase)
    err = cudaMemcpy(p->mmaBase, mBase.data(), sizeof(uint32_t) * mBase.size(), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return cuda_fail(err, "plan: skewed gather tables");
  return MCK_OK;
}

}  // namespace mck
