// Training-side kernels: the softmax cross-entropy of Sec. "Empirical
// Analysis" (the multi-class form of the logistic loss, Eq. etn:loss) and the
// adjoint of the Fastfood feature map, which Sec. "Empirical Analysis"
// motivates ("learn the appropriate Calibration C and G" by backpropagation).
//
// The adjoint recomputes the forward and runs the chain rule backwards,
// using H^T = H (Sylvester H is symmetric) and Pi^T = Pi^{-1} (the gather
// becomes a scatter to the same addresses):
//   dz  = -sin z dphi_cos + cos z dphi_sin
//   dCs += h dz            dh = Cs dz         dw = H dh
//   dG  += v dw            dv = G dw          du[pi(k)] = dv[k]      du0 = H du
//   dx  += (B du0)[:in_dim]
// Two warp kernels share that per-sample core:
//   k_bwd_params  work items (tile of samples, expansion), expansion-major,
//                 accumulate dCs, dG per warp, write one partial row per warp;
//                 k_reduce_params sums the rows of each expansion in order.
//   k_bwd_input   each warp owns samples and loops over all expansions,
//                 accumulating dx in registers (no cross-warp sum needed).
// With fused logits the upstream gradient is dphi = W^T dlogits, formed on
// the fly from W; k_bwd_params then also writes the recomputed features so
// k_logit_weight_grads can form dW = dlogits^T phi and db = sum dlogits.
// All sums run in a fixed order, so results are bit-reproducible.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace mck {
namespace {

constexpr int kBW = 4;  // warps per block
constexpr int CMAX = MCK_MAX_CLASSES;

// ---------------------------------------------------------------------------
// Softmax cross-entropy: one block, fixed-order sums (deterministic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_softmax_xent(const float* __restrict__ logits,
                                                       const int32_t* __restrict__ labels,
                                                       int64_t n, int C, float* __restrict__ loss,
                                                       float* __restrict__ dlogits) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float* l = logits + i * C;
    const int y = labels[i];
    const bool ok = y >= 0 && y < C;
    float m = l[0];
    for (int c = 1; c < C; ++c) m = fmaxf(m, l[c]);
    float s = 0.f;
    for (int c = 0; c < C; ++c) s += expf(l[c] - m);
    const float lse = m + logf(s);
    if (ok) acc += (double)(lse - l[y]);
    if (dlogits) {
      const float inv_n = 1.0f / (float)n;
      for (int c = 0; c < C; ++c) {
        const float p = expf(l[c] - lse);
        dlogits[i * C + c] = ok ? (p - (c == y ? 1.f : 0.f)) * inv_n : 0.f;
      }
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = n > 0 ? (float)(red[0] / (double)n) : 0.f;
}

// ---------------------------------------------------------------------------
// Backward core.
// ---------------------------------------------------------------------------
template <int L>
struct BShape {
  static constexpr int T = Lay<L>::T;
  static constexpr int VPW = 32 / T;
  static constexpr int R = VPW >= 8 ? 1 : 8 / VPW;
  static constexpr int SPI = VPW * R;
};

struct BwdLaunch {
  BackwardArgs b;
  bool vec_x;
  float* partials;  // [warps][2][d]
  int wpe;          // warps per expansion (k_bwd_params)
};

__device__ __forceinline__ void apply_signs(float (&w)[32], uint32_t mask) {
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = __int_as_float(__float_as_int(w[j]) ^ ((mask << (31 - j)) & 0x80000000u));
}

template <int L>
__device__ __forceinline__ uint32_t load_bmask_A(const uint32_t* __restrict__ Bw, int lam) {
  uint32_t mask = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Lay<L>::kA(lam, 4 * m);
    mask |= ((__ldg(Bw + (k0 >> 5)) >> (k0 & 31)) & 0xFu) << (4 * m);
  }
  return mask;
}

// Per-warp shared state of the backward kernels. Arrays indexed [j][lane]
// are private to a lane (bank-conflict free).
template <int L>
struct BwdSmem {
  float buf[BShape<L>::VPW * Lay<L>::SLOT];
  float gl[32 * 32];   // G in layout B
  float csl[32 * 32];  // Cs in layout A
  float vl[32 * 32];   // v = Pi u of the current sample, layout B
  float dcs[32 * 32];  // running sum of h dz, layout A
  float dg[32 * 32];   // running sum of v dw, layout B
};

template <int L>
__device__ __forceinline__ void load_tables(const FeatureArgs& a, int e, int g, int lam, int lane,
                                            uint32_t buf_addr, BwdSmem<L>& S, uint32_t& bmask,
                                            uint32_t (&paddr)[32]) {
  using Y = Lay<L>;
  constexpr int d = Y::d;
  const int64_t off = (int64_t)e * d;
  bmask = load_bmask_A<L>(a.B_bits + (int64_t)e * (d / 32), lam);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int k = Y::kB(lam, j);
    S.gl[j * 32 + lane] = __ldg(a.G + off + k);
    paddr[j] = buf_addr + 4u * (uint32_t)spos<L>(g, (int)__ldg(a.perm + off + k));
    S.csl[j * 32 + lane] = __ldg(a.Cs + off + Y::kA(lam, j));
  }
}

// One sample of one expansion: forward recompute and backward. On return w
// holds B du0 (layout A), the sample's contribution to dx-hat.
template <int L, bool FUSED, bool PARAMS>
__device__ __forceinline__ void bwd_core(const BwdLaunch& P, int64_t n, int e, bool valid, int g,
                                         int lam, int lane, BwdSmem<L>& S, uint32_t bmask,
                                         const uint32_t (&paddr)[32], float (&w)[32]) {
  using Y = Lay<L>;
  constexpr int d = Y::d;
  const FeatureArgs& a = P.b.f;
  const int64_t F = 2ll * a.E * d;
  float* buf = S.buf;
  // ---- forward: u = H B x-hat, v = Pi u, h = H G v ----
  {
    const float* row = a.x + n * a.ldx;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k0 = Y::kA(lam, 4 * m);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) {
        if (P.vec_x) {
          if (k0 < a.in_dim) v = __ldg(reinterpret_cast<const float4*>(row + k0));
        } else {
          if (k0 + 0 < a.in_dim) v.x = __ldg(row + k0 + 0);
          if (k0 + 1 < a.in_dim) v.y = __ldg(row + k0 + 1);
          if (k0 + 2 < a.in_dim) v.z = __ldg(row + k0 + 2);
          if (k0 + 3 < a.in_dim) v.w = __ldg(row + k0 + 3);
        }
      }
      w[4 * m] = v.x;
      w[4 * m + 1] = v.y;
      w[4 * m + 2] = v.z;
      w[4 * m + 3] = v.w;
    }
  }
  apply_signs(w, bmask);
  hreg<Y::maskA()>(w);
  if constexpr (L > 5) {
    store_A<L>(buf, g, lam, w);
    __syncwarp();
    load_B<L>(buf, g, lam, w);
  }
  hreg<Y::maskB()>(w);
  store_B<L>(buf, g, lam, w);
  __syncwarp();
  float gt[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    w[j] = lds32(paddr[j]);
    if constexpr (PARAMS) S.vl[j * 32 + lane] = w[j];
    gt[j] = S.gl[j * 32 + lane];
  }
  hreg_scaled<Y::maskB()>(w, gt);
  __syncwarp();
  if constexpr (L > 5) {
    store_B<L>(buf, g, lam, w);
    __syncwarp();
    load_A<L>(buf, g, lam, w);
  }
  hreg<Y::maskA()>(w);  // w = h, layout A
  // ---- dz from the upstream gradient ----
  float dl[CMAX];
  if constexpr (FUSED) {
#pragma unroll
    for (int c = 0; c < CMAX; ++c)
      dl[c] = (valid && c < P.b.C) ? __ldg(P.b.dlogits + n * P.b.C + c) : 0.f;
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Y::kA(lam, 4 * m);
    float dc[4] = {0.f, 0.f, 0.f, 0.f}, ds[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (FUSED) {
      const float* wr = P.b.W + 2ll * e * d + k0;
#pragma unroll
      for (int c = 0; c < CMAX; ++c) {
        if (c < P.b.C) {
          const float4 wc = __ldg(reinterpret_cast<const float4*>(wr + c * F));
          const float4 ws = __ldg(reinterpret_cast<const float4*>(wr + c * F + d));
          dc[0] = fmaf(dl[c], wc.x, dc[0]);
          dc[1] = fmaf(dl[c], wc.y, dc[1]);
          dc[2] = fmaf(dl[c], wc.z, dc[2]);
          dc[3] = fmaf(dl[c], wc.w, dc[3]);
          ds[0] = fmaf(dl[c], ws.x, ds[0]);
          ds[1] = fmaf(dl[c], ws.y, ds[1]);
          ds[2] = fmaf(dl[c], ws.z, ds[2]);
          ds[3] = fmaf(dl[c], ws.w, ds[3]);
        }
      }
    } else if (valid) {
      const float* gr = P.b.dphi + n * F + 2ll * e * d + k0;
      const float4 vc = __ldg(reinterpret_cast<const float4*>(gr));
      const float4 vs = __ldg(reinterpret_cast<const float4*>(gr + d));
      dc[0] = vc.x; dc[1] = vc.y; dc[2] = vc.z; dc[3] = vc.w;
      ds[0] = vs.x; ds[1] = vs.y; ds[2] = vs.z; ds[3] = vs.w;
    }
    float cz[4], sz[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * m + q;
      const float csj = S.csl[j * 32 + lane];
      cos_sin(csj * w[j], cz[q], sz[q]);
      const float dz = fmaf(-sz[q], dc[q], cz[q] * ds[q]);
      if constexpr (PARAMS) S.dcs[j * 32 + lane] = fmaf(w[j], dz, S.dcs[j * 32 + lane]);
      w[j] = csj * dz;  // dh
    }
    if constexpr (FUSED && PARAMS) {
      if (valid && P.b.phi_out) {
        float* o = P.b.phi_out + n * F + 2ll * e * d + k0;
        *reinterpret_cast<float4*>(o) = make_float4(cz[0], cz[1], cz[2], cz[3]);
        *reinterpret_cast<float4*>(o + d) = make_float4(sz[0], sz[1], sz[2], sz[3]);
      }
    }
  }
  // ---- dw = H dh (A phase, then B phase) ----
  hreg<Y::maskA()>(w);
  if constexpr (L > 5) {
    store_A<L>(buf, g, lam, w);
    __syncwarp();
    load_B<L>(buf, g, lam, w);
  }
  hreg<Y::maskB()>(w);
  // ---- dG, dv = G dw, scatter du[pi(k)] = dv[k] ----
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if constexpr (PARAMS) S.dg[j * 32 + lane] = fmaf(S.vl[j * 32 + lane], w[j], S.dg[j * 32 + lane]);
    w[j] *= S.gl[j * 32 + lane];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) sts32(paddr[j], w[j]);
  __syncwarp();
  load_B<L>(buf, g, lam, w);
  // ---- du0 = H du ----
  hreg<Y::maskB()>(w);
  if constexpr (L > 5) {
    store_B<L>(buf, g, lam, w);
    __syncwarp();
    load_A<L>(buf, g, lam, w);
  }
  hreg<Y::maskA()>(w);
  apply_signs(w, bmask);
  __syncwarp();
}

template <int L, bool FUSED>
__global__ void __launch_bounds__(kBW * 32) k_bwd_params(const BwdLaunch P, int64_t nwarps) {
  using Y = Lay<L>;
  using BS = BShape<L>;
  constexpr int d = Y::d;
  extern __shared__ float4 sm4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdSmem<L>& S = reinterpret_cast<BwdSmem<L>*>(sm4)[warp];
  const int64_t wid = (int64_t)blockIdx.x * kBW + warp;
  if (wid >= nwarps) return;
  const int g = lane / Y::T, lam = lane % Y::T;
  const uint32_t buf_addr = smem_addr(S.buf);
  const FeatureArgs& a = P.b.f;
  const int e = (int)(wid / P.wpe), sub = (int)(wid % P.wpe);
  const int64_t tiles = (a.n + BS::SPI - 1) / BS::SPI;
  const int64_t t0 = tiles * sub / P.wpe, t1 = tiles * (sub + 1) / P.wpe;
  uint32_t bmask;
  uint32_t paddr[32];
  load_tables<L>(a, e, g, lam, lane, buf_addr, S, bmask, paddr);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    S.dcs[j * 32 + lane] = 0.f;
    S.dg[j * 32 + lane] = 0.f;
  }
  for (int64_t t = t0; t < t1; ++t) {
    for (int r = 0; r < BS::R; ++r) {
      const int64_t n = t * BS::SPI + r * BS::VPW + g;
      const bool valid = n < a.n;
      float w[32];
      // An invalid sample contributes exactly zero: x-hat = 0 gives h = 0,
      // and its upstream gradient is read as 0 (dphi) or dlogits = 0.
      bwd_core<L, FUSED, true>(P, n, e, valid, g, lam, lane, S, bmask, paddr, w);
    }
  }
  // Sum the warp's sample groups (lanes with equal lam) and write the row.
  float* pr = P.partials + wid * 2 * d;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float s1 = S.dcs[j * 32 + lane], s2 = S.dg[j * 32 + lane];
#pragma unroll
    for (int o = Y::T; o < 32; o <<= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (g == 0) {
      pr[Y::kA(lam, j)] = s1;
      pr[d + Y::kB(lam, j)] = s2;
    }
  }
}

template <int L, bool FUSED>
__global__ void __launch_bounds__(kBW * 32) k_bwd_input(const BwdLaunch P) {
  using Y = Lay<L>;
  using BS = BShape<L>;
  extern __shared__ float4 sm4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdSmem<L>& S = reinterpret_cast<BwdSmem<L>*>(sm4)[warp];
  const int g = lane / Y::T, lam = lane % Y::T;
  const uint32_t buf_addr = smem_addr(S.buf);
  const FeatureArgs& a = P.b.f;
  const int64_t steps = (a.n + BS::VPW - 1) / BS::VPW;
  for (int64_t st = (int64_t)blockIdx.x * kBW + warp; st < steps;
       st += (int64_t)gridDim.x * kBW) {
    const int64_t n = st * BS::VPW + g;
    const bool valid = n < a.n;
    float dx[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) dx[j] = 0.f;
    for (int e = 0; e < a.E; ++e) {
      uint32_t bmask;
      uint32_t paddr[32];
      __syncwarp();
      load_tables<L>(a, e, g, lam, lane, buf_addr, S, bmask, paddr);
      __syncwarp();
      float w[32];
      bwd_core<L, FUSED, false>(P, n, e, valid, g, lam, lane, S, bmask, paddr, w);
#pragma unroll
      for (int j = 0; j < 32; ++j) dx[j] += w[j];
    }
    if (valid) {
      float* row = P.b.dx + n * a.ldx;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int k = Y::kA(lam, j);
        if (k < a.in_dim) row[k] = dx[j];
      }
    }
  }
}

// dCs[e][k] = sum over the expansion's warps of row 0; dG likewise row 1.
__global__ void k_reduce_params(const float* __restrict__ partials, int64_t d, int E, int wpe,
                                float* __restrict__ dCs, float* __restrict__ dG) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d * E) return;
  const int64_t e = t / d, k = t % d;
  float s1 = 0.f, s2 = 0.f;
  for (int q = 0; q < wpe; ++q) {
    const float* pr = partials + ((e * wpe + q) * 2) * d;
    s1 += pr[k];
    s2 += pr[d + k];
  }
  if (dCs) dCs[t] = s1;
  if (dG) dG[t] = s2;
}

// dW[c][f] = sum_n dlogits[n][c] phi[n][f]. A block owns 32 consecutive
// columns; its 8 warps take the rows n = w, w + 8, ... (one column per lane,
// coalesced 128-byte row segments) and the 8 partial sums are added in warp
// order through shared memory, so the result does not depend on scheduling.
constexpr int kWgRowGroups = 8;

__global__ void __launch_bounds__(32 * kWgRowGroups) k_weight_grads(const float* __restrict__ dl,
                                                                   const float* __restrict__ phi,
                                                                   int64_t n, int C, int64_t F,
                                                                   float* __restrict__ dW) {
  __shared__ float part[kWgRowGroups][CMAX][32];
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int64_t f = (int64_t)blockIdx.x * 32 + lane;
  float acc[CMAX];
#pragma unroll
  for (int c = 0; c < CMAX; ++c) acc[c] = 0.f;
  if (f < F) {
    for (int64_t i = rg; i < n; i += kWgRowGroups) {
      const float p = phi[i * F + f];
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) acc[c] = fmaf(__ldg(dl + i * C + c), p, acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < CMAX; ++c) part[rg][c][lane] = acc[c];
  __syncthreads();
  if (rg == 0 && f < F) {
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
      if (c < C) {
        float t = 0.f;
        for (int q = 0; q < kWgRowGroups; ++q) t += part[q][c][lane];
        dW[c * F + f] = t;
      }
    }
  }
}

__global__ void k_bias_grads(const float* __restrict__ dl, int64_t n, int C, float* __restrict__ db) {
  const int c = threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int64_t i = 0; i < n; ++i) s += dl[i * C + c];
  db[c] = s;
}

template <int L, bool FUSED>
cudaError_t run_bwd(const BwdLaunch& P0, int64_t num_partials, cudaStream_t s) {
  BwdLaunch P = P0;
  const FeatureArgs& a = P.b.f;
  const size_t smem = sizeof(BwdSmem<L>) * kBW;
  cudaError_t err;
  if (P.b.dCs || P.b.dG || P.b.phi_out) {
    err = cudaFuncSetAttribute(k_bwd_params<L, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    P.wpe = (int)(num_partials / a.E);
    const unsigned grid = (unsigned)((num_partials + kBW - 1) / kBW);
    k_bwd_params<L, FUSED><<<grid, kBW * 32, smem, s>>>(P, num_partials);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (P.b.dCs || P.b.dG) {
      const int64_t total = (int64_t)a.E << L;
      k_reduce_params<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
          P.partials, (int64_t)1 << L, a.E, P.wpe, P.b.dCs, P.b.dG);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
  }
  if (P.b.dx) {
    err = cudaFuncSetAttribute(k_bwd_input<L, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bwd_input<L, FUSED>, kBW * 32, smem) !=
        cudaSuccess)
      occ = 1;
    occ = std::max(occ, 1);
    const int64_t steps = (a.n + BShape<L>::VPW - 1) / BShape<L>::VPW;
    const int64_t need = (steps + kBW - 1) / kBW;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)a.num_sms * occ));
    k_bwd_input<L, FUSED><<<grid, kBW * 32, smem, s>>>(P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <bool FUSED>
cudaError_t dispatch_bwd(const BwdLaunch& P, int64_t num_partials, cudaStream_t s) {
  switch (P.b.f.L) {
    case 5: return run_bwd<5, FUSED>(P, num_partials, s);
    case 6: return run_bwd<6, FUSED>(P, num_partials, s);
    case 7: return run_bwd<7, FUSED>(P, num_partials, s);
    case 8: return run_bwd<8, FUSED>(P, num_partials, s);
    case 9: return run_bwd<9, FUSED>(P, num_partials, s);
    case 10: return run_bwd<10, FUSED>(P, num_partials, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_softmax_xent(const float* logits, const int32_t* labels, int64_t n, int C,
                                float* loss, float* dlogits, cudaStream_t s) {
  k_softmax_xent<<<1, 1024, 0, s>>>(logits, labels, n, C, loss, dlogits);
  return cudaGetLastError();
}

cudaError_t launch_backward(const BackwardArgs& b, float* partials, int64_t num_partials,
                            cudaStream_t s) {
  if (b.f.n == 0) return cudaSuccess;
  BwdLaunch P{};
  P.b = b;
  P.vec_x = (b.f.in_dim % 4 == 0) && (b.f.ldx % 4 == 0) &&
            (reinterpret_cast<uintptr_t>(b.f.x) % 16 == 0);
  P.partials = partials;
  return b.W ? dispatch_bwd<true>(P, num_partials, s) : dispatch_bwd<false>(P, num_partials, s);
}

cudaError_t launch_logit_weight_grads(const float* dlogits, const float* phi, int64_t n, int C,
                                      int64_t F, float* dW, float* db, cudaStream_t s) {
  if (dW) {
    k_weight_grads<<<(unsigned)((F + 31) / 32), 32 * kWgRowGroups, 0, s>>>(dlogits, phi, n, C, F, dW);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (db) {
    k_bias_grads<<<1, 32, 0, s>>>(dlogits, n, C, db);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace mck
