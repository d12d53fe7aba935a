// Training-side kernels: the softmax cross-entropy of Sec. "Empirical
// Analysis" (the multi-class form of the logistic loss, Eq. etn:loss) and the
// adjoint of the Fastfood feature map, which Sec. "Empirical Analysis"
// motivates (the calibration C and the Gaussian G are trained by backpropagation).
//
// The adjoint recomputes the forward and runs the chain rule backwards,
// using H^T = H (Sylvester H is symmetric) and Pi^T = Pi^{-1} (the gather
// becomes a scatter to the same addresses):
//   dz  = -sin z dphi_cos + cos z dphi_sin
//   dCs += h dz            dh = Cs dz         dw = H dh
//   dG  += v dw            dv = G dw          du[pi(k)] = dv[k]      du0 = H du
//   dx  += (B du0)[:in_dim]
//   dB  += x-hat du0       (B read as a real diagonal; optional)
// Two kernels share that per-sample core:
//   k_bwd_params  a block of 8 warps per (expansion, range of samples): G_e,
//                 Cs_e (and, fused, W_e or the block's dphi rows) staged in
//                 shared memory; per-warp running sums of h dz and v dw
//                 (and x-hat B du0 for dB), added over the warps in order
//                 into one partial row per block; k_reduce_params sums the
//                 rows of each expansion in order.
//   k_bwd_input   each warp owns samples and loops over all expansions,
//                 accumulating dx in registers (no cross-warp sum needed).
// With fused logits the upstream gradient is dphi = W^T dlogits, formed
// from W (at d = 1024 for 8 rows at a time by the whole block);
// k_bwd_params then also writes the recomputed features so k_weight_grads
// can form dW = dlogits^T phi and db = sum dlogits in one launch.
// All sums run in a fixed order, so results are bit-reproducible.
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace mck {
namespace {

namespace cg = cooperative_groups;

constexpr int kBW = 1;         // warps per block
constexpr int kBwdMinBlocks = 12;  // resident single-warp blocks per SM the registers must allow
constexpr int kBwdInputMinBlocks = 8;  // k_bwd_input keeps dx in registers as well
constexpr int CMAX = MCK_MAX_CLASSES;

// ---------------------------------------------------------------------------
// Softmax cross-entropy: one block; thread i takes rows i, i + 1024, ...; the
// loss is summed in FP64 in a fixed order (lanes by a shuffle tree, then the
// warps in order), so it is bit-reproducible.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_softmax_xent(const float* __restrict__ logits,
                                                       const int32_t* __restrict__ labels,
                                                       int64_t n, int C, float* __restrict__ loss,
                                                       float* __restrict__ dlogits) {
  __shared__ double red[32];
  double acc = 0.0;
  const float inv_n = n > 0 ? 1.0f / (float)n : 0.f;
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
      for (int c = 0; c < C; ++c) {
        const float p = expf(l[c] - lse);
        dlogits[i * C + c] = ok ? (p - (c == y ? 1.f : 0.f)) * inv_n : 0.f;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *loss = n > 0 ? (float)(t / (double)n) : 0.f;
  }
}

// ---------------------------------------------------------------------------
// Backward core.
// ---------------------------------------------------------------------------
template <int L>
struct BShape {
  static constexpr int T = Lay<L>::T;
  static constexpr int VPW = 32 / T;  // samples a warp holds at once
};

struct BwdLaunch {
  BackwardArgs b;
  bool vec_x;
  float* partials;  // [E][bpe][2][d]
  int bpe;          // blocks per expansion (k_bwd_params)
  bool w_smem;      // k_bwd_params stages W_e in shared memory
  bool d_tile;      // k_bwd_params forms dphi for kBP rows at a time in shared memory (d = 1024)
};

__device__ __forceinline__ void apply_signs(float (&w)[32], uint32_t mask) {
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = __int_as_float(__float_as_int(w[j]) ^ ((mask << (31 - j)) & 0x80000000u));
}

// Per-lane arrays in shared memory hold a lane's 32 values as 8 float4s,
// float4 m of lane l at index m * 32 + l: private to the lane, and a warp's
// 128-bit accesses are conflict free.
__device__ __forceinline__ float4& lane4(float* a, int m, int lane) {
  return reinterpret_cast<float4*>(a)[m * 32 + lane];
}

// Per-warp shared state of the backward kernels. Only k_bwd_params keeps the
// sample's v and the running sums.
template <int L, bool PARAMS>
struct BwdSmem {
  alignas(16) float buf[BShape<L>::VPW * Lay<L>::SLOT];
  alignas(16) float vl[PARAMS ? 32 * 32 : 4];   // v = Pi u of the current sample, layout B
  alignas(16) float dcs[PARAMS ? 32 * 32 : 4];  // running sum of h dz, layout A
  alignas(16) float dg[PARAMS ? 32 * 32 : 4];   // running sum of v dw, layout B
  alignas(16) float dl[BShape<L>::VPW * CMAX];  // dlogits of the warp's current samples (fused)
};

// Where bwd_core finds G_e, Cs_e and W_e: per-lane copies in shared memory
// ([j][lane], shared by the block's warps, which all work on expansion e) and
// W_e's 2d columns per class (stride 2d), or else global memory.
struct BwdTabs {
  float* gl;   // per-lane G in layout B, or null: read G from global
  float* csl;  // per-lane Cs in layout A, or null: read Cs from global
  uint32_t ws;       // shared address of W_e (C x 2d), or 0: read W from global
  uint32_t dt;       // shared address of the sample's dphi row (2d), formed by the block, or 0
};

// Tables of expansion e held in registers for the warp's samples: B as a bit
// mask over layout A, Pi as byte offsets into the vector slot (packed two per
// register; the gather reads and the adjoint's scatter writes them).
template <int L>
__device__ __forceinline__ void load_tables(const FeatureArgs& a, int e, int lam, uint32_t& bmask,
                                            uint32_t (&poff)[16]) {
  using Y = Lay<L>;
  const int64_t off = (int64_t)e * Y::d;
  bmask = __ldg(a.maskA + (int64_t)e * Y::T + lam);
  const uint4* pb = reinterpret_cast<const uint4*>(a.permB + off) + lam;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint4 v = __ldg(pb + m * Y::T);
    poff[2 * m] = v.x | (v.y << 16);
    poff[2 * m + 1] = v.z | (v.w << 16);
  }
}

__device__ __forceinline__ uint32_t poff_of(const uint32_t (&poff)[16], int j) {
  return (j & 1) ? (poff[j >> 1] >> 16) : (poff[j >> 1] & 0xffffu);
}

__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

// G_e in layout B: from the block's shared copy, the plan's lane-ordered
// copy, or an overriding G.
template <int L>
__device__ __forceinline__ void load_G_B(const FeatureArgs& a, const BwdTabs& tb, int e, int lam,
                                         float (&gt)[32]) {
  using Y = Lay<L>;
  const int lane = threadIdx.x & 31;
  const int64_t off = (int64_t)e * Y::d;
  if (tb.gl) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 v = lane4(tb.gl, m, lane);
      gt[4 * m] = v.x;
      gt[4 * m + 1] = v.y;
      gt[4 * m + 2] = v.z;
      gt[4 * m + 3] = v.w;
    }
  } else if (a.GB) {
    const float4* gb = reinterpret_cast<const float4*>(a.GB + off) + lam;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 v = __ldg(gb + m * Y::T);
      gt[4 * m] = v.x;
      gt[4 * m + 1] = v.y;
      gt[4 * m + 2] = v.z;
      gt[4 * m + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) gt[j] = __ldg(a.G + off + Y::kB(lam, j));
  }
}

// x-hat of sample n in layout A (zero past in_dim, and for an invalid sample).
template <int L>
__device__ __forceinline__ void load_x_A(const BwdLaunch& P, int64_t n, bool valid, int lam,
                                         float (&w)[32]) {
  using Y = Lay<L>;
  const FeatureArgs& a = P.b.f;
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

// One sample of one expansion: forward recompute and backward. On return w
// holds B du0 (layout A), the sample's contribution to dx-hat.
template <int L, bool FUSED, bool PARAMS>
__device__ __forceinline__ void bwd_core(const BwdLaunch& P, const BwdTabs& tb, int64_t n, int e,
                                         bool valid, int g, int lam, BwdSmem<L, PARAMS>& S,
                                         uint32_t slot, uint32_t bmask,
                                         const uint32_t (&poff)[16], float (&w)[32]) {
  using Y = Lay<L>;
  constexpr int d = Y::d;
  const FeatureArgs& a = P.b.f;
  const int64_t F = 2ll * a.E * d;
  const int64_t off = (int64_t)e * d;
  const int lane = threadIdx.x & 31;
  float* buf = S.buf;
  // ---- forward: u = H B x-hat, v = Pi u, h = H G v ----
  load_x_A<L>(P, n, valid, lam, w);
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
  {
    float gt[32];
    load_G_B<L>(a, tb, e, lam, gt);
#pragma unroll
    for (int j = 0; j < 32; ++j) w[j] = lds32(slot + poff_of(poff, j));
    if constexpr (PARAMS) {
#pragma unroll
      for (int m = 0; m < 8; ++m)
        lane4(S.vl, m, lane) = make_float4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]);
    }
    hreg_scaled<Y::maskB()>(w, gt);
  }
  __syncwarp();
  if constexpr (L > 5) {
    store_B<L>(buf, g, lam, w);
    __syncwarp();
    load_A<L>(buf, g, lam, w);
  }
  hreg<Y::maskA()>(w);  // w = h, layout A
  // ---- dz from the upstream gradient ----
  // dphi for the lane's elements: from memory, or formed as W_e^T dlogits
  // class by class (64 accumulators, one dlogits value per class).
  float dc[32], ds[32];
  if (FUSED && tb.dt) {  // the row the block formed in shared memory
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint32_t at = tb.dt + 4u * (uint32_t)Y::kA(lam, 4 * m);
      const float4 vc = lds128(at), vs = lds128(at + 4u * d);
      dc[4 * m] = vc.x; dc[4 * m + 1] = vc.y; dc[4 * m + 2] = vc.z; dc[4 * m + 3] = vc.w;
      ds[4 * m] = vs.x; ds[4 * m + 1] = vs.y; ds[4 * m + 2] = vs.z; ds[4 * m + 3] = vs.w;
    }
  } else if constexpr (FUSED) {
    for (int c = lam; c < P.b.C; c += Y::T)  // dlogits of sample n, shared by its group's lanes
      S.dl[g * CMAX + c] = valid ? __ldg(P.b.dlogits + n * P.b.C + c) : 0.f;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) dc[j] = ds[j] = 0.f;
    const float* wr = P.b.W + 2ll * e * d;
#pragma unroll 1
    for (int c = 0; c < P.b.C; ++c) {
      const float dlc = S.dl[g * CMAX + c];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k0 = Y::kA(lam, 4 * m);
        float4 wc, ws;
        if (tb.ws) {
          const uint32_t wa = tb.ws + 4u * (uint32_t)(c * 2 * d + k0);
          wc = lds128(wa);
          ws = lds128(wa + 4u * d);
        } else {
          wc = __ldg(reinterpret_cast<const float4*>(wr + c * F + k0));
          ws = __ldg(reinterpret_cast<const float4*>(wr + c * F + d + k0));
        }
        dc[4 * m] = fmaf(dlc, wc.x, dc[4 * m]);
        dc[4 * m + 1] = fmaf(dlc, wc.y, dc[4 * m + 1]);
        dc[4 * m + 2] = fmaf(dlc, wc.z, dc[4 * m + 2]);
        dc[4 * m + 3] = fmaf(dlc, wc.w, dc[4 * m + 3]);
        ds[4 * m] = fmaf(dlc, ws.x, ds[4 * m]);
        ds[4 * m + 1] = fmaf(dlc, ws.y, ds[4 * m + 1]);
        ds[4 * m + 2] = fmaf(dlc, ws.z, ds[4 * m + 2]);
        ds[4 * m + 3] = fmaf(dlc, ws.w, ds[4 * m + 3]);
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k0 = Y::kA(lam, 4 * m);
      float4 vc = make_float4(0.f, 0.f, 0.f, 0.f), vs = vc;
      if (valid) {
        const float* gr = P.b.dphi + n * F + 2ll * e * d + k0;
        vc = __ldg(reinterpret_cast<const float4*>(gr));
        vs = __ldg(reinterpret_cast<const float4*>(gr + d));
      }
      dc[4 * m] = vc.x; dc[4 * m + 1] = vc.y; dc[4 * m + 2] = vc.z; dc[4 * m + 3] = vc.w;
      ds[4 * m] = vs.x; ds[4 * m + 1] = vs.y; ds[4 * m + 2] = vs.z; ds[4 * m + 3] = vs.w;
    }
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Y::kA(lam, 4 * m);
    float csq[4];
    if (tb.csl) {
      const float4 c4 = lane4(tb.csl, m, lane);
      csq[0] = c4.x; csq[1] = c4.y; csq[2] = c4.z; csq[3] = c4.w;
    } else {
      const float4 c4 = __ldg(reinterpret_cast<const float4*>(a.Cs + off + k0));
      csq[0] = c4.x; csq[1] = c4.y; csq[2] = c4.z; csq[3] = c4.w;
    }
    float cz[4], sz[4], hz[4];
    cos_sin4(csq, &w[4 * m], cz, sz);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * m + q;
      const float dz = fmaf(-sz[q], dc[j], cz[q] * ds[j]);
      hz[q] = w[j] * dz;
      w[j] = csq[q] * dz;  // dh
    }
    if constexpr (PARAMS) {
      float4& acc = lane4(S.dcs, m, lane);
      float4 t = acc;
      t.x += hz[0]; t.y += hz[1]; t.z += hz[2]; t.w += hz[3];
      acc = t;
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
  {
    float gt[32];
    load_G_B<L>(a, tb, e, lam, gt);
    if constexpr (PARAMS) {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4 v = lane4(S.vl, m, lane);
        float4& acc = lane4(S.dg, m, lane);
        float4 t = acc;
        t.x = fmaf(v.x, w[4 * m], t.x);
        t.y = fmaf(v.y, w[4 * m + 1], t.y);
        t.z = fmaf(v.z, w[4 * m + 2], t.z);
        t.w = fmaf(v.w, w[4 * m + 3], t.w);
        acc = t;
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) w[j] *= gt[j];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) sts32(slot + poff_of(poff, j), w[j]);
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

// dCs and dG partial sums. Block (e, sb) of kBP warps works on expansion e:
// it stages G_e and Cs_e per lane (and W_e, when it fits) in shared memory;
// warp q takes sample units (groups of VPW samples) [U q / W, U (q+1) / W) of
// the W = bpe * kBP warps of e; at the end the warps' sums are added in warp
// order and the block writes one partial row (E x bpe rows in all).
constexpr int kBP = 8;  // warps per block of k_bwd_params

template <int L, bool DB>
struct BwdBlockSmem {
  alignas(16) float gl[32 * 32];
  alignas(16) float csl[32 * 32];
  BwdSmem<L, true> warp[kBP];
  alignas(16) float db[DB ? kBP * 32 * 32 : 4];  // per-warp running sums of x-hat B du0, layout A
  // followed by W_e (C x 2d floats) when staged
};

// dB: x-hat (B du0) of the sample just processed, added to the warp's sums
// (B is applied once, when the block writes its row: x-hat du0 = B x-hat (B du0)).
template <int L>
__device__ __forceinline__ void add_db(const BwdLaunch& P, int64_t n, bool valid, int lam,
                                       float* dbw, const float (&w)[32]) {
  const int lane = threadIdx.x & 31;
  float xv[32];
  load_x_A<L>(P, n, valid, lam, xv);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    float4& acc = lane4(dbw, m, lane);
    float4 t = acc;
    t.x = fmaf(xv[4 * m], w[4 * m], t.x);
    t.y = fmaf(xv[4 * m + 1], w[4 * m + 1], t.y);
    t.z = fmaf(xv[4 * m + 2], w[4 * m + 2], t.z);
    t.w = fmaf(xv[4 * m + 3], w[4 * m + 3], t.w);
    acc = t;
  }
}

template <int L, bool FUSED, bool DB>
__global__ void __launch_bounds__(kBP * 32, 1) k_bwd_params(const BwdLaunch P) {
  using Y = Lay<L>;
  using BS = BShape<L>;
  constexpr int d = Y::d;
  constexpr int rows = DB ? 3 : 2;  // partial rows per block: dCs, dG (, dB)
  extern __shared__ float4 sm4[];
  BwdBlockSmem<L, DB>& B = *reinterpret_cast<BwdBlockSmem<L, DB>*>(sm4);
  float* Wsm = reinterpret_cast<float*>(&B + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdSmem<L, true>& S = B.warp[warp];
  const int g = lane / Y::T, lam = lane % Y::T;
  const uint32_t slot = smem_addr(S.buf) + 4u * (uint32_t)(g * Y::SLOT);
  const FeatureArgs& a = P.b.f;
  const int e = (int)(blockIdx.x / P.bpe), sb = (int)(blockIdx.x % P.bpe);
  const int64_t off = (int64_t)e * d;
  // ---- stage the expansion's tables ----
  if (warp == 0) {
    float gt[32];
    const BwdTabs none{nullptr, nullptr, 0u, 0u};  // read G from global
    load_G_B<L>(a, none, e, lam, gt);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      lane4(B.gl, m, lane) = make_float4(gt[4 * m], gt[4 * m + 1], gt[4 * m + 2], gt[4 * m + 3]);
      lane4(B.csl, m, lane) =
          __ldg(reinterpret_cast<const float4*>(a.Cs + off + Y::kA(lam, 4 * m)));
    }
  }
  if (FUSED && P.w_smem && !P.d_tile) {
    const int64_t F = 2ll * a.E * d;
    const int per_class4 = 2 * d / 4;
    for (int i = threadIdx.x; i < P.b.C * per_class4; i += blockDim.x) {
      const int c = i / per_class4, f4 = i % per_class4;
      reinterpret_cast<float4*>(Wsm)[i] =
          __ldg(reinterpret_cast<const float4*>(P.b.W + c * F + 2ll * e * d) + f4);
    }
  }
  BwdTabs tb{B.gl, B.csl, (FUSED && P.w_smem && !P.d_tile) ? smem_addr(Wsm) : 0u, 0u};
  uint32_t bmask;
  uint32_t poff[16];
  load_tables<L>(a, e, lam, bmask, poff);
  float* dbw = B.db + (DB ? warp * 32 * 32 : 0);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    lane4(S.dcs, m, lane) = make_float4(0.f, 0.f, 0.f, 0.f);
    lane4(S.dg, m, lane) = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (DB) lane4(dbw, m, lane) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  if constexpr (FUSED && L == 10) {
    if (P.d_tile) {
      // The block walks its rows kBP at a time, warp w taking row r0 + w. Per
      // tile the 256 threads first form dphi = dlogits W_e for all kBP rows
      // (thread t owns float4 columns t and t + 256: its weights are loaded
      // once per tile and used for every row), then each warp runs its row.
      float* dtile = Wsm;                 // [kBP][2d]
      float* dls = dtile + kBP * 2 * d;   // [kBP][CMAX]
      const int C = P.b.C;
      const int64_t F = 2ll * a.E * d;
      const float* We = P.b.W + 2ll * e * d;
      const int64_t n0 = a.n * sb / P.bpe, n1 = a.n * (sb + 1) / P.bpe;
      tb.dt = smem_addr(dtile + warp * 2 * d);
      for (int64_t r0 = n0; r0 < n1; r0 += kBP) {
        for (int i = threadIdx.x; i < kBP * CMAX; i += blockDim.x) {
          const int r = i / CMAX, c = i % CMAX;
          dls[i] = (c < C && r0 + r < n1) ? __ldg(P.b.dlogits + (r0 + r) * C + c) : 0.f;
        }
        __syncthreads();  // dlogits staged; the previous tile's rows are done with dtile
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int q4 = threadIdx.x + h * (kBP * 32);  // float4 column of 2d / 4 = 512
          float4 wv[CMAX];
#pragma unroll
          for (int c = 0; c < CMAX; ++c)
            wv[c] = c < C ? __ldg(reinterpret_cast<const float4*>(We + c * F) + q4)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int r = 0; r < kBP; ++r) {
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c4 = 0; c4 < CMAX / 4; ++c4) {
              const float4 g4 = reinterpret_cast<const float4*>(dls + r * CMAX)[c4];
              const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const int c = 4 * c4 + qq;
                if (c < C) {
                  t.x = fmaf(gv[qq], wv[c].x, t.x);
                  t.y = fmaf(gv[qq], wv[c].y, t.y);
                  t.z = fmaf(gv[qq], wv[c].z, t.z);
                  t.w = fmaf(gv[qq], wv[c].w, t.w);
                }
              }
            }
            reinterpret_cast<float4*>(dtile + r * 2 * d)[q4] = t;
          }
        }
        __syncthreads();  // the tile's dphi rows are complete
        const int64_t n = r0 + warp;
        float w[32];
        // a row past the block's range has x-hat = 0 and dphi = 0: it adds nothing
        bwd_core<L, FUSED, true>(P, tb, n, e, n < n1, g, lam, S, slot, bmask, poff, w);
        if constexpr (DB) add_db<L>(P, n, n < n1, lam, dbw, w);
      }
    }
  }
  if (!(FUSED && L == 10 && P.d_tile)) {
    const int64_t units = (a.n + BS::VPW - 1) / BS::VPW;
    const int64_t nw = (int64_t)P.bpe * kBP, q = (int64_t)sb * kBP + warp;
    const int64_t u0 = units * q / nw, u1 = units * (q + 1) / nw;
    for (int64_t u = u0; u < u1; ++u) {
      const int64_t n = u * BS::VPW + g;
      const bool valid = n < a.n;
      float w[32];
      // An invalid sample contributes exactly zero: x-hat = 0 gives h = 0,
      // and its upstream gradient is read as 0 (dphi) or dlogits = 0.
      bwd_core<L, FUSED, true>(P, tb, n, e, valid, g, lam, S, slot, bmask, poff, w);
      if constexpr (DB) add_db<L>(P, n, valid, lam, dbw, w);
    }
  }
  // Sum the warp's sample groups (lanes with equal lam) into lanes of group 0,
  // then the block's warps in order, and write the block's row.
  // (element j of a lane sits at word (j / 4 * 32 + lane) * 4 + j % 4)
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int at = ((j >> 2) * 32 + lane) * 4 + (j & 3);
    float s1 = S.dcs[at], s2 = S.dg[at], s3 = DB ? dbw[at] : 0.f;
#pragma unroll
    for (int o = Y::T; o < 32; o <<= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if constexpr (DB) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
    S.dcs[at] = s1;
    S.dg[at] = s2;
    if constexpr (DB) dbw[at] = s3;
  }
  __syncthreads();
  float* pr = P.partials + ((int64_t)e * P.bpe + sb) * rows * d;
  for (int j = warp; j < 32; j += kBP) {
    const int at = ((j >> 2) * 32 + lane) * 4 + (j & 3);
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int w2 = 0; w2 < kBP; ++w2) {
      s1 += B.warp[w2].dcs[at];
      s2 += B.warp[w2].dg[at];
      if constexpr (DB) s3 += B.db[w2 * 32 * 32 + at];
    }
    if (g == 0) {
      pr[Y::kA(lam, j)] = s1;
      pr[d + Y::kB(lam, j)] = s2;
      if constexpr (DB) pr[2 * d + Y::kA(lam, j)] = ((bmask >> j) & 1u) ? -s3 : s3;
    }
  }
}

template <int L, bool FUSED>
__global__ void __launch_bounds__(kBW * 32, kBwdInputMinBlocks) k_bwd_input(const BwdLaunch P) {
  using Y = Lay<L>;
  using BS = BShape<L>;
  extern __shared__ float4 sm4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BwdSmem<L, false>& S = reinterpret_cast<BwdSmem<L, false>*>(sm4)[warp];
  const int g = lane / Y::T, lam = lane % Y::T;
  const uint32_t slot = smem_addr(S.buf) + 4u * (uint32_t)(g * Y::SLOT);
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
      uint32_t poff[16];
      load_tables<L>(a, e, lam, bmask, poff);
      float w[32];
      const BwdTabs tb{nullptr, nullptr, 0u, 0u};
      bwd_core<L, FUSED, false>(P, tb, n, e, valid, g, lam, S, slot, bmask, poff, w);
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

// dCs[e][k] = sum over the expansion's partial rows of row 0; dG likewise
// row 1, and dB row 2 (rows = 3). A block owns 64 consecutive k of one
// expansion: thread (qg, c4) adds the partial rows q = qg, qg + 16, ... of
// float4 column c4 in order, and the 16 groups are then added in order
// through shared memory.
constexpr int kRpCols = 16, kRpGroups = 16;  // float4 columns x row groups per block

__global__ void __launch_bounds__(kRpCols * kRpGroups) k_reduce_params(
    const float* __restrict__ partials, int64_t d, int E, int rpe, int rows,
    float* __restrict__ dCs, float* __restrict__ dG, float* __restrict__ dB) {
  __shared__ float4 red[3][kRpGroups][kRpCols];
  const int c4 = threadIdx.x % kRpCols, qg = threadIdx.x / kRpCols;
  const int cols = d / 4 < kRpCols ? (int)(d / 4) : kRpCols;  // d = 32 has 8 float4 columns
  const int64_t blocks_per_e = d / (4 * cols);
  const int64_t e = blockIdx.x / blocks_per_e;
  const int64_t k = (blockIdx.x % blocks_per_e) * 4 * cols + 4 * c4;
  const bool on = c4 < cols;
  const float4* base = reinterpret_cast<const float4*>(partials + e * rpe * rows * d + k);
  const int64_t stride = rows * d / 4;  // float4s between consecutive partial rows
  float4 s[3];
  for (int r = 0; r < 3; ++r) s[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = qg; on && q < rpe; q += kRpGroups) {
    for (int r = 0; r < rows; ++r) {
      const float4 a = __ldg(base + q * stride + r * (d / 4));
      s[r].x += a.x; s[r].y += a.y; s[r].z += a.z; s[r].w += a.w;
    }
  }
  for (int r = 0; r < 3; ++r) red[r][qg][c4] = s[r];
  __syncthreads();
  if (qg < rows && on) {  // group 0 finishes dCs, group 1 dG, group 2 dB
    float4 t = red[qg][0][c4];
    for (int q = 1; q < kRpGroups; ++q) {
      const float4 v = red[qg][q][c4];
      t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
    }
    float* o = qg == 0 ? dCs : (qg == 1 ? dG : dB);  // may be only 4-byte aligned
    if (o) {
      o += e * d + k;
      o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
  }
}

// dW[c][f] = sum_n dlogits[n][c] phi[n][f]. A block owns 128 consecutive
// columns (a float4 per lane) and one of RS contiguous row ranges; the RS
// blocks of a column range form a thread-block cluster. In a block the 8
// warps take the rows r = w, w + 8, ... of its range, eight rows' loads in
// flight per warp, with dlogits staged in shared memory a chunk of rows at a
// time (rows padded to a multiple of 4 classes for 128-bit reads). Per class,
// each block adds its 8 warp sums in warp order, and the cluster's rank 0
// adds the RS block sums in rank order through distributed shared memory:
// the result does not depend on scheduling.
constexpr int kWgRowGroups = 8;
constexpr int kWgChunk = 256;  // rows of dlogits staged per pass

template <int C>
__global__ void __launch_bounds__(32 * kWgRowGroups, 2) k_weight_grads(const float* __restrict__ dl,
                                                                   const float* __restrict__ phi,
                                                                   int64_t n, int64_t F,
                                                                   float* __restrict__ dW,
                                                                   float* __restrict__ db) {
  constexpr int C4 = (C + 3) / 4 * 4;  // padded row of dlogits in shared memory
  constexpr int kWgUnroll = C <= 10 ? 16 : 8;  // rows in flight per warp (registers allowing)
  __shared__ float4 dls4[kWgChunk * C4 / 4];
  __shared__ float4 part[kWgRowGroups][32];
  __shared__ float4 bsum[C][32];
  __shared__ float4 bias4[C4 / 4];
  float* dls = reinterpret_cast<float*>(dls4);
  cg::cluster_group cluster = cg::this_cluster();
  const int RS = (int)gridDim.y, ry = (int)blockIdx.y;  // cluster = the RS blocks of a column
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int64_t f = ((int64_t)blockIdx.x * 32 + lane) * 4;  // F is a multiple of 4
  const bool active = dW && f < F;  // without dW only column block 0 runs, for db
  const int64_t rbeg = n * ry / RS, rend = n * (ry + 1) / RS;
  float4 acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fma_row = [&](const float4& p, const float* dr) {
#pragma unroll
    for (int c4 = 0; c4 < C4 / 4; ++c4) {
      const float4 g4 = reinterpret_cast<const float4*>(dr)[c4];
      const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 4 * c4 + q;
        if (c < C) {
          acc[c].x = fmaf(gv[q], p.x, acc[c].x);
          acc[c].y = fmaf(gv[q], p.y, acc[c].y);
          acc[c].z = fmaf(gv[q], p.z, acc[c].z);
          acc[c].w = fmaf(gv[q], p.w, acc[c].w);
        }
      }
    }
  };
  float4 bacc = make_float4(0.f, 0.f, 0.f, 0.f);  // column block 0: db partial sums
  for (int64_t r0 = rbeg; r0 < rend; r0 += kWgChunk) {
    const int rows = (int)((rend - r0) < kWgChunk ? (rend - r0) : kWgChunk);
    __syncthreads();  // the previous chunk is consumed
    {  // all of a thread's loads first, then the stores (one latency, not C4)
      static_assert(kWgChunk == 32 * kWgRowGroups, "one padded row per thread and pass");
      float v[C4];
#pragma unroll
      for (int k = 0; k < C4; ++k) {
        const int i = threadIdx.x + k * kWgChunk, r = i / C4, c = i % C4;
        v[k] = (r < rows && c < C) ? __ldg(dl + (r0 + r) * C + c) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < C4; ++k) dls[threadIdx.x + k * kWgChunk] = v[k];
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < C4 / 4) {  // db: this range's rows, in order
#pragma unroll 8
      for (int r = 0; r < rows; ++r) {
        const float4 g4 = dls4[r * (C4 / 4) + threadIdx.x];
        bacc.x += g4.x; bacc.y += g4.y; bacc.z += g4.z; bacc.w += g4.w;
      }
    }
    if (!active) continue;
    int i = rg;
    for (; i + (kWgUnroll - 1) * kWgRowGroups < rows; i += kWgUnroll * kWgRowGroups) {
      float4 p[kWgUnroll];
#pragma unroll
      for (int u = 0; u < kWgUnroll; ++u)
        p[u] = __ldg(reinterpret_cast<const float4*>(phi + (r0 + i + u * kWgRowGroups) * F + f));
#pragma unroll
      for (int u = 0; u < kWgUnroll; ++u) fma_row(p[u], dls + (i + u * kWgRowGroups) * C4);
    }
    for (; i < rows; i += kWgRowGroups)
      fma_row(__ldg(reinterpret_cast<const float4*>(phi + (r0 + i) * F + f)), dls + i * C4);
  }
  // Per class, warp 0 adds the 8 warp sums into bsum[c]; then, after one
  // cluster barrier, warp w of rank 0 adds classes w, w + 8 over the ranks.
#pragma unroll
  for (int c = 0; c < C; ++c) {
    part[rg][lane] = acc[c];
    __syncthreads();
    if (rg == 0) {
      float4 t = part[0][lane];
      for (int q = 1; q < kWgRowGroups; ++q) {
        const float4 v = part[q][lane];
        t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
      }
      bsum[c][lane] = t;
    }
    __syncthreads();  // part is free for the next class
  }
  if (blockIdx.x == 0 && threadIdx.x < C4 / 4) bias4[threadIdx.x] = bacc;
  cluster.sync();  // every block's sums are in place
  if (db && blockIdx.x == 0 && ry == 0 && threadIdx.x < C) {
    const int c = threadIdx.x;
    float t = reinterpret_cast<const float*>(bias4)[c];
    for (int q = 1; q < RS; ++q) t += reinterpret_cast<const float*>(cluster.map_shared_rank(bias4, q))[c];
    db[c] = t;
  }
  if (dW && ry == 0 && active) {
    for (int c = rg; c < C; c += kWgRowGroups) {
      float4 t = bsum[c][lane];
      for (int q = 1; q < RS; ++q) {
        const float4 v = cluster.map_shared_rank(&bsum[0][0], q)[c * 32 + lane];
        t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
      }
      float* o = dW + c * F + f;  // dW may be only 4-byte aligned
      o[0] = t.x;
      o[1] = t.y;
      o[2] = t.z;
      o[3] = t.w;
    }
  }
  cluster.sync();  // no block leaves while rank 0 still reads its bsum
}

template <int C>
cudaError_t run_weight_grads(const float* dlogits, const float* phi, int64_t n, int64_t F,
                             float* dW, float* db, cudaStream_t s) {
  // Row ranges per column range: a power of two up to the portable cluster
  // size 8, doubled while the grid still fits in one wave of two blocks per
  // SM and every range keeps at least 128 rows.
  const int64_t cols = dW ? (F + 127) / 128 : 1;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
  int rs = 1;
  while (rs < 8 && cols * rs * 2 <= 2ll * sms && n / (2 * rs) >= 128) rs *= 2;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)cols, (unsigned)rs, 1);
  cfg.blockDim = dim3(32 * kWgRowGroups, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = (unsigned)rs;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err = cudaLaunchKernelEx(&cfg, k_weight_grads<C>, dlogits, phi, n, F, dW, db);
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

template <int L, bool FUSED, bool DB>
cudaError_t run_params(BwdLaunch& P, int64_t num_partials, cudaStream_t s) {
  const FeatureArgs& a = P.b.f;
  size_t smem_p = sizeof(BwdBlockSmem<L, DB>);
  const size_t wbytes = FUSED ? sizeof(float) * (size_t)P.b.C * 2 * ((size_t)1 << L) : 0;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    optin = 0;
  const size_t tbytes = sizeof(float) * (size_t)kBP * (2 * ((size_t)1 << L) + CMAX);
  P.d_tile = FUSED && L == 10 && smem_p + tbytes <= (size_t)optin;
  P.w_smem = FUSED && !P.d_tile && smem_p + wbytes <= (size_t)optin;
  if (P.d_tile) smem_p += tbytes;
  else if (P.w_smem) smem_p += wbytes;
  cudaError_t err = cudaFuncSetAttribute(k_bwd_params<L, FUSED, DB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
  if (err != cudaSuccess) return err;
  P.bpe = (int)(num_partials / a.E);
  k_bwd_params<L, FUSED, DB><<<(unsigned)num_partials, kBP * 32, smem_p, s>>>(P);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (P.b.dCs || P.b.dG || DB) {
    const int cols = std::min(kRpCols, (1 << L) / 4);
    const unsigned blocks = (unsigned)(((int64_t)a.E << L) / (4 * cols));
    k_reduce_params<<<blocks, kRpCols * kRpGroups, 0, s>>>(
        P.partials, (int64_t)1 << L, a.E, P.bpe, DB ? 3 : 2, P.b.dCs, P.b.dG, P.b.dB);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <int L, bool FUSED>
cudaError_t run_bwd(const BwdLaunch& P0, int64_t num_partials, cudaStream_t s) {
  BwdLaunch P = P0;
  const FeatureArgs& a = P.b.f;
  const size_t smem_i = sizeof(BwdSmem<L, false>) * kBW;
  cudaError_t err;
  if (P.b.dCs || P.b.dG || P.b.dB || P.b.phi_out) {
    err = P.b.dB ? run_params<L, FUSED, true>(P, num_partials, s)
                 : run_params<L, FUSED, false>(P, num_partials, s);
    if (err != cudaSuccess) return err;
  }
  if (P.b.dx) {
    err = cudaFuncSetAttribute(k_bwd_input<L, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_i);
    if (err != cudaSuccess) return err;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bwd_input<L, FUSED>, kBW * 32, smem_i) !=
        cudaSuccess)
      occ = 1;
    occ = std::max(occ, 1);
    const int64_t steps = (a.n + BShape<L>::VPW - 1) / BShape<L>::VPW;
    const int64_t need = (steps + kBW - 1) / kBW;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)a.num_sms * occ));
    k_bwd_input<L, FUSED><<<grid, kBW * 32, smem_i, s>>>(P);
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

int64_t backward_partials(int L, int64_t n, int E, int num_sms) {
  const int vpw = 32 >> (L - 5);
  const int64_t units = (n + vpw - 1) / vpw;
  int64_t bpe = num_sms / E;
  bpe = std::max<int64_t>(1, std::min<int64_t>(bpe, units / kBP));
  return bpe * E;
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
  if (!dW && !db) return cudaSuccess;
  switch (C) {
    case 1: return run_weight_grads<1>(dlogits, phi, n, F, dW, db, s);
    case 2: return run_weight_grads<2>(dlogits, phi, n, F, dW, db, s);
    case 3: return run_weight_grads<3>(dlogits, phi, n, F, dW, db, s);
    case 4: return run_weight_grads<4>(dlogits, phi, n, F, dW, db, s);
    case 5: return run_weight_grads<5>(dlogits, phi, n, F, dW, db, s);
    case 6: return run_weight_grads<6>(dlogits, phi, n, F, dW, db, s);
    case 7: return run_weight_grads<7>(dlogits, phi, n, F, dW, db, s);
    case 8: return run_weight_grads<8>(dlogits, phi, n, F, dW, db, s);
    case 9: return run_weight_grads<9>(dlogits, phi, n, F, dW, db, s);
    case 10: return run_weight_grads<10>(dlogits, phi, n, F, dW, db, s);
    case 11: return run_weight_grads<11>(dlogits, phi, n, F, dW, db, s);
    case 12: return run_weight_grads<12>(dlogits, phi, n, F, dW, db, s);
    case 13: return run_weight_grads<13>(dlogits, phi, n, F, dW, db, s);
    case 14: return run_weight_grads<14>(dlogits, phi, n, F, dW, db, s);
    case 15: return run_weight_grads<15>(dlogits, phi, n, F, dW, db, s);
    default: return run_weight_grads<16>(dlogits, phi, n, F, dW, db, s);
  }
}

}  // namespace mck
