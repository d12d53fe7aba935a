// Fused Fastfood features at d = 1024 with both Walsh-Hadamard transforms on
// the tensor cores (Eq. etn:mckernel, Eq. etn:mcfeatures):
//
//   u = H (B_e x-hat);  v = Pi_e u;  h = H (G_e v);  phi = [cos | sin](Cs_e h)
//
// Each H is the Kronecker factorisation H_4 (x) H_16 (x) H_16 of mma_h16.cuh:
// two H16 digits as mma.m16n8k16 products (bf16 or fp16 operands, FP32
// accumulation, optionally with the hi + lo split of the data operand) and the
// last two index bits as FP32 butterflies, all in registers (8 x 8 transposes
// with movmatrix), so the only shared-memory traffic is the Pi gather: u is
// stored in the skewed slot (register j of lane lam at word base[lam] + 33 j,
// bases annealed at plan time for this layout) and gathered straight into the
// second product's operand order (mma_layout.h). The data operand is scaled
// per row by a power of two (exact) so that its largest magnitude lies in
// [2^10, 2^11): the 16-bit operands and the first digit's sums stay inside
// fp16's range, and the split keeps about 22 bits of every value relative to
// the row's largest. The scales come off before z = Cs h.
//
// Same work items as the FP32 warp kernel: one warp per block, a work item is
// (4-row tile, expansion), expansions fastest; the expansion's tables (B mask,
// G in input order, Cs in output order, packed gather offsets, slot bases) are
// loaded once per item. The 16-bit products round differently from FP32
// butterflies, so outputs match the oracle to the tolerance the tests state,
// not the FP32 kernel bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "mma_h16.cuh"
#include "mma_layout.h"

namespace mck {
namespace {

using namespace h16;

constexpr int kR = 4;  // rows per work item (tables loaded once per item)

struct MmaLaunch {
  FeatureArgs a;
  float* phi;
  bool vec_x;  // rows 8-byte aligned with even in_dim and ldx: float2 loads
};

// Power of two s with max |v| s in [2^10, 2^11) (1 for an all-zero row).
__device__ __forceinline__ float row_scale(const float (&v)[4][8]) {
  float m = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 8; ++i) m = fmaxf(m, fabsf(v[q][i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (m == 0.f) return 1.f;
  const int ex = ((__float_as_int(m) >> 23) & 0xff) - 127;  // floor(log2 m); -127 if subnormal
  const int se = min(max(127 + 10 - ex, 1), 254);
  return __int_as_float(se << 23);
}

__device__ __forceinline__ void scale_all(float (&v)[4][8], float s) {
  const float2 s2 = make_float2(s, s);
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      const float2 p = mul2(make_float2(v[q][i], v[q][i + 1]), s2);
      v[q][i] = p.x;
      v[q][i + 1] = p.y;
    }
}

// 16 resident single-warp blocks per SM (128 registers; up to 72 bytes of
// spills in the split forms): measured on the 60000-row, E = 16 batch against
// 12 blocks at 168 registers without spills, fp16 hi/lo 2.43 -> 2.33 ms,
// bf16 hi/lo 2.49 -> 2.29, unsplit 2.12 -> 1.96 ms.
template <int PREC, bool SPLIT>
__global__ void __launch_bounds__(32, 16) k_feat_mma(const MmaLaunch P) {
  constexpr int d = 1024;
  __shared__ __align__(16) float slot[Lay<10>::SLOT];
  const int lane = threadIdx.x;
  const int g = lane >> 2, t = lane & 3;
  const uint32_t sbase = smem_addr(slot);
  const int E = P.a.E;
  const int64_t F = 2ll * E * d;
  const int64_t tiles = (P.a.n + kR - 1) / kR;
  const int64_t items = tiles * E;
  const int64_t it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
  uint32_t hb[4];
  h16_operand<PREC>(g, t, hb);

  uint32_t bmask = 0, ubase = 0;
  uint32_t poff[16];
  float gt[32], cs[32];
  int cur_e = -1;
  for (int64_t it = it0; it < it1; ++it) {
    const int64_t tile = it / E;
    const int e = (int)(it % E);
    if (e != cur_e) {
      cur_e = e;
      const int64_t off = (int64_t)e * d;
      bmask = __ldg(P.a.mmaMask + (int64_t)e * 32 + lane);
      ubase = __ldg(P.a.mmaBase + (int64_t)e * 32 + lane);
      const uint4* pb = reinterpret_cast<const uint4*>(P.a.mmaPerm + off / 2) + lane;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 v = __ldg(pb + q * 32);
        poff[4 * q] = v.x;
        poff[4 * q + 1] = v.y;
        poff[4 * q + 2] = v.z;
        poff[4 * q + 3] = v.w;
      }
      if (P.a.mmaG) {  // the plan's G, lane-ordered in input order
        const float4* gp = reinterpret_cast<const float4*>(P.a.mmaG + off) + lane;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float4 v = __ldg(gp + m * 32);
          gt[4 * m] = v.x;
          gt[4 * m + 1] = v.y;
          gt[4 * m + 2] = v.z;
          gt[4 * m + 3] = v.w;
        }
      } else {  // caller-supplied G, natural order
#pragma unroll
        for (int j = 0; j < 32; ++j) gt[j] = __ldg(P.a.G + off + mma_in(lane, j));
      }
      if (P.a.mmaCs) {  // the plan's Cs, lane-ordered in output order
        const float4* cp = reinterpret_cast<const float4*>(P.a.mmaCs + off) + lane;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float4 v = __ldg(cp + m * 32);
          cs[4 * m] = v.x;
          cs[4 * m + 1] = v.y;
          cs[4 * m + 2] = v.z;
          cs[4 * m + 3] = v.w;
        }
      } else {  // caller-supplied Cs, natural order
#pragma unroll
        for (int j = 0; j < 32; ++j) cs[j] = __ldg(P.a.Cs + off + mma_out(lane, j));
      }
    }
    for (int r = 0; r < kR; ++r) {
      const int64_t n = tile * kR + r;
      if (n >= P.a.n) break;  // uniform over the warp
      const float* xr = P.a.x + n * P.a.ldx;
      // x-hat in input order (register j = 8 q + i of tile q), signs B applied
      float v[4][8];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          const int k0 = mma_in(lane, 8 * q + i);  // k0 + 1 is register i + 1
          float2 p = make_float2(0.f, 0.f);
          if (P.vec_x) {
            if (k0 < P.a.in_dim) p = __ldg(reinterpret_cast<const float2*>(xr + k0));
          } else {
            if (k0 < P.a.in_dim) p.x = __ldg(xr + k0);
            if (k0 + 1 < P.a.in_dim) p.y = __ldg(xr + k0 + 1);
          }
          v[q][i] = p.x;
          v[q][i + 1] = p.y;
        }
      if (r + 1 < kR && n + 1 < P.a.n && (int64_t)lane * 32 < P.a.in_dim)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(xr + P.a.ldx + lane * 32));
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float& w = v[j >> 3][j & 7];
        w = __int_as_float(__float_as_int(w) ^ ((bmask << (31 - j)) & 0x80000000u));
      }
      // u = H B x-hat, scaled by s1
      const float s1 = row_scale(v);
      scale_all(v, s1);
      chunk_transform<10, PREC, SPLIT>(v, hb);
      // v = Pi u: u to the skewed slot (output order), gathered into input order
      __syncwarp();  // the previous row's gather is done with the slot
      {
        float* q = slot + ubase;
#pragma unroll
        for (int j = 0; j < 32; ++j) q[33 * j] = v[j >> 3][j & 7];
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 32; ++j)
        v[j >> 3][j & 7] =
            lds32(sbase + ((j & 1) ? (poff[j >> 1] >> 16) : (poff[j >> 1] & 0xffffu)));
      // w = G v, rescaled by s2; h = H w
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const float2 p = mul2(make_float2(gt[j], gt[j + 1]),
                              make_float2(v[j >> 3][j & 7], v[j >> 3][(j & 7) + 1]));
        v[j >> 3][j & 7] = p.x;
        v[j >> 3][(j & 7) + 1] = p.y;
      }
      const float s2 = row_scale(v);
      scale_all(v, s2);
      chunk_transform<10, PREC, SPLIT>(v, hb);
      // z = Cs h with the scales removed (exact powers of two); [cos | sin]
      scale_all(v, (1.f / s1) * (1.f / s2));
      float* o = P.phi + n * F + 2ll * e * d;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        float c[4], sn[4];
        const float hq[4] = {v[j >> 3][j & 7], v[j >> 3][(j & 7) + 1], v[j >> 3][(j & 7) + 2],
                             v[j >> 3][(j & 7) + 3]};
        cos_sin4(&cs[j], hq, c, sn);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int k = mma_out(lane, j + i);
          __stcs(o + k, c[i]);
          __stcs(o + d + k, sn[i]);
        }
      }
    }
  }
}

template <int PREC, bool SPLIT>
cudaError_t run(const MmaLaunch& P, cudaStream_t s) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_feat_mma<PREC, SPLIT>, 32, 0) !=
      cudaSuccess)
    occ = 1;
  occ = std::max(occ, 1);
  const int64_t items = (P.a.n + kR - 1) / kR * P.a.E;
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)P.a.num_sms * occ));
  k_feat_mma<PREC, SPLIT><<<grid, 32, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_features_mma(const FeatureArgs& a, float* phi, int prec, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.L != 10 || !a.mmaPerm) return cudaErrorInvalidValue;
  MmaLaunch P{a, phi,
              (a.in_dim % 2 == 0) && (a.ldx % 2 == 0) && (reinterpret_cast<uintptr_t>(a.x) % 8 == 0)};
  switch (prec) {
    case MCK_BF16: return run<MCK_BF16, false>(P, s);
    case MCK_FP16: return run<MCK_FP16, false>(P, s);
    case MCK_BF16_SPLIT: return run<MCK_BF16, true>(P, s);
    case MCK_FP16_SPLIT: return run<MCK_FP16, true>(P, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mck
