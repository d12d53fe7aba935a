// Tensor-core building blocks of the Kronecker-H16 transform, shared by the
// standalone transform (fwht_mma.cu) and the tensor-core feature kernel
// (features_mma.cu).
//
// A warp owns a chunk of 1024 floats, viewed as four 16 x 16 tiles X_t[r][c]
// (element t*256 + 16 r + c). Stage 1 computes D_t = X_t H16 (digit c) with
// mma.m16n8k16, X_t as the A operand and H16 (+-1, exact in both types) as the
// B operand. The accumulator fragment of a 16 x 16 result has the same lane
// layout as an A operand, so after rounding D_t to 16-bit and transposing each
// 8 x 8 block in registers (movmatrix.trans), stage 2 computes
// E_t = D_t^T H16 = (H16 X_t H16)^T (digit r). Index bits 8 and 9 (the tile
// index) are transformed with FP32 butterflies across the four tiles a lane
// holds at identical positions (H_1024 = H_4 (x) H_16 (x) H_16; Sec. "Fast Walsh
// Hadamard": each Kronecker step of the recursion is one digit).
//
// Split precision: before each product the FP32 operand x is written as
// hi + lo with hi = round16(x), lo = round16(x - hi) and both halves are
// multiplied (two MMAs into one FP32 accumulator), which recovers ~11 more
// bits of the input; the +-1 operand is exact either way.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mck.h"

namespace mck {
namespace h16 {

// Round two floats to a packed pair of 16-bit values (low half = a).
template <int PREC>
__device__ __forceinline__ uint32_t pack16(float a, float b) {
  if constexpr (PREC == MCK_BF16) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
  } else {
    const __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
}

template <int PREC>
__device__ __forceinline__ float2 unpack16(uint32_t u) {
  if constexpr (PREC == MCK_BF16) {
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(&u);
    return __bfloat1622float2(v);
  } else {
    const __half2 v = *reinterpret_cast<const __half2*>(&u);
    return __half22float2(v);
  }
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  if constexpr (PREC == MCK_BF16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

// d = A B with a zero accumulator (no running sum enters the product).
template <int PREC>
__device__ __forceinline__ void mma16816_zero(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                              uint32_t b1) {
  const float z = 0.f;
  if constexpr (PREC == MCK_BF16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(z));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(z));
  }
}

// The two products above as plain (non-volatile) asm: pure functions of their
// operands that the compiler may schedule among independent chains.
__device__ __forceinline__ void mma16816_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                             uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma16816_f16_zero(float (&d)[4], const uint32_t (&a)[4],
                                                  uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}

__device__ __forceinline__ uint32_t transpose8x8(uint32_t v) {
  uint32_t r;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(r) : "r"(v));
  return r;
}

// A-operand registers (hi and optionally lo) of one tile from 8 FP32 values in
// fragment order: value i sits at register i/2, half i%2.
template <int PREC, bool SPLIT>
__device__ __forceinline__ void to_operand(const float (&v)[8], uint32_t (&hi)[4],
                                           uint32_t (&lo)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    hi[r] = pack16<PREC>(v[2 * r], v[2 * r + 1]);
    if constexpr (SPLIT) {
      const float2 h = unpack16<PREC>(hi[r]);
      lo[r] = pack16<PREC>(v[2 * r] - h.x, v[2 * r + 1] - h.y);
    }
  }
}

// D = A H16 for one tile: two n-halves of 8 columns. Output in fragment order
// (the A layout): out[0..1] = (g, 2t..2t+1), out[2..3] = (g+8, 2t..),
// out[4..5] = (g, 8+2t..), out[6..7] = (g+8, 8+2t..).
template <int PREC, bool SPLIT>
__device__ __forceinline__ void times_h16(const uint32_t (&hi)[4], const uint32_t (&lo)[4],
                                          const uint32_t (&hb)[4], float (&out)[8]) {
  float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
  if constexpr (SPLIT) {
    mma16816<PREC>(c0, lo, hb[0], hb[1]);
    mma16816<PREC>(c1, lo, hb[2], hb[3]);
  }
  mma16816<PREC>(c0, hi, hb[0], hb[1]);
  mma16816<PREC>(c1, hi, hb[2], hb[3]);
  out[0] = c0[0];
  out[1] = c0[1];
  out[2] = c0[2];
  out[3] = c0[3];
  out[4] = c1[0];
  out[5] = c1[1];
  out[6] = c1[2];
  out[7] = c1[3];
}

// Register r of the fragment holds elements (row, col) = (g + 8*(r&1), 2t + 8*(r>>1) + {0,1}).
__device__ __forceinline__ int frag_row(int r, int g) { return g + 8 * (r & 1); }
__device__ __forceinline__ int frag_col(int r, int t) { return 2 * t + 8 * (r >> 1); }

// B operand of H16 for n-halves 0 and 1: H[k][n] = (-1)^popcount(k & n),
// k = 2t, 2t+1 (register 0) and 2t+8, 2t+9 (register 1), n = g (+8).
template <int PREC>
__device__ __forceinline__ void h16_operand(int g, int t, uint32_t (&hb)[4]) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int n = g + 8 * half;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int k0 = 2 * t + 8 * r;
      const float e0 = (__popc(k0 & n) & 1) ? -1.f : 1.f;
      const float e1 = (__popc((k0 + 1) & n) & 1) ? -1.f : 1.f;
      hb[2 * half + r] = pack16<PREC>(e0, e1);
    }
  }
}

// One warp transforms index bits 0..L-1 (L <= 10) of its 1024-float chunk
// held in v in fragment order: two H16 digits on the tensor cores, then bits
// 8 and 9 as FP32 butterflies. On return tile `tile`, fragment (row, col) of
// v holds chunk element tile*256 + 16*col + row.
template <int L, int PREC, bool SPLIT>
__device__ __forceinline__ void chunk_transform(float (&v)[4][8], const uint32_t (&hb)[4]) {
  // Stage 1: digit c (bits 0-3).
#pragma unroll
  for (int tile = 0; tile < 4; ++tile) {
    uint32_t hi[4], lo[4];
    to_operand<PREC, SPLIT>(v[tile], hi, lo);
    times_h16<PREC, SPLIT>(hi, lo, hb, v[tile]);
  }
  // Stage 2: transpose each tile (16-bit, per 8 x 8 block) and apply digit r (bits 4-7).
#pragma unroll
  for (int tile = 0; tile < 4; ++tile) {
    uint32_t hi[4], lo[4], hiT[4], loT[4];
    to_operand<PREC, SPLIT>(v[tile], hi, lo);
    hiT[0] = transpose8x8(hi[0]);
    hiT[1] = transpose8x8(hi[2]);
    hiT[2] = transpose8x8(hi[1]);
    hiT[3] = transpose8x8(hi[3]);
    if constexpr (SPLIT) {
      loT[0] = transpose8x8(lo[0]);
      loT[1] = transpose8x8(lo[2]);
      loT[2] = transpose8x8(lo[1]);
      loT[3] = transpose8x8(lo[3]);
    }
    times_h16<PREC, SPLIT>(hiT, loT, hb, v[tile]);
  }
  // Index bits 8 and 9 (which tile): FP32 butterflies within each vector.
  if constexpr (L >= 9) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a0 = v[0][i], a1 = v[1][i], a2 = v[2][i], a3 = v[3][i];
      v[0][i] = a0 + a1;
      v[1][i] = a0 - a1;
      v[2][i] = a2 + a3;
      v[3][i] = a2 - a3;
    }
  }
  if constexpr (L >= 10) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float a0 = v[0][i], a1 = v[1][i], a2 = v[2][i], a3 = v[3][i];
      v[0][i] = a0 + a2;
      v[2][i] = a0 - a2;
      v[1][i] = a1 + a3;
      v[3][i] = a1 - a3;
    }
  }
}


}  // namespace h16
}  // namespace mck
