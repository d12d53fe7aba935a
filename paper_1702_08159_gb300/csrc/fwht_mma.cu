// Walsh-Hadamard transform on tensor cores: the Kronecker factorisation
// H_1024 = H_4 (x) H_16 (x) H_16 (Sec. "Fast Walsh Hadamard": H_n is built from
// H_{n-1} by a Kronecker step, so any split of the index bits into digits
// factors H) with each H_16 digit applied as a bf16/fp16 matrix product with
// FP32 accumulation.
//
// A warp owns a chunk of 1024 consecutive floats, viewed as four 16 x 16
// tiles X_t[r][c] (element t*256 + 16 r + c). Stage 1 computes D_t = X_t H16
// (digit c) with mma.m16n8k16, X_t as the A operand and H16 (+-1, exact in
// both types) as the B operand. The accumulator fragment of a 16 x 16 result
// has the same lane layout as an A operand, so after rounding D_t to 16-bit
// and transposing each 8 x 8 block in registers (movmatrix.trans), stage 2
// computes E_t = D_t^T H16 = (H16 X_t H16)^T (digit r). Index bits 8 and 9
// (the tile index) are transformed with FP32 butterflies across the four
// tiles a lane holds at identical positions.
//
// Split precision: before each product the FP32 operand x is written as
// hi + lo with hi = round16(x), lo = round16(x - hi) and both halves are
// multiplied (two MMAs into one FP32 accumulator), which recovers ~16 more
// bits of the input; the +-1 operand is exact either way.
//
// d = 256, 512, 1024: one or more vectors per warp chunk. 2^11 <= d <= 2^15:
// a block of d/1024 warps per vector, the index bits above 10 in FP32 after a
// shared-memory exchange. Larger d: that on every 2^15 block, then FP32
// column passes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "mma_h16.cuh"

namespace mck {
namespace {

using namespace h16;

constexpr int kMmaWarps = 4;

__device__ __forceinline__ void load_chunk(const float* __restrict__ base, int g, int t,
                                           float (&v)[4][8]) {
#pragma unroll
  for (int tile = 0; tile < 4; ++tile)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float2 p = __ldcs(reinterpret_cast<const float2*>(
          base + tile * 256 + 16 * frag_row(r, g) + frag_col(r, t)));
      v[tile][2 * r] = p.x;
      v[tile][2 * r + 1] = p.y;
    }
}

template <int L, int PREC, bool SPLIT>
__global__ void __launch_bounds__(kMmaWarps * 32) k_fwht_mma(float* __restrict__ x,
                                                             int64_t chunks) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  uint32_t hb[4];
  h16_operand<PREC>(g, t, hb);
  for (int64_t ch = (int64_t)blockIdx.x * kMmaWarps + (threadIdx.x >> 5); ch < chunks;
       ch += (int64_t)gridDim.x * kMmaWarps) {
    float* base = x + ch * 1024;
    float v[4][8];
    load_chunk(base, g, t, v);
    chunk_transform<L, PREC, SPLIT>(v, hb);
    // The tile now holds E = Y^T (Y = H16 X H16): fragment (row, col) of E is
    // element 16*col + row of the chunk tile.
#pragma unroll
    for (int tile = 0; tile < 4; ++tile)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = frag_row(r, g), col = frag_col(r, t);
        __stcs(base + tile * 256 + 16 * col + row, v[tile][2 * r]);
        __stcs(base + tile * 256 + 16 * (col + 1) + row, v[tile][2 * r + 1]);
      }
  }
}

// One pass for 2^11 <= d <= 2^15: a block of W = d/1024 warps per vector.
// Warp w transforms chunk w (index bits 0..9) on the tensor cores and leaves
// it in shared memory (word i at i + 8 floor(i/32): the fragment stores fall
// on 32 distinct banks); after a barrier thread j takes columns c = j,
// j + 32W, ... (32/W of them) with their W values at stride 1024 and applies
// H_W over index bits 10..L-1 in FP32 registers on the way out to HBM.
__host__ __device__ __forceinline__ constexpr int mpad(int i) { return i + 8 * (i >> 5); }

template <int L, int PREC, bool SPLIT>
__global__ void __launch_bounds__(1 << (L - 5)) k_fwht_mma_cta(float* __restrict__ x, int64_t n) {
  constexpr int W = 1 << (L - 10), NT = 32 * W, CPT = 32 / W;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  uint32_t hb[4];
  h16_operand<PREC>(g, t, hb);
  for (int64_t vec = blockIdx.x; vec < n; vec += gridDim.x) {
    float* row = x + (vec << L);
    {
      float v[4][8];
      load_chunk(row + warp * 1024, g, t, v);
      chunk_transform<10, PREC, SPLIT>(v, hb);
#pragma unroll
      for (int tile = 0; tile < 4; ++tile)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = warp * 1024 + tile * 256 + 16 * frag_col(r, t) + frag_row(r, g);
          sm[mpad(i)] = v[tile][2 * r];
          sm[mpad(i + 16)] = v[tile][2 * r + 1];
        }
    }
    __syncthreads();
    // At 2^15 (one block per SM) the block's next vector goes into L2 while this
    // one is transformed, as in the FP32 block transform.
    if constexpr (L == 15)
      if (vec + gridDim.x < n && lane == 0)
        prefetch_l2_bulk(row + ((int64_t)gridDim.x << L) + warp * 1024, 4096u);
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int c = threadIdx.x + NT * j;
      float u[W];
#pragma unroll
      for (int i = 0; i < W; ++i) u[i] = sm[mpad(c + 1024 * i)];
#pragma unroll
      for (int h = 1; h < W; h <<= 1)
#pragma unroll
        for (int i = 0; i < W; ++i)
          if (!(i & h)) {
            const float a = u[i], b = u[i | h];
            u[i] = a + b;
            u[i | h] = a - b;
          }
#pragma unroll
      for (int i = 0; i < W; ++i) __stcs(row + c + 1024 * i, u[i]);
    }
    __syncthreads();  // the slice is read before the next vector overwrites it
  }
}

template <int L, int PREC, bool SPLIT>
cudaError_t run(float* x, int64_t chunks, int num_sms, cudaStream_t s) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fwht_mma<L, PREC, SPLIT>,
                                                    kMmaWarps * 32, 0) != cudaSuccess)
    occ = 1;
  occ = std::max(occ, 1);
  const int64_t need = (chunks + kMmaWarps - 1) / kMmaWarps;
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * occ));
  k_fwht_mma<L, PREC, SPLIT><<<grid, kMmaWarps * 32, 0, s>>>(x, chunks);
  return cudaGetLastError();
}

template <int L, int PREC, bool SPLIT>
cudaError_t run_cta(float* x, int64_t n, int num_sms, cudaStream_t s) {
  auto kern = k_fwht_mma_cta<L, PREC, SPLIT>;
  const size_t smem = sizeof(float) * (size_t)mpad(1 << L);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 1 << (L - 5), smem) != cudaSuccess)
    occ = 1;
  occ = std::max(occ, 1);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms * occ));
  kern<<<grid, 1 << (L - 5), smem, s>>>(x, n);
  return cudaGetLastError();
}

template <int L>
cudaError_t run_cta_prec(float* x, int64_t n, int prec, int num_sms, cudaStream_t s) {
  switch (prec) {
    case MCK_BF16: return run_cta<L, MCK_BF16, false>(x, n, num_sms, s);
    case MCK_FP16: return run_cta<L, MCK_FP16, false>(x, n, num_sms, s);
    case MCK_BF16_SPLIT: return run_cta<L, MCK_BF16, true>(x, n, num_sms, s);
    case MCK_FP16_SPLIT: return run_cta<L, MCK_FP16, true>(x, n, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int L>
cudaError_t run_prec(float* x, int64_t chunks, int prec, int num_sms, cudaStream_t s) {
  switch (prec) {
    case MCK_BF16: return run<L, MCK_BF16, false>(x, chunks, num_sms, s);
    case MCK_FP16: return run<L, MCK_FP16, false>(x, chunks, num_sms, s);
    case MCK_BF16_SPLIT: return run<L, MCK_BF16, true>(x, chunks, num_sms, s);
    case MCK_FP16_SPLIT: return run<L, MCK_FP16, true>(x, chunks, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool fwht_mma_supported(int L) { return L >= 8 && L <= 20; }

cudaError_t launch_fwht_mma(float* x, int64_t n, int L, int prec, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  // Vectors are packed into 1024-float chunks; n * 2^L is a multiple of 1024
  // whenever n is a multiple of 2^(10-L) (the caller checks).
  const int64_t chunks = (n << L) >> 10;
  switch (L) {
    case 8: return run_prec<8>(x, chunks, prec, num_sms, s);
    case 9: return run_prec<9>(x, chunks, prec, num_sms, s);
    default: break;
  }
  if (L == 10) return run_prec<10>(x, chunks, prec, num_sms, s);
  // 2^11 <= d <= 2^15: one pass, a block of d/1024 warps per vector (the
  // tensor cores on each 1024-float block, FP32 for index bits 10..L-1).
  switch (L) {
    case 11: return run_cta_prec<11>(x, n, prec, num_sms, s);
    case 12: return run_cta_prec<12>(x, n, prec, num_sms, s);
    case 13: return run_cta_prec<13>(x, n, prec, num_sms, s);
    case 14: return run_cta_prec<14>(x, n, prec, num_sms, s);
    case 15: return run_cta_prec<15>(x, n, prec, num_sms, s);
    default: break;
  }
  // d > 2^15: that pass on every 2^15 block, then an FP32 column pass over
  // index bits 15..L-1 (H_d = H_{d/2^15} (x) H_{2^15}).
  cudaError_t err = run_cta_prec<15>(x, n << (L - 15), prec, num_sms, s);
  if (err != cudaSuccess) return err;
  return launch_fwht_high_bits(x, n, L, num_sms, s);
}

}  // namespace mck
