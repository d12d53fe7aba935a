// Fused Fastfood features at 2^11 <= d <= 2^14 in the chunked block form
// (common.cuh): per sample n and expansion e, u = H (B_e x-hat),
// v = Pi_e u, z = Cs_e H (G_e v), phi = [cos z | sin z] (Eq. etn:mckernel,
// Eq. etn:mcfeatures), one block of 2^(L-10) warps per work item.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace mck {
namespace {

struct ChunkLaunch {
  FeatureArgs a;
  bool vec_x;  // x rows 16-byte aligned and in_dim % 4 == 0
  float* phi;  // n x 2Ed
};

// ---------------------------------------------------------------------------
// Chunked block kernel, 11 <= L <= 14 (features): one block of W = 2^(L-10)
// warps per work item, the chunked form described in common.cuh, with the
// chunk tables made at plan time (B mask, Pi word offsets packed two per
// register, G) and Cs read at the output. A work item is (tile of R rows,
// expansion), expansions fastest: the warps load their chunk's tables once
// and keep them in registers for the R rows (an expansion's tables are as
// large as a row's features at these d, so per-row reloads would cost about
// as much traffic through L1 as the output itself).
// ---------------------------------------------------------------------------
template <int L, int R>  // 16 warps per SM at 128 registers (measured best; 64 registers spill)
__global__ void __launch_bounds__(Chunked<L>::NT, 512 / Chunked<L>::NT) k_feat_chunks(const ChunkLaunch P) {
  constexpr int d = 1 << L;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int tid = threadIdx.x;
  const int E = P.a.E;
  const int64_t tiles = (P.a.n + R - 1) / R;
  const int64_t items = tiles * E;
  const float* Gov = P.a.GB ? nullptr : P.a.G;
  const int64_t F = 2ll * E * d;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t n0 = (it / E) * R;
    const int e = (int)(it % E);
    const int64_t eo = (int64_t)e * d;
    ChunkTabs t;
    load_chunk_tabs<L>(P.a.permB + eo, Gov ? nullptr : P.a.GB + eo, Gov ? Gov + eo : nullptr,
                       P.a.maskA + eo / 32, tid, t);
    for (int r = 0; r < R; ++r) {
      const int64_t n = n0 + r;
      if (n >= P.a.n) break;  // uniform over the block
      chunked_body<L, false>(t, P.a.x + n * P.a.ldx, P.a.in_dim, P.vec_x, P.a.Cs + eo,
                             P.phi + n * F + 2ll * e * d, sm, tid, [] { __syncthreads(); },
                             nullptr, nullptr, [] {});
    }
  }
}

// The same with the input staged: the block copies the next row's x-hat (its
// warps' chunks) and, once per item, the expansion's Cs into shared memory
// with cp.async, so neither load is waited for in a row's critical path (the
// block holds one row at a time and every warp starts it together). Needs
// 16-byte aligned rows with in_dim % 4 == 0 (vec_x); shared memory: the
// chunk slots plus 2 d floats. Used at d = 2^14.
template <int L, int R>
__global__ void __launch_bounds__(Chunked<L>::NT, 512 / Chunked<L>::NT)
    k_feat_chunks_staged(const ChunkLaunch P) {
  using C = Chunked<L>;
  constexpr int d = 1 << L;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* xs = sm + C::WORDS + warp * 1024;  // this warp's chunk of x-hat
  float* css = sm + C::WORDS + d;           // Cs of the item's expansion
  const int E = P.a.E;
  const int64_t tiles = (P.a.n + R - 1) / R;
  const int64_t items = tiles * E;
  const float* Gov = P.a.GB ? nullptr : P.a.G;
  const int64_t F = 2ll * E * d;
  // One commit group per call: the warp's chunk of row n (none past the end).
  auto copy_x = [&](int64_t n) {
    if (n >= 0) {
      const float* row = P.a.x + n * P.a.ldx;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int c = 4 * (lane + 32 * m);
        const int64_t k = (int64_t)warp * 1024 + c;
        const bool in = k < P.a.in_dim;
        cp_async16(smem_addr(xs + c), in ? row + k : row, in ? 16 : 0);
      }
    }
    cp_async_commit();
  };
  // The row after row r of item `it` in this block's order (-1: none).
  auto next_row = [&](int64_t it, int r) -> int64_t {
    const int64_t n = (it / E) * R + r + 1;
    if (r + 1 < R && n < P.a.n) return n;
    const int64_t it2 = it + gridDim.x;
    return it2 < items ? (it2 / E) * R : -1;
  };
  int64_t it = blockIdx.x;
  copy_x(it < items ? (it / E) * R : -1);
  for (; it < items; it += gridDim.x) {
    const int64_t n0 = (it / E) * R;
    const int e = (int)(it % E);
    const int64_t eo = (int64_t)e * d;
    ChunkTabs t;
    load_chunk_tabs<L>(P.a.permB + eo, Gov ? nullptr : P.a.GB + eo, Gov ? Gov + eo : nullptr,
                       P.a.maskA + eo / 32, tid, t);
    cp_async_wait<0>();  // this thread's copies of the first row's x-hat
    const float* cs = P.a.Cs + eo;
#pragma unroll
    for (int j = 0; j < d / (4 * C::NT); ++j) {
      const int q = 4 * (tid + C::NT * j);
      cp_async16(smem_addr(css + q), cs + q, 16);
    }
    cp_async_commit();
    for (int r = 0; r < R; ++r) {
      const int64_t n = n0 + r;
      if (n >= P.a.n) break;  // uniform over the block
      if (r > 0) cp_async_wait<0>();  // this row's x-hat (queued during the previous row)
      const int64_t nn = next_row(it, r);
      chunked_body<L, true>(t, nullptr, P.a.in_dim, true, nullptr, P.phi + n * F + 2ll * e * d, sm,
                            tid, [] { __syncthreads(); }, xs, css, [&] { copy_x(nn); });
    }
  }
  cp_async_wait<0>();
}

template <class K>
int occ_blocks(K kernel, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess)
    b = 1;
  return std::max(b, 1);
}

template <int L, int R>
cudaError_t run_chunks(const ChunkLaunch& P, bool staged, cudaStream_t s) {
  using C = Chunked<L>;
  const size_t smem_u = sizeof(float) * C::WORDS;
  const size_t smem_s = sizeof(float) * (C::WORDS + 2 * (1 << L));
  auto go = [&](auto kernel, size_t smem) -> cudaError_t {
    cudaError_t err =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int occ = occ_blocks(kernel, C::NT, smem);
    const int64_t items = (P.a.n + R - 1) / R * P.a.E;
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)P.a.num_sms * occ));
    kernel<<<grid, C::NT, smem, s>>>(P);
    return cudaGetLastError();
  };
  return staged ? go(k_feat_chunks_staged<L, R>, smem_s) : go(k_feat_chunks<L, R>, smem_u);
}

template <int L>
cudaError_t run_l(const ChunkLaunch& P, int rows, bool staged, cudaStream_t s) {
  switch (rows) {
    case 1: return run_chunks<L, 1>(P, staged, s);
    case 2: return run_chunks<L, 2>(P, staged, s);
    default: return run_chunks<L, 4>(P, staged, s);
  }
}

}  // namespace

cudaError_t launch_chunked_features(const FeatureArgs& a, bool vec_x, float* phi, cudaStream_t s) {
  ChunkLaunch P{a, vec_x, phi};
  // Automatic shape, from the autotuner's sweep on one GB300 (E = 4, 1 GiB of
  // features per d): staged items of 4 rows (tables kept in registers across
  // the rows, the next row's input and the item's Cs copied ahead) beat one
  // unstaged row per item by 2, 4, 5 and 12% at 2^11..2^14 (0.324 -> 0.317,
  // 0.341 -> 0.329, 0.390 -> 0.371, 0.493 -> 0.433 ms); unstaged, 4 rows
  // gain nothing. Batches with fewer than 8 four-row items per resident block
  // keep one row per item so every block gets work.
  const bool can_stage = vec_x && (reinterpret_cast<uintptr_t>(a.Cs) % 16) == 0;
  const bool staged = can_stage && (a.staged < 0 || a.staged == 1);
  int rows = a.rows_per_item;
  if (rows <= 0) {
    const int blocks_per_sm = std::max(1, 512 / (32 << (a.L - 10)));
    const int64_t items4 = (a.n + 3) / 4 * a.E;
    rows = staged && items4 >= 8ll * a.num_sms * blocks_per_sm ? 4 : 1;
  }
  switch (a.L) {
    case 11: return run_l<11>(P, rows, staged, s);
    case 12: return run_l<12>(P, rows, staged, s);
    case 13: return run_l<13>(P, rows, staged, s);
    case 14: return run_l<14>(P, rows, staged, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mck
